"""Pins for oracle.lattice (Section 2.2) against hand-derived offsets and identities."""
import json
import math
import os

import numpy as np
import pytest

from oracle.lattice import make_lattice, paper_round, reciprocal, choose_order
from paper_1806_10284_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lattice_offsets.json")))


def test_paper_rounding_rule():
    # floor below 1/2, ceiling at and above 1/2 (Section 2.2, cases I and II)
    assert paper_round(2.0) == 2
    assert paper_round(2.4999999) == 2
    assert paper_round(2.5) == 3
    assert paper_round(2.75) == 3
    assert paper_round(0.0) == 0


@pytest.mark.parametrize("name", ["fcc64", "bcc96", "hex96", "sc16"])
def test_golden_offsets(name):
    g = GOLD[name]
    w = W.WORKLOADS[name]
    lat = make_lattice(w["vectors"], w["n"], W.bloch_vectors(name)[0])
    assert list(lat.perm) == g["perm"]
    assert [lat.m1, lat.m2, lat.m3] == g["m"]
    assert [lat.rho1, lat.rho2, lat.rho3] == g["rho"]
    assert [lat.s1, lat.s2, lat.s3] == g["s"]
    if "cos_alpha" in g:
        assert lat.cos_alpha == pytest.approx(g["cos_alpha"], abs=1e-14)
    if "kappa" in g:
        np.testing.assert_allclose(lat.kappa, g["kappa"], atol=1e-14)


@pytest.mark.parametrize("name", list(W.WORKLOADS))
def test_corrected_vectors_sit_on_grid(name):
    """eq. (transvec): lengths kept, a2 and a3 end on grid points with the index shifts s."""
    w = W.WORKLOADS[name]
    lat = make_lattice(w["vectors"], w["n"], np.zeros(3))
    a = lat.a
    v = np.asarray(w["vectors"])[list(lat.perm)]
    for l in range(3):
        assert np.linalg.norm(a[:, l]) == pytest.approx(np.linalg.norm(v[l]), rel=1e-13)
    assert a[0, 1] == pytest.approx(lat.s1 * lat.dx, abs=1e-13)
    assert a[0, 2] == pytest.approx(lat.s2 * lat.dx, abs=1e-13)
    assert a[1, 2] == pytest.approx(lat.s3 * lat.dy, abs=1e-13)
    assert a[1, 1] == pytest.approx(lat.n2 * lat.dy, rel=1e-14)
    assert a[2, 2] == pytest.approx(lat.n3 * lat.dz, rel=1e-14)
    # the angle correction keeps the offsets within the bounds stated in Section 2.2
    assert 0 <= lat.m1 <= lat.n1 and 0 <= lat.m2 <= lat.n1 and 0 <= lat.m3 <= lat.n2


def test_uncorrected_when_on_grid():
    """Section 2.2: theta = theta' when the offsets are already integers (BCC: cos = -1/3 exactly)."""
    w = W.WORKLOADS["bcc96"]
    lat = make_lattice(w["vectors"], w["n"], np.zeros(3))
    assert lat.cos_gamma == pytest.approx(-1.0 / 3.0, abs=1e-15)
    assert lat.cos_beta == pytest.approx(-1.0 / 3.0, abs=1e-15)
    assert lat.cos_alpha == pytest.approx(-1.0 / 3.0, abs=1e-14)


def test_reciprocal_duality():
    w = W.WORKLOADS["tri192"]
    lat = make_lattice(w["vectors"], (12, 10, 8), np.zeros(3))
    b = reciprocal(lat)
    np.testing.assert_allclose(lat.a.T @ b, 2 * math.pi * np.eye(3), atol=1e-12)


def test_kappa_is_reduced_coordinate():
    """kappa_l = k . a_l equals the reduced coordinate of 2 pi k in b~ (Section 2.3 map Omega)."""
    w = W.WORKLOADS["mono80"]
    c = np.array([0.11, -0.27, 0.4])
    K = W.bloch_from_reduced(w["vectors"], c)
    lat = make_lattice(w["vectors"], w["n"], K)
    np.testing.assert_allclose(lat.kappa, c[list(lat.perm)], atol=1e-13)


def test_degenerate_lattice_rejected():
    # coplanar vectors span no cell; for non-degenerate cells some ordering always meets the
    # Section 2.2 conditions, so only degenerate input is refused
    v = np.array([[1.0, 0, 0], [0.0, 0.8, 0], [0.3, 0.5, 0.0]])
    with pytest.raises(ValueError):
        make_lattice(v, (8, 8, 8), np.zeros(3))
    with pytest.raises(ValueError):
        choose_order(np.array([[1.0, 0, 0], [0.5, 0, 0], [0.2, 0.0, 0.0]]))
