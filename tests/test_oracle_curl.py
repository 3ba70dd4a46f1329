"""Pins for oracle.curl (Section 3): wrap-built C vs the paper's printed matrices, CG = 0, rank."""
import numpy as np
import pytest

from oracle.curl import (difference_ops, paper_difference_ops, curl, gradient, wrap_index)
from small_lattices import category_cover, named_small, random_triclinics, j3_category

COVER = category_cover()
NAMED = named_small()


@pytest.mark.parametrize("idx", range(len(COVER)))
def test_wrap_matches_printed_K_forms(idx):
    """C1 = I (x) I (x) K1, C2 = I (x) K2 with eq. (J2), C3 = K3 with the four J3 categories."""
    lat = COVER[idx]
    ours = difference_ops(lat)
    paper = paper_difference_ops(lat)
    for l in range(3):
        np.testing.assert_allclose(ours[l].toarray(), paper[l], atol=1e-12,
                                   err_msg=f"C{l+1}, J3 category {j3_category(lat)}")


def test_category_cover_is_complete():
    assert sorted({j3_category(l) for l in COVER}) == [1, 2, 3, 4]


@pytest.mark.parametrize("name", sorted(NAMED))
def test_printed_J2_on_workload_lattices(name):
    lat = NAMED[name]
    ours = difference_ops(lat)
    paper = paper_difference_ops(lat)
    np.testing.assert_allclose(ours[0].toarray(), paper[0], atol=1e-12)
    np.testing.assert_allclose(ours[1].toarray(), paper[1], atol=1e-12)


def test_wrap_is_quasi_periodic():
    """eq. (quasi_periodic): moving by a lattice shift multiplies by e^{i 2 pi kappa_l}."""
    lat = COVER[0]
    shifts = [(lat.n1, 0, 0), (lat.s1, lat.n2, 0), (lat.s2, lat.s3, lat.n3)]
    for (i, j, k) in [(0, 0, 0), (2, 1, 1), (lat.n1 - 1, lat.n2 - 1, lat.n3 - 1)]:
        for l, sh in enumerate(shifts):
            ii, jj, kk, ph = wrap_index(lat, i + sh[0], j + sh[1], k + sh[2])
            assert (ii, jj, kk) == (i, j, k)
            assert ph == pytest.approx(np.exp(2j * np.pi * lat.kappa[l]), abs=1e-13)


@pytest.mark.parametrize("lat", list(NAMED.values()) + random_triclinics(3, 4, generic_only=False),
                         ids=lambda l: f"{l.n1}x{l.n2}x{l.n3}-m{l.m1}.{l.m2}.{l.m3}")
def test_curl_grad_zero_and_commute(lat):
    """C G = 0 (Section 5.1, null space of C^*C) because C1, C2, C3 commute."""
    ops = difference_ops(lat)
    C, G = curl(lat, ops), gradient(lat, ops)
    assert abs(C @ G).max() < 1e-9 * max(1.0, abs(C).max() ** 2)


@pytest.mark.parametrize("name", ["fcc64", "tri192", "hex96"])
def test_rank_of_curl(name):
    """Null space of C^*C has dimension n = one third of 3n (Section 1.3, Section 5.1)."""
    lat = NAMED[name]
    C = curl(lat).toarray()
    sv = np.linalg.svd(C, compute_uv=False)
    tol = 1e-9 * sv.max()
    assert int(np.sum(sv > tol)) == 2 * lat.n
