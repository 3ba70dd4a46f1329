"""Pins for the extra workloads of the paper's Section 6 and 7 (the gyroid on the BCC
lattice, the permittivity sweep 3..30, supercells with a vacancy), checked with the
oracle's dense A_r against facts that hold exactly:

* a supercell of N_1 x N_2 x N_3 primitive cells with the permittivity repeated is
  the same periodic operator, so its spectrum at a Bloch vector K is the union of
  the primitive cell's spectra at K + sum_l (j_l / N_l) b_l (band folding);
* raising B pointwise lowers every eigenvalue of C^*C e = lambda B e (min-max: the
  Rayleigh quotient's denominator grows), so the sweep's bands fall monotonically;
* the gyroid sampler, which maps each Yee point through fractional coordinates,
  agrees with the rotation of the canonical frame back to the input frame.
"""
import math

import numpy as np
import pytest

from oracle.eigs import eigs_dense
from oracle.lattice import make_lattice
from oracle.nfsep import Ar_dense
from paper_1806_10284_gb300 import workloads as W


def _spectrum(lat, B):
    A = Ar_dense(lat, 1.0 / np.stack(B))
    return np.linalg.eigvalsh(0.5 * (A + A.conj().T))


def _geom(lat):
    return W.Geometry(n=(lat.n1, lat.n2, lat.n3), s=(lat.s1, lat.s2, lat.s3),
                      delta=(lat.dx, lat.dy, lat.dz), perm=tuple(lat.perm))


@pytest.mark.parametrize("reps", [(2, 1, 1), (2, 2, 1)])
def test_supercell_spectrum_is_the_folded_primitive_spectrum(reps):
    rng = np.random.default_rng(11)
    V, n = W.simple_cubic(), (4, 4, 4)
    K = W.bloch_from_reduced(V, [0.13, -0.21, 0.07])
    lat_p = make_lattice(V, n, K)
    B = [1.0 + 12.0 * (rng.random(lat_p.shape) < 0.4) for _ in range(3)]
    Vs, ns = W.supercell(V, n, reps)
    lat_s = make_lattice(Vs, ns, K)
    assert tuple(lat_s.perm) == (0, 1, 2) and (lat_s.s1, lat_s.s2, lat_s.s3) == (0, 0, 0)
    got = _spectrum(lat_s, W.tile_eps(B, reps))
    parts = []
    for j1 in range(reps[0]):
        for j2 in range(reps[1]):
            for j3 in range(reps[2]):
                shift = W.bloch_from_reduced(V, [j1 / reps[0], j2 / reps[1], j3 / reps[2]])
                parts.append(_spectrum(make_lattice(V, n, K + shift), B))
    ref = np.sort(np.concatenate(parts))
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * ref.max())


def test_vacancy_breaks_the_folding():
    """Removing one cell's inclusion changes the spectrum (the vacancy is really there)."""
    V, n, reps = W.simple_cubic(), (4, 4, 4), (2, 1, 1)
    K = W.bloch_from_reduced(V, [0.1, 0.2, 0.3])
    lat_p = make_lattice(V, n, K)
    B = W.sample_inclusions(_geom(lat_p), [dict(kind="sphere", center=np.full(3, 0.5), radius=0.3)], 13.0)
    Vs, ns = W.supercell(V, n, reps)
    lat_s = make_lattice(Vs, ns, K)
    full = W.tile_eps(B, reps)
    vac = W.tile_eps(B, reps, [(1, 0, 0)])
    assert np.all(vac[0][:, :, 4:] == 1.0) and np.array_equal(vac[0][:, :, :4], full[0][:, :, :4])
    assert np.max(np.abs(_spectrum(lat_s, vac) - _spectrum(lat_s, full))) > 1e-3


@pytest.mark.parametrize("name", ["fcc64", "tri192"])
def test_eigenvalues_fall_as_eps_grows(name):
    w = W.WORKLOADS[name]
    rng = np.random.default_rng(5)
    lat = make_lattice(w["vectors"], (4, 4, 4), W.bloch_from_reduced(w["vectors"], [0.2, 0.1, -0.3]))
    B = np.stack([1.0 + 12.0 * (rng.random(lat.shape) < 0.4) for _ in range(3)])
    lo = _spectrum(lat, B)
    hi = _spectrum(lat, B + rng.random(B.shape) * (rng.random(B.shape) < 0.5))
    assert np.all(hi <= lo * (1 + 1e-12))
    assert np.any(hi < lo * (1 - 1e-6))


def test_gyroid_sweep_bands_fall_monotonically():
    w = W.WORKLOADS["gyroid96"]
    lat = make_lattice(w["vectors"], (6, 6, 6), W.bloch_from_reduced(w["vectors"], w["reduced_k"][0]))
    prev = None
    for e in w["eps_sweep"]:
        lam, _ = eigs_dense(lat, 1.0 / np.stack(W.eps_for("gyroid96", _geom(lat), eps_in=e)), 10)
        if prev is not None:
            assert np.all(lam <= prev * (1 + 1e-12)), e
        prev = lam


def test_gyroid_sampler_matches_the_rotated_frame():
    """BCC at n = 24 sits on the grid without an angle correction, so the canonical
    frame is a rotation R of the input frame (A_c = R A_in): the gyroid evaluated at
    R^T X must give the sampler's mask at every Yee point X."""
    w = W.WORKLOADS["gyroid96"]
    lat = make_lattice(w["vectors"], (24, 24, 24), np.zeros(3))
    geom = _geom(lat)
    Ac = geom.lattice_matrix()
    Ain = np.asarray(w["vectors"], dtype=np.float64)[list(lat.perm)].T
    R = Ac @ np.linalg.inv(Ain)
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
    B = W.eps_for("gyroid96", geom)
    for comp in range(3):
        X = W.yee_points(geom, comp)
        Xin = np.tensordot(R.T, X, axes=(1, 0))
        ref = np.where(W.gyroid_value(Xin) > w["level"], w["eps_in"], 1.0)
        # points within rounding of the level set may fall either way
        near = np.abs(W.gyroid_value(Xin) - w["level"]) < 1e-9
        assert np.array_equal(B[comp][~near], ref[~near]), comp


def test_gyroid_fill_fraction():
    """The sampled fraction of eps_in equals the volume fraction of {G > 1.1} in the
    cubic cell (Monte Carlo), to the discretisation error of a 24^3 grid."""
    w = W.WORKLOADS["gyroid96"]
    lat = make_lattice(w["vectors"], (24, 24, 24), np.zeros(3))
    B = W.eps_for("gyroid96", _geom(lat))
    frac = np.mean([np.mean(b == w["eps_in"]) for b in B])
    rng = np.random.default_rng(2)
    mc = np.mean(W.gyroid_value(rng.random((3, 400000))) > w["level"])
    assert 0.02 < mc < 0.2
    assert abs(frac - mc) < 0.015, (frac, mc)
    # and the function itself: G(x + a/2 (-1, 1, 1)) = G(x), a BCC translation
    X = rng.random((3, 1000))
    np.testing.assert_allclose(W.gyroid_value(X + 0.5 * np.array([-1.0, 1.0, 1.0])[:, None]),
                               W.gyroid_value(X), atol=1e-12)
    assert math.isclose(float(W.gyroid_value(np.zeros((3, 1)))[0]), 0.0, abs_tol=1e-15)
