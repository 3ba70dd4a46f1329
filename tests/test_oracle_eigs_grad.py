"""Pins for oracle.eigs (LOBPCG vs dense, closed forms) and oracle.grad (Hellmann-Feynman)."""
import numpy as np
import pytest

from oracle.eigs import lobpcg, eigs_dense
from oracle.grad import band_gradients, clusters
from oracle.lattice import make_lattice, with_kappa
from oracle.nfsep import bases
from small_lattices import named_small
from paper_1806_10284_gb300 import workloads as W

NAMED = named_small()


def _eps(lat, seed, contrast=12.0):
    rng = np.random.default_rng(seed)
    return np.stack([1.0 + contrast * (rng.random(lat.shape) < 0.35) for _ in range(3)])


@pytest.mark.parametrize("name", ["fcc64", "tri192", "mono80"])
def test_lobpcg_matches_dense(name):
    lat = NAMED[name]
    invB = 1.0 / _eps(lat, 4)
    ref, _ = eigs_dense(lat, invB, 8)
    lam, Y, it, res = lobpcg(lat, invB, 8, block=14, tol=1e-11, seed=1)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)
    assert np.all(res <= 1e-11)


def test_lobpcg_gamma_deflation():
    lat = with_kappa(NAMED["fcc64"], [0.0, 0.0, 0.0])
    invB = 1.0 / _eps(lat, 6)
    ref, _ = eigs_dense(lat, invB, 6)
    lam, *_ = lobpcg(lat, invB, 6, block=10, tol=1e-11, seed=2)
    assert ref[0] > 1e-3
    np.testing.assert_allclose(lam, ref, rtol=1e-10)


def test_lobpcg_homogeneous_closed_form():
    """B = c: eigenvalues are the smallest Lq / c (each twice), at a size beyond dense reach."""
    w = W.WORKLOADS["sc16"]
    lat = make_lattice(w["vectors"], w["n"], W.bloch_vectors("sc16")[0])
    c = 4.0
    invB = np.full((3,) + lat.shape, 1.0 / c)
    lam, *_ = lobpcg(lat, invB, 10, block=16, tol=1e-11, seed=3)
    ref = np.sort(np.concatenate([bases(lat)[3].ravel() ** 2] * 2))[:10] / c
    np.testing.assert_allclose(lam, ref, rtol=1e-10)


def test_scaling_of_eps():
    """B -> c B scales every eigenvalue by 1/c (A_r is homogeneous of degree -1 in B)."""
    lat = NAMED["hex96"]
    invB = 1.0 / _eps(lat, 8)
    l1, _ = eigs_dense(lat, invB, 5)
    l2, _ = eigs_dense(lat, invB / 3.0, 5)
    np.testing.assert_allclose(l2, l1 / 3.0, rtol=1e-12)


def test_euler_sum_rule():
    """sum_{l,v} B_l(v) d lambda / d B_l(v) = -lambda (Euler, degree -1 homogeneity)."""
    lat = NAMED["tri192"]
    B = _eps(lat, 10)
    lam, V = eigs_dense(lat, 1.0 / B, 6)
    G = band_gradients(lat, 1.0 / B, V, lam)
    for j in range(len(lam)):
        assert np.sum(B * G[j]) == pytest.approx(-lam[j], rel=1e-10)


def test_gradient_central_differences():
    """Central finite differences of a nondegenerate band, step 1e-4, several voxels."""
    lat = NAMED["fcc64"]
    B = _eps(lat, 12)
    lam, V = eigs_dense(lat, 1.0 / B, 6)
    G = band_gradients(lat, 1.0 / B, V, lam)
    groups = clusters(lam, 1e-8)
    j = next(g[0] for g in groups if len(g) == 1)
    rng = np.random.default_rng(0)
    h = 1e-4
    for _ in range(6):
        l, k, jj, i = (int(rng.integers(0, s)) for s in (3,) + lat.shape)
        Bp, Bm = B.copy(), B.copy()
        Bp[l, k, jj, i] += h
        Bm[l, k, jj, i] -= h
        fd = (eigs_dense(lat, 1.0 / Bp, 6)[0][j] - eigs_dense(lat, 1.0 / Bm, 6)[0][j]) / (2 * h)
        assert G[j, l, k, jj, i] == pytest.approx(fd, rel=2e-5, abs=1e-9 * lam[j])


def test_degenerate_cluster_mean():
    """Homogeneous B at a symmetric k gives exactly degenerate pairs; each member's gradient
    is the cluster mean, whose sum rule gives -lambda of the cluster."""
    w = W.WORKLOADS["sc16"]
    lat = make_lattice(w["vectors"], (4, 4, 4), np.array([0.3, 0.3, 0.3]))
    B = np.full((3,) + lat.shape, 2.0)
    lam, V = eigs_dense(lat, 1.0 / B, 6)
    groups = clusters(lam, 1e-8)
    assert any(len(g) > 1 for g in groups)
    G = band_gradients(lat, 1.0 / B, V, lam)
    for g in groups:
        for j in g:
            np.testing.assert_allclose(G[j], G[g[0]], atol=1e-14)
            assert np.sum(B * G[j]) == pytest.approx(-np.mean(lam[g]), rel=1e-10)
