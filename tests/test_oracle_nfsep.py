"""Pins for oracle.nfsep (Section 5.1-5.2): Q unitary, C^*C Q = Q diag(Lq, Lq, 0), SVD of C,
spectrum of A_r = nonzero spectrum of the GEP, homogeneous closed form."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.curl import curl, difference_ops
from oracle.lattice import make_lattice, with_kappa
from oracle.nfsep import (bases, Qr_dense, Q0_dense, Ar_dense, apply_Ar, gep_nonzero_eigs,
                          expand, contract, G_TOL)
from oracle.spectral import lambdas
from small_lattices import category_cover, named_small
from paper_1806_10284_gb300 import workloads as W

NAMED = named_small()
COVER = category_cover()
SET = [NAMED["fcc64"], NAMED["tri192"], NAMED["hex96"], NAMED["mono80"], COVER[0], COVER[5]]


def _id(l):
    return f"{l.n1}x{l.n2}x{l.n3}-m{l.m1}.{l.m2}.{l.m3}"


def _random_eps(lat, seed):
    rng = np.random.default_rng(seed)
    return [1.0 + 12.0 * (rng.random(lat.shape) < 0.3) for _ in range(3)]


@pytest.mark.parametrize("lat", SET, ids=_id)
def test_Q_unitary(lat):
    """Q = [Q1 Q2 Q0] is unitary (Section 5.1, before eq. double_eigendecomposition)."""
    b = bases(lat)
    Q = np.concatenate([Qr_dense(lat, b), Q0_dense(lat, b)], axis=1)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(3 * lat.n), atol=1e-11)


@pytest.mark.parametrize("lat", SET, ids=_id)
def test_double_curl_eigendecomposition(lat):
    """C^*C Q1 = Q1 Lq, C^*C Q2 = Q2 Lq, C^*C Q0 = 0 (eqs. null_basis, range_basis1/2)."""
    b = bases(lat)
    C = curl(lat)
    A = (C.conj().T @ C).toarray()
    Qr, Q0 = Qr_dense(lat, b), Q0_dense(lat, b)
    Lq = np.concatenate([b[3].ravel() ** 2] * 2)
    scale = Lq.max()
    np.testing.assert_allclose(A @ Qr, Qr * Lq[None, :], atol=1e-10 * scale)
    np.testing.assert_allclose(A @ Q0, 0.0, atol=1e-10 * scale)


@pytest.mark.parametrize("lat", SET[:3], ids=_id)
def test_singular_values_of_curl(lat):
    """eq. (SVD): the singular values of C are Lq^{1/2}, each twice, and n zeros."""
    sv = np.sort(np.linalg.svd(curl(lat).toarray(), compute_uv=False))
    sigma = np.sort(np.concatenate([bases(lat)[3].ravel()] * 2 + [np.zeros(lat.n)]))
    np.testing.assert_allclose(sv, sigma, atol=1e-9 * sigma.max())


@pytest.mark.parametrize("lat", SET, ids=_id)
def test_Ar_spectrum_equals_gep(lat):
    """Theorem invariant_space / eq. NFSEP: eig(A_r) = nonzero eig of A x = lambda B x."""
    B = _random_eps(lat, 3)
    invB = np.stack([1.0 / x for x in B])
    C = curl(lat)
    A = (C.conj().T @ C).toarray()
    gep = gep_nonzero_eigs(A, np.concatenate([x.ravel() for x in B]))
    ar = np.sort(np.linalg.eigvalsh(0.5 * (Ar_dense(lat, invB) + Ar_dense(lat, invB).conj().T)))
    assert len(gep) == 2 * lat.n
    np.testing.assert_allclose(ar, gep, rtol=1e-9, atol=1e-9 * gep.max())


@pytest.mark.parametrize("lat", SET, ids=_id)
def test_fft_apply_matches_dense(lat, rng):
    """A_r y through Algorithms 5.2/5.1 equals the dense Sigma_r Q_r^* B^{-1} Q_r Sigma_r y."""
    B = _random_eps(lat, 5)
    invB = np.stack([1.0 / x for x in B])
    y = rng.standard_normal(2 * lat.n) + 1j * rng.standard_normal(2 * lat.n)
    got = apply_Ar(lat, y.reshape((2,) + lat.shape), invB).ravel()
    np.testing.assert_allclose(got, Ar_dense(lat, invB) @ y, atol=1e-10 * np.abs(got).max())


def test_homogeneous_closed_form(rng):
    """B = c I: A_r = Sigma_r^2 / c, so A_r y = (Lq / c) y exactly (eq. SVD, eq. NFSEP)."""
    w = W.WORKLOADS["tri192"]
    lat = make_lattice(w["vectors"], (12, 10, 8), W.bloch_vectors("tri192")[0])
    c = 7.5
    invB = np.full((3,) + lat.shape, 1.0 / c)
    y = rng.standard_normal((2,) + lat.shape) + 1j * rng.standard_normal((2,) + lat.shape)
    Lq = bases(lat)[3] ** 2
    np.testing.assert_allclose(apply_Ar(lat, y, invB), y * (Lq / c)[None], rtol=1e-11,
                               atol=1e-11 * Lq.max() / c)


def test_gamma_point_zero_modes():
    """At 2 pi k = 0 only the (0,0,0) frequency has Lq = 0; A_r has exactly two zero eigenvalues
    and the rest equal the GEP's nonzero spectrum (the null space of C^*C grows by 2)."""
    lat = with_kappa(NAMED["fcc64"], [0.0, 0.0, 0.0])
    Lq = bases(lat)[3] ** 2
    assert int(np.sum(Lq == 0.0)) == 1
    B = _random_eps(lat, 9)
    invB = np.stack([1.0 / x for x in B])
    ar = np.sort(np.linalg.eigvalsh(Ar_dense(lat, invB)))
    assert np.all(np.abs(ar[:2]) < 1e-9) and ar[2] > 1e-3
    C = curl(lat)
    gep = gep_nonzero_eigs((C.conj().T @ C).toarray(), np.concatenate([x.ravel() for x in B]))
    np.testing.assert_allclose(ar[2:], gep, rtol=1e-9)


def test_basis_switch_keeps_orthonormality():
    """Where Lambda is parallel to (1,1,1) (simple cubic at Gamma, p = q = r) the paper's
    Pi_1, Pi_2 are undefined; the alternate reference vector still gives an orthonormal
    range basis orthogonal to Lambda."""
    w = W.WORKLOADS["sc16"]
    lat = make_lattice(w["vectors"], (6, 6, 6), np.zeros(3))
    Pi0, Pi1, Pi2, sig = bases(lat)
    L = np.stack(lambdas(lat))
    Lq = sig ** 2
    ratio = (3 * Lq - np.abs(L.sum(0)) ** 2) / np.where(Lq > 0, 3 * Lq, 1)
    switched = (ratio < G_TOL) & (Lq > 0)
    assert switched.sum() >= 5          # the diagonal p = q = r, at least
    for P in (Pi1, Pi2):
        np.testing.assert_allclose(np.sum(np.abs(P) ** 2, 0), 1.0, atol=1e-12)
        assert np.abs(np.sum(np.conj(L) * P, 0)).max() < 1e-10 * np.sqrt(Lq.max())
    assert np.abs(np.sum(np.conj(Pi1) * Pi2, 0)).max() < 1e-12


def test_expand_contract_adjoint(rng):
    """contract = expand^H (both carry Sigma_r once)."""
    lat = NAMED["mono80"]
    y = rng.standard_normal((2,) + lat.shape) + 1j * rng.standard_normal((2,) + lat.shape)
    v = rng.standard_normal((3,) + lat.shape) + 1j * rng.standard_normal((3,) + lat.shape)
    lhs = np.vdot(v, expand(lat, y))
    rhs = np.vdot(contract(lat, v), y)
    assert lhs == pytest.approx(rhs, rel=1e-12)
