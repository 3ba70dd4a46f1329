"""Pins for oracle.spectral (Section 4): T unitary, Algorithms 5.1/5.2, C_l T = T Lambda_l."""
import math

import numpy as np
import pytest

from oracle.curl import difference_ops
from oracle.spectral import T_dense, T_apply, Th_apply, lambdas, twist_fractions
from small_lattices import category_cover, named_small, random_triclinics

COVER = category_cover()
NAMED = named_small()
BOUNDARY = random_triclinics(21, 6, generic_only=False)
ALL = list(NAMED.values()) + COVER + BOUNDARY


def _id(l):
    return f"{l.n1}x{l.n2}x{l.n3}-m{l.m1}.{l.m2}.{l.m3}-r{l.rho1}{l.rho2}{l.rho3}"


@pytest.mark.parametrize("lat", ALL, ids=_id)
def test_T_unitary(lat):
    """T of eq. (T) is unitary with the n^{-1/2} scaling."""
    T = T_dense(lat)
    np.testing.assert_allclose(T.conj().T @ T, np.eye(lat.n), atol=1e-12)


@pytest.mark.parametrize("lat", ALL, ids=_id)
def test_diagonalises_difference_ops(lat):
    """C_l T = T Lambda_l (end of Section 4.2) with C_l from the quasi-periodic wrap."""
    T = T_dense(lat)
    ops = difference_ops(lat)
    for C, L in zip(ops, lambdas(lat)):
        np.testing.assert_allclose(C @ T, T * L.ravel()[None, :], atol=1e-10 * max(1, abs(L).max()))


@pytest.mark.parametrize("lat", ALL[:8], ids=_id)
def test_fft_matvecs_match_dense(lat, rng):
    """Algorithm 5.2 gives T q and Algorithm 5.1 gives T^* p."""
    T = T_dense(lat)
    q = rng.standard_normal(lat.n) + 1j * rng.standard_normal(lat.n)
    np.testing.assert_allclose(T_apply(lat, q.reshape(lat.shape)).ravel(), T @ q, atol=1e-12)
    np.testing.assert_allclose(Th_apply(lat, q.reshape(lat.shape)).ravel(), T.conj().T @ q,
                               atol=1e-12)


@pytest.mark.parametrize("lat", COVER + list(NAMED.values()), ids=_id)
def test_printed_theorem_phases(lat):
    """Lambda_2 and Lambda_3 are the eigenvalue sets of Theorems eigK2, eigK3_acute/obtuse.

    For each x-label the printed phases theta_{i,j} and theta_{i,j,k} (with the
    printed a^_2 and a^_3) give the same set of eigenvalues as ours; only the
    integer labels differ.
    """
    n1, n2, n3, m1, m2, m3 = lat.n1, lat.n2, lat.n3, lat.m1, lat.m2, lat.m3
    r1, r2, r3 = lat.rho1, lat.rho2, lat.rho3
    k1, k2, k3 = lat.kappa
    L1, L2, L3 = lambdas(lat)
    ka2 = k2 - m1 / n1 * k1 + r1 * k1                      # k . a^_2 (Theorem eigK2)
    acute = (lat.cos_alpha - lat.cos_beta * lat.cos_gamma) >= 0
    if acute:                                              # k . a^_3 (Theorem eigK3_acute)
        ka3 = (k3 - m3 / n2 * k2 - (n2 - m3) / n2 * m1 / n1 * k1 + (m1 - m2) / n1 * k1
               + r3 * k2 - m3 / n2 * r1 * k1 + r2 * k1)
    else:                                                  # Theorem eigK3_obtuse
        ka3 = (k3 - m3 / n2 * k2 - (n2 - m3) / n2 * m1 / n1 * k1 - m2 / n1 * k1
               + r3 * k2 - m3 / n2 * r1 * k1 + r1 * k1 + r2 * k1)
    for p in range(n1):
        # the paper's label i for our p is p itself (i and p differ by multiples of n1 only)
        i = p
        th2 = np.array([2 * math.pi * (j - m1 / n1 * i + ka2) / n2 for j in range(n2)])
        paper2 = (np.exp(1j * th2) - 1) / lat.dy
        np.testing.assert_allclose(np.sort_complex(np.round(paper2, 10)),
                                   np.sort_complex(np.round(L2[0, :, p], 10)), atol=1e-8)
        for q in range(n2):
            # our q pairs with the paper's j = q + (integer); find it from the phase
            j = int(round((n2 * np.angle(np.exp(2j * math.pi * ((q + twist_fractions(lat)[1][p])
                                                             / n2))) / (2 * math.pi)
                           + m1 / n1 * i - ka2))) % n2
            lab = j
            if acute:
                base = -m3 / n2 * lab - (n2 - m3) / n2 * m1 / n1 * i + (m1 - m2) / n1 * i + ka3
            else:
                base = -m3 / n2 * lab - (n2 - m3) / n2 * m1 / n1 * i - m2 / n1 * i + ka3
            paper3 = (np.exp(2j * math.pi * (np.arange(n3) + base) / n3) - 1) / lat.dz
            np.testing.assert_allclose(np.sort_complex(np.round(paper3, 10)),
                                       np.sort_complex(np.round(L3[:, q, p], 10)), atol=1e-8)


def test_sc_is_twisted_dft():
    """Simple cubic (all offsets zero): T = D_x U_{n1} (x) ... with constant twists; the
    column (p,q,r) of T is the separable plane wave e^{2 pi i (a(p+k1)/n1 + b(q+k2)/n2 + c(r+k3)/n3)}."""
    lat = NAMED["sc16"]
    T = T_dense(lat)
    k1, k2, k3 = lat.kappa
    a = np.arange(lat.n1); b = np.arange(lat.n2); c = np.arange(lat.n3)
    for (p, q, r) in [(0, 0, 0), (1, 2, 1), (lat.n1 - 1, lat.n2 - 1, lat.n3 - 1)]:
        col = p + lat.n1 * (q + lat.n2 * r)
        wave = (np.exp(2j * math.pi * c * (r + k3) / lat.n3)[:, None, None]
                * np.exp(2j * math.pi * b * (q + k2) / lat.n2)[None, :, None]
                * np.exp(2j * math.pi * a * (p + k1) / lat.n1)[None, None, :])
        np.testing.assert_allclose(T[:, col], wave.ravel() / math.sqrt(lat.n), atol=1e-13)
