"""Explicit Yee curl of Section 3 (oracle; test infrastructure only).

Two independent constructions of the forward-difference operators C1, C2, C3:

1. ``difference_ops``: straight from the quasi-periodic condition
   (eq. quasi_periodic) as used in Theorems period1, period2 and period3.  A
   neighbour (i, j, k) + e_l that leaves the box is written as a box point plus
   an integer combination of the lattice shifts a1 <-> (n1,0,0),
   a2 <-> (s1,n2,0), a3 <-> (s2,s3,n3); each shift by a_l multiplies the field
   by exp(i 2 pi kappa_l).

2. ``paper_K1``, ``paper_K2``, ``paper_K3``: the matrices as printed in
   eqs. (K1), (K2), (K3) with J2 from eq. (J2) and J3 from the four general
   categories (eqs. acuteJ3, obtuseJ3) built on J1 (eq. J1) and the integers
   rho1..rho5, psi1, psi2 defined beside them.

The curl is C = [[0, -C3, C2], [C3, 0, -C1], [-C2, C1, 0]] (Section 3.1) and the
gradient G = [C1; C2; C3].  Field vectors use vec order (x index fastest),
component blocks e1, e2, e3 stacked.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .lattice import Lattice


def wrap_index(lat: Lattice, i: int, j: int, k: int):
    """Return (i', j', k', phase) with the box point and the quasi-periodic factor.

    The field at the (possibly out-of-box) index (i, j, k) equals
    phase * field(i', j', k'), per eq. (quasi_periodic).
    """
    t = np.zeros(3)
    q3 = k // lat.n3
    i, j, k = i - q3 * lat.s2, j - q3 * lat.s3, k - q3 * lat.n3
    t[2] += q3
    q2 = j // lat.n2
    i, j = i - q2 * lat.s1, j - q2 * lat.n2
    t[1] += q2
    q1 = i // lat.n1
    i = i - q1 * lat.n1
    t[0] += q1
    phase = np.exp(2j * math.pi * float(np.dot(t, lat.kappa)))
    return i, j, k, phase


def _lin(lat, i, j, k):
    return i + lat.n1 * (j + lat.n2 * k)


def difference_ops(lat: Lattice):
    """Sparse C1, C2, C3 (each n x n): forward differences with quasi-periodic wrap."""
    n1, n2, n3 = lat.n1, lat.n2, lat.n3
    n = lat.n
    deltas = (lat.dx, lat.dy, lat.dz)
    mats = []
    for ax in range(3):
        rows, cols, vals = [], [], []
        for k in range(n3):
            for j in range(n2):
                for i in range(n1):
                    r = _lin(lat, i, j, k)
                    rows.append(r); cols.append(r); vals.append(-1.0 / deltas[ax])
                    ii, jj, kk = i + (ax == 0), j + (ax == 1), k + (ax == 2)
                    ii, jj, kk, ph = wrap_index(lat, ii, jj, kk)
                    rows.append(r); cols.append(_lin(lat, ii, jj, kk))
                    vals.append(ph / deltas[ax])
        mats.append(sp.csr_matrix((np.array(vals, dtype=np.complex128),
                                   (rows, cols)), shape=(n, n)))
    return tuple(mats)


def curl(lat: Lattice, ops=None):
    """C = [[0, -C3, C2], [C3, 0, -C1], [-C2, C1, 0]] (Section 3.1)."""
    C1, C2, C3 = ops if ops is not None else difference_ops(lat)
    Z = sp.csr_matrix(C1.shape, dtype=np.complex128)
    return sp.bmat([[Z, -C3, C2], [C3, Z, -C1], [-C2, C1, Z]], format="csr")


def gradient(lat: Lattice, ops=None):
    """G = [C1; C2; C3], the discrete gradient whose range is the null space of C."""
    C1, C2, C3 = ops if ops is not None else difference_ops(lat)
    return sp.vstack([C1, C2, C3], format="csr")


def eps_matrix(B1, B2, B3):
    """B = diag(vec B1, vec B2, vec B3) (Section 3)."""
    return sp.diags(np.concatenate([np.ravel(B1), np.ravel(B2), np.ravel(B3)]).astype(np.float64))


# ---------------------------------------------------------------------------
# The paper's printed forms (eqs. K1, K2, K3, J2, J1, acuteJ3, obtuseJ3).
# ---------------------------------------------------------------------------

def _ex(x):
    return np.exp(2j * math.pi * x)


def _cyc(n1, s, k1):
    """[[0, e^{-i2pi k.a1} I_s], [I_{n1-s}, 0]] (n1 x n1), the block used throughout."""
    M = np.zeros((n1, n1), dtype=np.complex128)
    for r in range(s):
        M[r, n1 - s + r] = _ex(-k1)
    for r in range(s, n1):
        M[r, r - s] = 1.0
    return M


def _paper_ints(lat: Lattice):
    """rho1..rho5, psi1, psi2 as defined beside eqs. (J2), (J1)."""
    cg, cb, ca = lat.cos_gamma, lat.cos_beta, lat.cos_alpha
    rho1, rho2, rho3 = lat.rho1, lat.rho2, lat.rho3
    rho4 = int(math.ceil(cg * cb * (cg * cb - ca)))
    rho5 = int(math.ceil(cb))
    n1, m1, m2 = lat.n1, lat.m1, lat.m2
    psi1 = 1 if ((rho2 * n1 - m2) - (rho1 * n1 - m1) > 0 and rho3 == 0) else 0
    psi2 = 1 if ((rho1 * n1 - m1) + (rho2 * n1 - m2) > 0 and rho3 == 1) else 0
    return rho1, rho2, rho3, rho4, rho5, psi1, psi2


def paper_J2(lat: Lattice):
    k1 = lat.kappa[0]
    return _ex(lat.rho1 * k1) * _cyc(lat.n1, lat.m1, k1)


def paper_J1(lat: Lattice):
    k1 = lat.kappa[0]
    return _ex(lat.rho2 * k1) * _cyc(lat.n1, lat.m2, k1)


def paper_J3(lat: Lattice):
    """J3 from the four general categories of Section 3.1."""
    n1, n2, m1, m2, m3 = lat.n1, lat.n2, lat.m1, lat.m2, lat.m3
    k1, k2 = lat.kappa[0], lat.kappa[1]
    rho1, rho2, rho3, rho4, rho5, psi1, psi2 = _paper_ints(lat)
    J1 = paper_J1(lat)
    N = n1 * n2
    J3 = np.zeros((N, N), dtype=np.complex128)
    top = m3 * n1
    acute = (lat.cos_alpha - lat.cos_gamma * lat.cos_beta) >= 0.0
    if acute:
        if m1 <= m2:      # category (1)
            f = _ex(-(k2 + rho1 * rho4 * k1 - psi1 * k1))
            inner = _cyc(n1, m2 - m1, k1)
        else:             # category (2)
            f = _ex(-(k2 - rho2 * rho4 * k1 - psi1 * k1))
            inner = _cyc(n1, n1 - m1 + m2, k1)
        J3[:top, N - top:] = f * np.kron(np.eye(m3), inner)
        J3[top:, :N - top] = np.kron(np.eye(n2 - m3), J1)
    else:
        J3[:top, N - top:] = _ex(-k2) * np.kron(np.eye(m3), J1)
        if m1 + m2 <= n1:  # category (3)
            f = _ex((rho1 * rho4 + psi2) * k1)
            inner = _cyc(n1, m1 + m2, k1)
        else:              # category (4)
            f = _ex(-(rho5 * rho4 - psi2) * k1)
            inner = _cyc(n1, m1 + m2 - n1, k1)
        J3[top:, :N - top] = f * np.kron(np.eye(n2 - m3), inner)
    return _ex(rho3 * k2) * J3


def _bidiag(nb, bs, corner, delta):
    """(1/delta) * block bidiagonal [-I I; ...; corner ... -I] with nb blocks of size bs."""
    N = nb * bs
    K = np.zeros((N, N), dtype=np.complex128)
    for b in range(nb):
        K[b * bs:(b + 1) * bs, b * bs:(b + 1) * bs] = -np.eye(bs)
        if b + 1 < nb:
            K[b * bs:(b + 1) * bs, (b + 1) * bs:(b + 2) * bs] = np.eye(bs)
    K[(nb - 1) * bs:, :bs] += corner
    return K / delta


def paper_K1(lat: Lattice):
    return _bidiag(lat.n1, 1, _ex(lat.kappa[0]) * np.eye(1), lat.dx)


def paper_K2(lat: Lattice):
    return _bidiag(lat.n2, lat.n1, _ex(lat.kappa[1]) * paper_J2(lat), lat.dy)


def paper_K3(lat: Lattice):
    return _bidiag(lat.n3, lat.n1 * lat.n2, _ex(lat.kappa[2]) * paper_J3(lat), lat.dz)


def paper_difference_ops(lat: Lattice):
    """C1 = I (x) I (x) K1, C2 = I (x) K2, C3 = K3 as dense matrices (small n only)."""
    C1 = np.kron(np.eye(lat.n2 * lat.n3), paper_K1(lat))
    C2 = np.kron(np.eye(lat.n3), paper_K2(lat))
    C3 = paper_K3(lat)
    return C1, C2, C3
