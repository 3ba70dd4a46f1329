"""Simultaneous diagonalisation of C1, C2, C3 (Section 4; oracle, test infrastructure).

Frequency labels (p, q, r), p in [0, n1), q in [0, n2), r in [0, n3), with the
twisted fractions of Theorems eigK1, eigK2, eigK3_acute and eigK3_obtuse,
written on the index-shift lattice a1 <-> (n1,0,0), a2 <-> (s1,n2,0),
a3 <-> (s2,s3,n3):

    c1       = kappa1
    c2(p)    = kappa2 - s1 (p + c1) / n1
    c3(p, q) = kappa3 - s2 (p + c1) / n1 - s3 (q + c2(p)) / n2

    theta_1 = 2 pi (p + c1) / n1,  theta_2 = 2 pi (q + c2) / n2,
    theta_3 = 2 pi (r + c3) / n3,  Lambda_l = (e^{i theta_l} - 1) / delta_l.

These reproduce the theorems' phases up to an integer relabelling of q and r
(the rho's and the i-dependent integer parts move into the labels).  The
column of T for (p, q, r) is n^{-1/2} z (x) y (x) x with
x[a] = e^{i a theta_1}, y[b] = e^{i b theta_2}, z[c] = e^{i c theta_3}
(eq. T); columns are ordered p fastest, then q, then r, a permutation of the
paper's ordering of eq. (T).

Arrays of one grid field have numpy shape (n3, n2, n1): axis 2 is x/p.
"""
from __future__ import annotations

import math

import numpy as np

from .lattice import Lattice


def twist_fractions(lat: Lattice):
    """c1 (scalar), c2[p] (n1,), c3[q, p] (n2, n1)."""
    p = np.arange(lat.n1, dtype=np.float64)
    q = np.arange(lat.n2, dtype=np.float64)
    c1 = float(lat.kappa[0])
    c2 = lat.kappa[1] - lat.s1 * (p + c1) / lat.n1
    c3 = (lat.kappa[2] - lat.s2 * (p[None, :] + c1) / lat.n1
          - lat.s3 * (q[:, None] + c2[None, :]) / lat.n2)
    return c1, c2, c3


def phases(lat: Lattice):
    """theta_1, theta_2, theta_3 / (2 pi) broadcast to shape (n3, n2, n1)."""
    c1, c2, c3 = twist_fractions(lat)
    p = np.arange(lat.n1, dtype=np.float64)
    q = np.arange(lat.n2, dtype=np.float64)
    r = np.arange(lat.n3, dtype=np.float64)
    f1 = np.broadcast_to(((p + c1) / lat.n1)[None, None, :], lat.shape)
    f2 = np.broadcast_to(((q[:, None] + c2[None, :]) / lat.n2)[None, :, :], lat.shape)
    f3 = (r[:, None, None] + c3[None, :, :]) / lat.n3
    return f1, f2, f3


def lambdas(lat: Lattice):
    """Lambda_1, Lambda_2, Lambda_3 (eq. eigenvalue_K), each of shape (n3, n2, n1)."""
    f1, f2, f3 = phases(lat)
    L1 = (np.exp(2j * math.pi * f1) - 1.0) / lat.dx
    L2 = (np.exp(2j * math.pi * f2) - 1.0) / lat.dy
    L3 = (np.exp(2j * math.pi * f3) - 1.0) / lat.dz
    return L1, L2, L3


def T_dense(lat: Lattice) -> np.ndarray:
    """The n x n matrix T of eq. (T) with columns in (p, q, r) order (small n only)."""
    f1, f2, f3 = phases(lat)
    a = np.arange(lat.n1)
    b = np.arange(lat.n2)
    c = np.arange(lat.n3)
    n = lat.n
    T = np.empty((n, n), dtype=np.complex128)
    F1, F2, F3 = f1.ravel(), f2.ravel(), f3.ravel()
    # row index a + n1 (b + n2 c)
    A = np.broadcast_to(a[None, None, :], lat.shape).ravel()
    Bi = np.broadcast_to(b[None, :, None], lat.shape).ravel()
    Ci = np.broadcast_to(c[:, None, None], lat.shape).ravel()
    for col in range(n):
        T[:, col] = np.exp(2j * math.pi * (A * F1[col] + Bi * F2[col] + Ci * F3[col]))
    return T / math.sqrt(n)


def T_apply(lat: Lattice, q: np.ndarray) -> np.ndarray:
    """u = T q by Algorithm 5.2 (z transform and D_a3 twist, then y with D_a2, then x with D_a1).

    ``q`` has shape (n3, n2, n1) indexed [r, q, p]; returns u indexed [c, b, a].
    The U_n of eq. (DFT_matrix) are inverse DFTs without normalisation:
    U[a, p] = e^{+2 pi i a p / n}; numpy's ifft carries 1/n, undone here.
    """
    n1, n2, n3 = lat.n1, lat.n2, lat.n3
    c1, c2, c3 = twist_fractions(lat)
    x = np.asarray(q, dtype=np.complex128).reshape(lat.shape)
    # Step 1: for each (p, q): U_{n3} along r, then D_{a3}(p, q) indexed by c.
    x = np.fft.ifft(x, axis=0) * n3
    c = np.arange(n3, dtype=np.float64)
    x = x * np.exp(2j * math.pi * c[:, None, None] * c3[None, :, :] / n3)
    # Step 2: for each (p, c): U_{n2} along q, then D_{a2}(p) indexed by b.
    x = np.fft.ifft(x, axis=1) * n2
    b = np.arange(n2, dtype=np.float64)
    x = x * np.exp(2j * math.pi * b[None, :, None] * c2[None, None, :] / n2)
    # Step 3: for each (b, c): D_{a1} U_{n1} along p.
    x = np.fft.ifft(x, axis=2) * n1
    a = np.arange(n1, dtype=np.float64)
    x = x * np.exp(2j * math.pi * a[None, None, :] * c1 / n1)
    return x / math.sqrt(lat.n)


def Th_apply(lat: Lattice, p: np.ndarray) -> np.ndarray:
    """w = T^* p by Algorithm 5.1 (x with D_a1^*, then y with D_a2^*, then z with D_a3^*).

    ``p`` has shape (n3, n2, n1) indexed [c, b, a]; returns w indexed [r, q, p].
    Normalisation n^{-1/2}, which makes T unitary (eq. T), is used in place of
    the 1/n printed in the last lines of Algorithms 5.1 and 5.2.
    """
    n1, n2, n3 = lat.n1, lat.n2, lat.n3
    c1, c2, c3 = twist_fractions(lat)
    x = np.asarray(p, dtype=np.complex128).reshape(lat.shape)
    a = np.arange(n1, dtype=np.float64)
    x = x * np.exp(-2j * math.pi * a[None, None, :] * c1 / n1)
    x = np.fft.fft(x, axis=2)
    b = np.arange(n2, dtype=np.float64)
    x = x * np.exp(-2j * math.pi * b[None, :, None] * c2[None, None, :] / n2)
    x = np.fft.fft(x, axis=1)
    c = np.arange(n3, dtype=np.float64)
    x = x * np.exp(-2j * math.pi * c[:, None, None] * c3[None, :, :] / n3)
    x = np.fft.fft(x, axis=0)
    return x / math.sqrt(lat.n)
