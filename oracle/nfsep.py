"""SVD of the curl and the null-space-free reduction (Section 5.1-5.2; oracle).

Per frequency, with Lambda = (Lambda_1, Lambda_2, Lambda_3)^T:

    Lambda_q = |Lambda_1|^2 + |Lambda_2|^2 + |Lambda_3|^2
    Pi_0 = Lambda / Lambda_q^{1/2}                                 (eq. null_basis)
    Pi_1 = (Lambda_q e - Lambda (Lambda^H e)) / sqrt(Lambda_q g)   (eq. range_basis1)
    Pi_2 = conj(e x Lambda) / sqrt(g)                              (eq. range_basis2)
    g    = |e|^2 Lambda_q - |e . Lambda|^2
    Sigma_r = diag(Lambda_q^{1/2}, Lambda_q^{1/2})                 (eq. SVD)

With the reference vector e = (1, 1, 1) these are the paper's Pi_1 (with
Lambda^H e = conj(Lambda_s), Lambda_s = Lambda_1 + Lambda_2 + Lambda_3) and
Pi_2 = (Lambda_3^* - Lambda_2^*, Lambda_1^* - Lambda_3^*, Lambda_2^* - Lambda_1^*),
normalised to unit columns.  The paper's formulas divide by zero when Lambda
is parallel to (1, 1, 1); where g < G_TOL * 3 Lambda_q the reference vector
e = (1, -1, 0) is used instead (any orthonormal pair orthogonal to Lambda
gives the same A_r spectrum).  Where Lambda = 0 (the Gamma point, (p,q,r) =
(0,0,0)) Sigma_r = 0 and the basis is (1, w, w^2)/sqrt3, (1, w^2, w)/sqrt3,
w = e^{2 pi i/3}.

A_r y = Sigma_r Q_r^* B^{-1} Q_r Sigma_r y with Q_r = (I_3 (x) T) [Pi_1 Pi_2]
(eq. NFSEP).  Vectors y of A_r are (2, n3, n2, n1) arrays: y[0] the Pi_1
coordinate, y[1] the Pi_2 coordinate.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .lattice import Lattice
from .spectral import lambdas, T_apply, Th_apply, T_dense

# Relative size of g below which the reference vector switches from (1,1,1) to (1,-1,0).
G_TOL = 1.0 / 16.0


def bases(lat: Lattice):
    """Return (Pi0, Pi1, Pi2, sigma): Pi's of shape (3, n3, n2, n1), sigma (n3, n2, n1)."""
    L = np.stack(lambdas(lat))                      # (3, ...)
    Lq = np.sum(np.abs(L) ** 2, axis=0)
    ones = np.ones(3)
    alt = np.array([1.0, -1.0, 0.0])
    g_one = 3.0 * Lq - np.abs(np.sum(L, axis=0)) ** 2
    use_alt = g_one < G_TOL * 3.0 * Lq
    e = np.where(use_alt[None], alt[:, None, None, None], ones[:, None, None, None])
    e_dot_L = np.sum(e * L, axis=0)                 # e . Lambda (e real)
    e2 = np.sum(e * e, axis=0)
    g = e2 * Lq - np.abs(e_dot_L) ** 2
    zero = Lq == 0.0
    safe_Lq = np.where(zero, 1.0, Lq)
    safe_g = np.where(zero, 1.0, g)
    Pi1 = (Lq[None] * e - L * np.conj(e_dot_L)[None]) / np.sqrt(safe_Lq * safe_g)[None]
    cross = np.stack([e[1] * L[2] - e[2] * L[1],
                      e[2] * L[0] - e[0] * L[2],
                      e[0] * L[1] - e[1] * L[0]])
    Pi2 = np.conj(cross) / np.sqrt(safe_g)[None]
    w = np.exp(2j * math.pi / 3.0)
    if np.any(zero):
        Pi1[:, zero] = (np.array([1.0, w, w * w]) / math.sqrt(3.0))[:, None]
        Pi2[:, zero] = (np.array([1.0, w * w, w]) / math.sqrt(3.0))[:, None]
    Pi0 = L / np.sqrt(safe_Lq)[None]
    Pi0[:, zero] = 0.0
    sigma = np.sqrt(Lq)
    return Pi0, Pi1, Pi2, sigma


def basis_margin(lat: Lattice) -> float:
    """Smallest |g/(3 Lambda_q) - G_TOL| over nonzero frequencies (how far from a basis switch)."""
    L = np.stack(lambdas(lat))
    Lq = np.sum(np.abs(L) ** 2, axis=0)
    nz = Lq > 0
    ratio = (3.0 * Lq[nz] - np.abs(np.sum(L, axis=0)[nz]) ** 2) / (3.0 * Lq[nz])
    return float(np.min(np.abs(ratio - G_TOL)))


def expand(lat: Lattice, y, bases_=None):
    """v = [Pi_1 Pi_2] Sigma_r y, a (3, n3, n2, n1) frequency field."""
    _, Pi1, Pi2, sigma = bases_ if bases_ is not None else bases(lat)
    y = np.asarray(y).reshape((2,) + lat.shape)
    return Pi1 * (sigma * y[0])[None] + Pi2 * (sigma * y[1])[None]


def contract(lat: Lattice, w, bases_=None):
    """Sigma_r [Pi_1 Pi_2]^H w for a (3, n3, n2, n1) frequency field."""
    _, Pi1, Pi2, sigma = bases_ if bases_ is not None else bases(lat)
    z0 = np.sum(np.conj(Pi1) * w, axis=0) * sigma
    z1 = np.sum(np.conj(Pi2) * w, axis=0) * sigma
    return np.stack([z0, z1])


def lift(lat: Lattice, y, invB, bases_=None):
    """x = B^{-1} Q_r Sigma_r y (the eigenvector map below Theorem invariant_space)."""
    v = expand(lat, y, bases_)
    return np.stack([T_apply(lat, v[l]) * invB[l] for l in range(3)])


def apply_Ar(lat: Lattice, y, invB, bases_=None):
    """A_r y = Sigma_r Q_r^* B^{-1} Q_r Sigma_r y (eq. NFSEP) via Algorithms 5.2 and 5.1.

    ``invB``: (3, n3, n2, n1) array of 1/B_l.  ``y``: (2, n3, n2, n1).
    """
    b = bases_ if bases_ is not None else bases(lat)
    x = lift(lat, y, invB, b)
    w = np.stack([Th_apply(lat, x[l]) for l in range(3)])
    return contract(lat, w, b)


def Qr_dense(lat: Lattice, bases_=None):
    """Q_r = (I_3 (x) T)[Pi_1 Pi_2] as a dense 3n x 2n matrix (small n only)."""
    _, Pi1, Pi2, _ = bases_ if bases_ is not None else bases(lat)
    T = T_dense(lat)
    n = lat.n
    Q = np.zeros((3 * n, 2 * n), dtype=np.complex128)
    for l in range(3):
        Q[l * n:(l + 1) * n, :n] = T * Pi1[l].ravel()[None, :]
        Q[l * n:(l + 1) * n, n:] = T * Pi2[l].ravel()[None, :]
    return Q


def Q0_dense(lat: Lattice, bases_=None):
    """Q_0 = (I_3 (x) T) Pi_0 (eq. null_basis), dense 3n x n."""
    Pi0 = (bases_ if bases_ is not None else bases(lat))[0]
    T = T_dense(lat)
    n = lat.n
    return np.concatenate([T * Pi0[l].ravel()[None, :] for l in range(3)], axis=0)


def Ar_dense(lat: Lattice, invB, bases_=None):
    """Dense A_r = Sigma_r Q_r^* B^{-1} Q_r Sigma_r (small n only)."""
    b = bases_ if bases_ is not None else bases(lat)
    Q = Qr_dense(lat, b)
    s = np.concatenate([b[3].ravel(), b[3].ravel()])
    M = Q.conj().T @ (np.ravel(invB)[:, None] * Q)
    return s[:, None] * M * s[None, :]


def gep_nonzero_eigs(A, Bdiag, tol=1e-9):
    """Nonzero eigenvalues of the GEP A x = lambda B x (eq. GEP), dense, ascending."""
    w = sla.eigh(A, np.diag(Bdiag), eigvals_only=True)
    scale = max(1.0, float(np.max(np.abs(w))))
    return np.sort(w[np.abs(w) > tol * scale])
