"""Eigenvalue gradient with respect to the permittivity samples (oracle).

lambda_j = y_j^H A_r y_j with ||y_j|| = 1 and A_r = Sigma_r Q_r^* B^{-1} Q_r Sigma_r
(eq. NFSEP).  A_r is Hermitian and depends on B only through B^{-1}, so by the
Hellmann-Feynman argument

    d lambda_j / d B_l(v) = -|x_{j,l}(v)|^2,   x_j = B^{-1} Q_r Sigma_r y_j,

x_j being the eigenvector of the GEP given below Theorem invariant_space.  For
a cluster c of (numerically) equal eigenvalues the individual derivatives are
not defined; the cluster mean -(1/|c|) sum_{j in c} |x_j|^2 is the derivative
of the cluster's mean eigenvalue and is used for every member.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice
from .nfsep import lift, bases


def clusters(lam, rel_tol):
    """Group consecutive ascending eigenvalues whose gaps are <= rel_tol * lambda."""
    groups = [[0]]
    for j in range(1, len(lam)):
        if abs(lam[j] - lam[j - 1]) <= rel_tol * abs(lam[j - 1]):
            groups[-1].append(j)
        else:
            groups.append([j])
    return groups


def band_gradients(lat: Lattice, invB, Y, lam, rel_tol=1e-8):
    """d lambda_j / d B_l(v) for every band j: array (nev, 3, n3, n2, n1)."""
    b = bases(lat)
    invB = np.asarray(invB, dtype=np.float64).reshape((3,) + lat.shape)
    g = []
    for j in range(Y.shape[1]):
        y = Y[:, j] / np.linalg.norm(Y[:, j])
        x = lift(lat, y.reshape((2,) + lat.shape), invB, b)
        g.append(-np.abs(x) ** 2)
    g = np.array(g)
    out = np.empty_like(g)
    for c in clusters(lam, rel_tol):
        out[c] = np.mean(g[c], axis=0)[None]
    return out


def objective_gradient(lat, invB, Y, lam, dobj_dlam, rel_tol=1e-8):
    """sum_j dobj/dlambda_j * d lambda_j / d B: array (3, n3, n2, n1)."""
    G = band_gradients(lat, invB, Y, lam, rel_tol)
    return np.tensordot(np.asarray(dobj_dlam, dtype=np.float64), G, axes=(0, 0))
