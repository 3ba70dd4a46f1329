"""Smallest eigenvalues of A_r (oracle; test infrastructure only).

The paper finds the smallest eigenvalues of A_r with inverse Lanczos (Section
5.2, Section 6); any convergent Hermitian eigensolver yields the same
numbers, so the oracle uses the plainest one it can state in a few lines: the
locally optimal block preconditioned conjugate gradient method of Knyazev
(SIAM J. Sci. Comput. 23(2), 2001), in FP64, with a Rayleigh-Ritz step on
span{X, W, P} each iteration, and the preconditioner
T = Sigma_r^{-2} / mean(B^{-1}), which is A_r^{-1} exactly when B is constant.
For small n, ``eigs_dense`` diagonalises the dense A_r instead.

At the Gamma point (Lambda = 0 at (p,q,r) = (0,0,0)) A_r has two exact zero
eigenvalues carried by the zero-frequency coordinates; they are removed by
keeping every block orthogonal to those coordinates, so the returned values
are the smallest nonzero ones.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .lattice import Lattice
from .nfsep import bases, apply_Ar, Ar_dense


def _svqb(S, AS, drop=1e-12):
    """Orthonormalise the columns of S (and carry AS along): Stathopoulos-Wu SVQB."""
    G = S.conj().T @ S
    G = 0.5 * (G + G.conj().T)
    d = np.sqrt(np.maximum(np.real(np.diag(G)), 1e-300))
    Gs = G / d[:, None] / d[None, :]
    w, U = np.linalg.eigh(Gs)
    keep = w > drop * max(w.max(), 1e-300)
    M = (U[:, keep] / np.sqrt(w[keep])[None, :]) / d[:, None]
    return S @ M, (AS @ M if AS is not None else None)


def eigs_dense(lat: Lattice, invB, nev: int):
    """nev smallest nonzero eigenvalues (and vectors) of the dense A_r."""
    A = Ar_dense(lat, invB)
    A = 0.5 * (A + A.conj().T)
    w, V = np.linalg.eigh(A)
    zero = np.abs(w) <= 1e-10 * max(1.0, np.max(np.abs(w)))
    w, V = w[~zero], V[:, ~zero]
    return w[:nev], V[:, :nev]


def lobpcg(lat: Lattice, invB, nev: int, block: int | None = None, tol: float = 1e-11,
           max_iter: int = 500, seed: int = 0, X0=None, verbose: bool = False):
    """Block LOBPCG for the nev smallest nonzero eigenpairs of A_r.

    Returns (lam[nev], Y (2n x nev) with unit columns, iterations, residuals).
    The residual of pair j is ||A_r y_j - lam_j y_j|| / lam_j.
    """
    n2 = 2 * lat.n
    m = block if block is not None else nev + max(4, nev // 2)
    b = bases(lat)
    sigma = b[3]
    invB = np.asarray(invB, dtype=np.float64).reshape((3,) + lat.shape)
    sig2 = np.concatenate([sigma.ravel() ** 2] * 2)
    keep = sig2 > 0.0
    mean_invB = float(np.mean(invB))
    tinv = np.where(keep, 1.0 / np.where(keep, sig2 * mean_invB, 1.0), 0.0)

    def A(Y):
        out = np.empty_like(Y)
        for j in range(Y.shape[1]):
            out[:, j] = apply_Ar(lat, Y[:, j].reshape((2,) + lat.shape), invB, b).ravel()
        return out

    rng = np.random.default_rng(seed)
    if X0 is None:
        X = rng.standard_normal((n2, m)) + 1j * rng.standard_normal((n2, m))
    else:
        X = np.array(X0, dtype=np.complex128)
    X[~keep, :] = 0.0
    X, _ = _svqb(X, None)
    AX = A(X)
    P = AP = None
    lam = res = None
    it = 0
    for it in range(1, max_iter + 1):
        # Rayleigh-Ritz on span{X, W, P}; on the first pass span{X} only.
        if P is None and lam is None:
            S, AS = X, AX
        else:
            R = AX - X * lam[None, :]
            W = tinv[:, None] * R
            W = W - X @ (X.conj().T @ W)
            AW = A(W)
            if P is None:
                Q, AQ = W, AW
            else:
                Q, AQ = np.hstack([W, P]), np.hstack([AW, AP])
            Q, AQ = _svqb(Q, AQ)
            S, AS = np.hstack([X, Q]), np.hstack([AX, AQ])
        GA = S.conj().T @ AS
        GA = 0.5 * (GA + GA.conj().T)
        GB = S.conj().T @ S
        GB = 0.5 * (GB + GB.conj().T)
        w, C = sla.eigh(GA, GB)
        C = C[:, :m]
        lam = w[:m]
        Xn, AXn = S @ C, AS @ C
        if S.shape[1] > X.shape[1]:
            k = X.shape[1]
            P, AP = S[:, k:] @ C[k:, :], AS[:, k:] @ C[k:, :]
        X, AX = Xn, AXn
        nrm = np.linalg.norm(X, axis=0)
        X, AX = X / nrm, AX / nrm
        R = AX - X * lam[None, :]
        res = np.linalg.norm(R, axis=0) / np.abs(lam)
        if verbose:
            print(it, res[:nev].max(), lam[:nev])
        if np.all(res[:nev] <= tol):
            break
    return lam[:nev], X[:, :nev], it, res[:nev]
