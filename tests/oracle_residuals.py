"""Residuals ||A_r y - lambda y|| / (lambda ||y||) of eigenpairs, with A_r applied by
the CPU oracle (oracle.nfsep.apply_Ar, FP64) in a pool of worker processes.

Used by the full-size GPU tests to re-check every eigenpair the library returns with
an apply that shares no code with it.  The pool is started with the ``spawn`` method
(a worker forked from a process that already holds a CUDA context can hang), and each
worker builds the lattice and the range basis once.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle.lattice import make_lattice
from oracle.nfsep import apply_Ar, bases

_STATE = {}


def _init(vectors, n, bloch, invB):
    lat = make_lattice(vectors, n, bloch)
    _STATE.update(lat=lat, invB=np.asarray(invB).reshape((3,) + lat.shape), b=bases(lat))


def _residual(args):
    y, lam = args
    lat = _STATE["lat"]
    y = np.asarray(y, dtype=np.complex128).reshape((2,) + lat.shape)
    r = apply_Ar(lat, y, _STATE["invB"], _STATE["b"]) - lam * y
    return float(np.linalg.norm(r) / (abs(lam) * np.linalg.norm(y)))


def oracle_residuals(vectors, n, bloch, invB, lam, Y, workers=None):
    """Residual of each pair (lam[j], Y[j]) (Y: host complex array, one vector per row)."""
    cnt = len(lam)
    if workers is None:
        workers = max(1, min(cnt, (os.cpu_count() or 2) // 2, 8))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_init, initargs=(np.asarray(vectors), tuple(n), np.asarray(bloch),
                                                         np.asarray(invB))) as pool:
        return np.array(pool.map(_residual, [(Y[j], float(lam[j])) for j in range(cnt)], chunksize=1))
