"""Writes workload_eigs.json: the 10 smallest eigenvalues of A_r, computed by the FP64
oracle alone (block LOBPCG to residual 1e-10 relative), for

* the gyroid on the BCC lattice (sin X cos Y + sin Y cos Z + sin Z cos X > 1.1,
  Section 6) at 24^3, Bloch vector (1/2, 1/2, 0) in reduced coordinates, with the
  gyroid's permittivity 3, 13 and 30 (the ends and the middle of the paper's sweep);
* the simple cubic supercell of 2 x 2 x 2 cells with one cell's sphere removed (the
  supercell of the concluding remarks) at 12^3 per cell (24^3 in all).

Run from the repository root (a few CPU minutes):

    python tests/golden/make_workload_eigs.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.lattice import make_lattice            # noqa: E402
from oracle.eigs import lobpcg                     # noqa: E402
from paper_1806_10284_gb300 import workloads as W  # noqa: E402  (seeded inputs only)

NEV, TOL = 10, 1e-10
GYROID_N = (24, 24, 24)
GYROID_EPS = (3.0, 13.0, 30.0)
VAC_CELL_N = (12, 12, 12)


def geometry(lat):
    return W.Geometry(n=(lat.n1, lat.n2, lat.n3), s=(lat.s1, lat.s2, lat.s3),
                      delta=(lat.dx, lat.dy, lat.dz), perm=tuple(lat.perm))


def solve(lat, B):
    invB = np.stack([1.0 / b for b in B])
    t0 = time.time()
    lam, _, iters, res = lobpcg(lat, invB, NEV, block=14, tol=TOL, seed=0, max_iter=500)
    if res.max() > TOL:
        raise SystemExit(f"oracle did not converge: {res.max()}")
    return dict(eigenvalues=[float(x) for x in lam], iterations=int(iters),
                max_residual=float(res.max()), seconds=round(time.time() - t0, 1))


def main():
    out = dict(nev=NEV, oracle_tol=TOL, gyroid=[], vacancy=None)
    w = W.WORKLOADS["gyroid96"]
    red = w["reduced_k"][0]
    K = W.bloch_from_reduced(w["vectors"], red)
    lat = make_lattice(w["vectors"], GYROID_N, K)
    for e in GYROID_EPS:
        r = solve(lat, W.eps_for("gyroid96", geometry(lat), eps_in=e))
        r.update(eps_in=e, n=list(GYROID_N), reduced_k=[float(x) for x in red], bloch=[float(x) for x in K])
        out["gyroid"].append(r)
        print(json.dumps(r), flush=True)
    v = W.WORKLOADS["scvac"]
    K = W.bloch_vectors("scvac")[0]
    cell = make_lattice(v["vectors"], VAC_CELL_N, K)
    Vs, ns = W.supercell(v["vectors"], VAC_CELL_N, v["reps"])
    lat = make_lattice(Vs, ns, K)
    r = solve(lat, W.eps_for("scvac", geometry(cell)))
    r.update(cell_n=list(VAC_CELL_N), n=list(ns), reps=list(v["reps"]), bloch=[float(x) for x in K])
    out["vacancy"] = r
    print(json.dumps(r), flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_eigs.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
