"""Writes <name>_eigs.json for the band-path lattices (BCC 96^3, hexagonal
96x96x80, base-centred monoclinic 80x96x64, seeded eps = 12 rods/spheres): the
10 smallest eigenvalues of A_r at one Bloch vector of each lattice's path (path
point 22 of 60, on the segment (1/2,0,0) -> (1/2,1/2,0) in reduced coordinates),
computed by the FP64 oracle alone (block LOBPCG to residual 1e-10 relative).

Run from the repository root, one lattice per process (each takes tens of CPU
minutes and a few GB of memory):

    python tests/golden/make_band_path_eigs.py bcc96
    python tests/golden/make_band_path_eigs.py hex96
    python tests/golden/make_band_path_eigs.py mono80
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

PATH_INDEX = 22
NAMES = ("bcc96", "hex96", "mono80")


def main(name):
    if name not in NAMES:
        raise SystemExit(f"workload must be one of {NAMES}")
    nev, tol = 10, 1e-10
    w = W.WORKLOADS[name]
    K = W.bloch_vectors(name)[PATH_INDEX]
    lat = make_lattice(w["vectors"], w["n"], K)
    geom = W.Geometry(n=w["n"], s=(lat.s1, lat.s2, lat.s3), delta=(lat.dx, lat.dy, lat.dz), perm=lat.perm)
    invB = np.stack([1.0 / b for b in W.eps_for(name, geom)])
    t0 = time.time()
    lam, _, iters, res = lobpcg(lat, invB, nev, block=14, tol=tol, seed=0, max_iter=400)
    out = dict(workload=name, n=list(w["n"]), path_index=PATH_INDEX,
               reduced_k=[float(x) for x in W.bz_path_reduced(w["path"])[PATH_INDEX]],
               bloch=[float(x) for x in K], nev=nev, oracle_tol=tol, iterations=int(iters),
               max_residual=float(res.max()), seconds=round(time.time() - t0, 1),
               eigenvalues=[float(x) for x in lam])
    if out["max_residual"] > tol:
        raise SystemExit(f"oracle did not converge: {out}")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_eigs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1])
