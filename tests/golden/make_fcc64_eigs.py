"""Writes fcc64_eigs.json: the 10 smallest eigenvalues of A_r for the FCC 64^3
diamond-site workload (eps = 13 spheres, reduced k = (0.3, 0.2, 0.1)), computed by
the FP64 oracle alone (block LOBPCG to residual 1e-10 relative).  Run from the
repository root:  python tests/golden/make_fcc64_eigs.py   (several CPU minutes)."""
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


def main():
    name, nev, tol = "fcc64", 10, 1e-10
    w = W.WORKLOADS[name]
    K = W.bloch_vectors(name)[0]
    lat = make_lattice(w["vectors"], w["n"], K)
    geom = W.Geometry(n=w["n"], s=(lat.s1, lat.s2, lat.s3), delta=(lat.dx, lat.dy, lat.dz), perm=lat.perm)
    invB = np.stack([1.0 / b for b in W.eps_for(name, geom)])
    t0 = time.time()
    lam, _, iters, res = lobpcg(lat, invB, nev, block=14, tol=tol, seed=0)
    out = dict(workload=name, n=list(w["n"]), bloch=[float(x) for x in K], nev=nev, oracle_tol=tol,
               iterations=int(iters), max_residual=float(res.max()), seconds=round(time.time() - t0, 1),
               eigenvalues=[float(x) for x in lam])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "fcc64_eigs.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
