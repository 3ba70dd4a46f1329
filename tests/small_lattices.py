"""Deterministic small lattices for the oracle pins (dense matrices stay a few hundred wide)."""
import numpy as np

from oracle.lattice import make_lattice
from paper_1806_10284_gb300 import workloads as W


def j3_category(lat):
    acute = (lat.cos_alpha - lat.cos_gamma * lat.cos_beta) >= 0
    if acute:
        return 1 if lat.m1 <= lat.m2 else 2
    return 3 if lat.m1 + lat.m2 <= lat.n1 else 4


def generic(lat):
    return (0 < lat.m1 < lat.n1 and 0 < lat.m2 < lat.n1 and 0 < lat.m3 < lat.n2
            and lat.m1 != lat.m2 and lat.m1 + lat.m2 != lat.n1)


def random_triclinics(seed, count, generic_only=True, nmax=(8, 6, 4)):
    """Triclinic lattices with small grids; by default offsets strictly inside (0, n)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        L = [1.0, rng.uniform(0.5, 1.0), rng.uniform(0.5, 1.0)]
        ang = rng.uniform(50, 130, size=3)
        try:
            v = W.triclinic(L[0], L[1], L[2], *ang)
            n = (int(rng.integers(4, nmax[0] + 1)), int(rng.integers(3, nmax[1] + 1)),
                 int(rng.integers(2, nmax[2] + 1)))
            lat = make_lattice(v, n, rng.uniform(-3, 3, size=3))
        except (ValueError, ZeroDivisionError):
            continue
        if generic_only and not generic(lat):
            continue
        out.append(lat)
    return out


def category_cover(seed=11):
    """At least two generic lattices from each of the four J3 categories."""
    lats = random_triclinics(seed, 120)
    picked = {}
    for lat in lats:
        picked.setdefault(j3_category(lat), [])
        if len(picked[j3_category(lat)]) < 2:
            picked[j3_category(lat)].append(lat)
    assert sorted(picked) == [1, 2, 3, 4]
    return [lat for c in sorted(picked) for lat in picked[c]]


def named_small():
    """The workload lattices on small grids with their own Bloch vectors."""
    out = {}
    for name, n in (("sc16", (5, 4, 3)), ("fcc64", (6, 6, 6)), ("bcc96", (6, 6, 6)),
                    ("hex96", (6, 6, 5)), ("mono80", (5, 6, 4)), ("tri192", (6, 5, 4))):
        w = W.WORKLOADS[name]
        rng = np.random.default_rng(len(name))
        out[name] = make_lattice(w["vectors"], n, W.bloch_from_reduced(w["vectors"],
                                                                         rng.uniform(-.5, .5, 3)))
    return out
