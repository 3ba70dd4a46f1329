"""Lattice plan of Section 2.2 (oracle; test infrastructure only).

Given three primitive vectors (any Cartesian frame), grid sizes n1, n2, n3 and
a Bloch vector 2*pi*k, this module

* chooses the order of the vectors so that the conditions stated under the
  rotated matrix [a1' a2' a3'] of Section 2.2 hold (a1 the longest, and
  |a2| sin(gamma) > |a3| |cos(alpha) - cos(gamma) cos(beta)| / sin(gamma));
* computes the grid offsets m1, m2 (cases I and II on theta_gamma, theta_beta)
  and m3 (cases I and II on cos(alpha) - cos(gamma) cos(beta)) with the paper's
  rounding (floor when the fractional part is below 1/2, ceiling otherwise)
  and the corrected angles;
* forms the corrected vectors of eq. (transvec), the cell sizes l1, l2, l3 and
  the mesh sizes delta_x, delta_y, delta_z;
* derives the integer index shift of each lattice vector on the grid:
  a1 <-> (n1, 0, 0), a2 <-> (s1, n2, 0), a3 <-> (s2, s3, n3) with
  s1 = m1 - rho1 n1, s2 = m2 - rho2 n1, s3 = m3 - rho3 n2 (the x and y
  components of a2 and a3 in eq. (transvec) divided by delta_x, delta_y; the
  rho's are those defined next to eq. (J2) and eq. (J1));
* computes the Bloch fractions kappa_l = k . a_l of the quasi-periodic
  condition (eq. quasi_periodic) from the vectors as given.  The angle
  correction moves the vectors but keeps the reduced coordinates of k (the
  map Omega of Section 2.3), so kappa is taken from the input vectors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Orders tried, in this fixed sequence, when choosing which input vector plays
# a1, a2, a3.
PERMUTATIONS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
# Relative slack on the "a1 is the longest" test so that equal lengths tie.
LENGTH_SLACK = 1e-12


def paper_round(x: float) -> int:
    """Section 2.2 rounding: floor(x) if x - floor(x) < 1/2, else ceil(x)."""
    f = math.floor(x)
    return int(f) if x - f < 0.5 else int(f) + 1


@dataclass
class Lattice:
    n1: int
    n2: int
    n3: int
    perm: tuple
    lengths: tuple           # |a1|, |a2|, |a3| after ordering
    cos_in: tuple            # cos(gamma'), cos(beta'), cos(alpha') as given
    m1: int
    m2: int
    m3: int
    rho1: int
    rho2: int
    rho3: int
    cos_gamma: float         # corrected angles
    cos_beta: float
    cos_alpha: float
    a: np.ndarray            # 3x3, columns a1, a2, a3 of eq. (transvec)
    l1: float
    l2: float
    l3: float
    dx: float
    dy: float
    dz: float
    s1: int
    s2: int
    s3: int
    kappa: np.ndarray = field(default_factory=lambda: np.zeros(3))

    @property
    def n(self) -> int:
        return self.n1 * self.n2 * self.n3

    @property
    def shape(self) -> tuple:
        """numpy array shape of one grid field, x index fastest: (n3, n2, n1)."""
        return (self.n3, self.n2, self.n1)


def _angles(v):
    L = [float(np.linalg.norm(x)) for x in v]
    cg = float(np.dot(v[0], v[1]) / (L[0] * L[1]))
    cb = float(np.dot(v[0], v[2]) / (L[0] * L[2]))
    ca = float(np.dot(v[1], v[2]) / (L[1] * L[2]))
    return L, cg, cb, ca


def choose_order(vectors) -> tuple:
    """First permutation (in PERMUTATIONS order) meeting the Section 2.2 conditions."""
    vecs = [np.asarray(x, dtype=np.float64) for x in vectors]
    for perm in PERMUTATIONS:
        v = [vecs[i] for i in perm]
        L, cg, cb, ca = _angles(v)
        if L[0] < L[1] * (1 - LENGTH_SLACK) or L[0] < L[2] * (1 - LENGTH_SLACK):
            continue
        sg = math.sqrt(max(0.0, 1.0 - cg * cg))
        if sg > 0.0 and L[1] * sg > L[2] * abs(ca - cg * cb) / sg:
            return perm
    raise ValueError("no ordering of the lattice vectors meets the Section 2.2 conditions")


def make_lattice(vectors, n, bloch) -> Lattice:
    """Build the corrected lattice for grid n = (n1, n2, n3).

    ``vectors``: three primitive vectors (rows), any Cartesian frame.
    ``n``: grid sizes along the chosen a1, a2, a3.
    ``bloch``: the Bloch vector 2*pi*k in the same Cartesian frame.
    """
    n1, n2, n3 = (int(x) for x in n)
    vecs = [np.asarray(x, dtype=np.float64) for x in vectors]
    vol = abs(float(np.linalg.det(np.array(vecs))))
    if vol <= 1e-12 * float(np.prod([np.linalg.norm(x) for x in vecs])):
        raise ValueError("lattice vectors are linearly dependent")
    perm = choose_order(vecs)
    v = [vecs[i] for i in perm]
    (L1, L2, L3), cg_in, cb_in, ca_in = _angles(v)

    dx = L1 / n1
    # m1, cases I and II on theta_gamma'.
    if cg_in >= 0.0:
        m1 = paper_round(L2 * cg_in / dx)
        cos_g = m1 * dx / L2
        rho1 = 0
    else:
        m1 = paper_round((L1 + L2 * cg_in) / dx)
        cos_g = (m1 * dx - L1) / L2
        rho1 = 1
    sin_g = math.sqrt(L2 * L2 - (L2 * cos_g) ** 2) / L2
    l2 = L2 * sin_g
    dy = l2 / n2
    # m2, cases I and II on theta_beta'.
    if cb_in >= 0.0:
        m2 = paper_round(L3 * cb_in / dx)
        cos_b = m2 * dx / L3
        rho2 = 0
    else:
        m2 = paper_round((L1 + L3 * cb_in) / dx)
        cos_b = (m2 * dx - L1) / L3
        rho2 = 1
    # m3, cases I and II on cos(alpha') - cos(gamma) cos(beta) (corrected gamma, beta).
    d = ca_in - cos_g * cos_b
    if d >= 0.0:
        m3 = paper_round(L3 / dy * d / sin_g)
        cos_a = m3 * dy / L3 * sin_g + cos_g * cos_b
        rho3 = 0
    else:
        m3 = paper_round((L2 * sin_g ** 2 + L3 * d) / (dy * sin_g))
        cos_a = (m3 * dy * sin_g - L2 * sin_g ** 2) / L3 + cos_g * cos_b
        rho3 = 1
    # eq. (transvec)
    zz = 1.0 - cos_g ** 2 - cos_b ** 2 - cos_a ** 2 + 2.0 * cos_g * cos_b * cos_a
    if zz <= 0.0:
        raise ValueError("corrected lattice is degenerate")
    a = np.array([
        [L1, L2 * cos_g, L3 * cos_b],
        [0.0, L2 * sin_g, L3 * (cos_a - cos_g * cos_b) / sin_g],
        [0.0, 0.0, L3 * math.sqrt(zz) / sin_g],
    ])
    l1, l3 = L1, a[2, 2]
    dz = l3 / n3
    s1 = m1 - rho1 * n1
    s2 = m2 - rho2 * n1
    s3 = m3 - rho3 * n2
    bloch = np.asarray(bloch, dtype=np.float64)
    kappa = np.array([float(np.dot(bloch, x)) / (2.0 * math.pi) for x in v])
    return Lattice(n1=n1, n2=n2, n3=n3, perm=perm, lengths=(L1, L2, L3),
                   cos_in=(cg_in, cb_in, ca_in), m1=m1, m2=m2, m3=m3,
                   rho1=rho1, rho2=rho2, rho3=rho3, cos_gamma=cos_g,
                   cos_beta=cos_b, cos_alpha=cos_a, a=a, l1=l1, l2=l2, l3=l3,
                   dx=dx, dy=dy, dz=dz, s1=s1, s2=s2, s3=s3, kappa=kappa)


def with_kappa(lat: Lattice, kappa) -> Lattice:
    """Same lattice, other Bloch fractions kappa_l = k . a_l."""
    out = Lattice(**{f: getattr(lat, f) for f in lat.__dataclass_fields__})
    out.kappa = np.asarray(kappa, dtype=np.float64).copy()
    return out


def reciprocal(lat: Lattice) -> np.ndarray:
    """Reciprocal vectors [b1 b2 b3] = 2 pi [a1 a2 a3]^{-T} (Section 2.3)."""
    return 2.0 * math.pi * np.linalg.inv(lat.a).T
