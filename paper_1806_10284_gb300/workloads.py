"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds no arithmetic of the method itself.  It describes the
workloads (primitive vectors, grid sizes, Bloch vectors, inclusion shapes)
and samples the permittivity on the Yee points of a grid whose geometry the
caller supplies (grid sizes, the integer index shifts of the lattice vectors,
the mesh sizes and the order chosen for the vectors), so the same sampler
serves inputs to the CUDA library and to the CPU oracle.

Grid geometry (``Geometry``): the point with grid coordinates (gx, gy, gz) sits
at (gx dx, gy dy, gz dz); the lattice vectors are the grid displacements
a1 = (n1, 0, 0), a2 = (s1, n2, 0), a3 = (s2, s3, n3).  The E_l samples sit at
(i + 1/2, j, k), (i, j + 1/2, k), (i, j, k + 1/2) (Section 3 of the paper).
Arrays of one field have numpy shape (n3, n2, n1), x index fastest.

The paper's experiments use 120^3 grids, eps = 13 inclusions (spheres and
cylinders, r/a = 0.15) in air, and the 10 smallest eigenvalues per Bloch
vector; the recipes below follow that shape at the grid sizes of the five
workloads, with seeds fixed in ``WORKLOADS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Geometry:
    n: tuple          # (n1, n2, n3)
    s: tuple          # (s1, s2, s3)
    delta: tuple      # (dx, dy, dz)
    perm: tuple       # input vector index used for canonical a1, a2, a3

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def lattice_matrix(self):
        """Columns a1, a2, a3 in Cartesian units (from the grid description)."""
        n1, n2, n3 = self.n
        s1, s2, s3 = self.s
        N = np.array([[n1, s1, s2], [0, n2, s3], [0, 0, n3]], dtype=np.float64)
        return np.diag(self.delta) @ N


# ---------------------------------------------------------------------------
# Primitive vectors (rows) of the lattices used by the workloads.
# ---------------------------------------------------------------------------

def simple_cubic(a=1.0):
    return np.eye(3) * a


def fcc(a=1.0):
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def bcc(a=1.0):
    return 0.5 * a * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])


def hexagonal(a=1.0, c_over_a=1.6):
    return a * np.array([[1.0, 0.0, 0.0], [-0.5, math.sqrt(3.0) / 2.0, 0.0],
                         [0.0, 0.0, c_over_a]])


def base_centred_monoclinic(a=1.0, b=1.2, c=0.9, beta_deg=105.0):
    """C-centred monoclinic, unique axis b: primitive (A-B)/2, (A+B)/2, C."""
    be = math.radians(beta_deg)
    A = np.array([a, 0.0, 0.0])
    B = np.array([0.0, b, 0.0])
    C = np.array([c * math.cos(be), 0.0, c * math.sin(be)])
    return np.array([(A - B) / 2.0, (A + B) / 2.0, C])


def triclinic(l1, l2, l3, alpha_deg, beta_deg, gamma_deg):
    """a1 along x, a2 in the xy plane; alpha = (a2, a3), beta = (a1, a3), gamma = (a1, a2)."""
    al, be, ga = (math.radians(x) for x in (alpha_deg, beta_deg, gamma_deg))
    a1 = np.array([l1, 0.0, 0.0])
    a2 = l2 * np.array([math.cos(ga), math.sin(ga), 0.0])
    cy = (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
    cz = math.sqrt(1.0 - math.cos(be) ** 2 - cy ** 2)
    a3 = l3 * np.array([math.cos(be), cy, cz])
    return np.array([a1, a2, a3])


def bloch_from_reduced(vectors, reduced):
    """Cartesian Bloch vector 2 pi k = sum_l c_l b_l with b = 2 pi A^{-T} (A rows = vectors)."""
    A = np.asarray(vectors, dtype=np.float64)
    return 2.0 * math.pi * np.linalg.solve(A, np.asarray(reduced, dtype=np.float64))


# ---------------------------------------------------------------------------
# Permittivity sampling on the Yee points.
# ---------------------------------------------------------------------------

YEE_OFFSETS = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5))


def yee_points(geom: Geometry, comp: int, k0: int = 0, k1: int | None = None):
    """Cartesian coordinates (3, k1-k0, n2, n1) of the E_comp samples in z-planes [k0, k1)."""
    n1, n2, n3 = geom.n
    k1 = n3 if k1 is None else k1
    ox, oy, oz = YEE_OFFSETS[comp]
    gz, gy, gx = np.meshgrid(np.arange(k0, k1) + oz, np.arange(n2) + oy,
                             np.arange(n1) + ox, indexing="ij")
    dx, dy, dz = geom.delta
    return np.stack([gx * dx, gy * dy, gz * dz])


def _to_fractional(geom: Geometry, X):
    """Fractional coordinates (w.r.t. the canonical a1, a2, a3) of Cartesian points X (3, ...)."""
    A = geom.lattice_matrix()
    flat = X.reshape(3, -1)
    return np.linalg.solve(A, flat).reshape(X.shape)


def _canonical_frac(geom: Geometry, frac_in):
    """Fractional coordinates given w.r.t. the input vectors, reordered to canonical axes."""
    f = np.asarray(frac_in, dtype=np.float64)
    return np.array([f[geom.perm[0]], f[geom.perm[1]], f[geom.perm[2]]])


def _min_image_disp(geom: Geometry, X, center_frac):
    """Cartesian displacement from the nearest periodic image of a centre to each point.

    Returns (27, 3, ...) candidate displacements; callers take the minimum of
    their own distance measure over axis 0.
    """
    A = geom.lattice_matrix()
    F = _to_fractional(geom, X)
    d = F - center_frac.reshape((3,) + (1,) * (F.ndim - 1))
    d = d - np.round(d)
    out = []
    for s1 in (-1, 0, 1):
        for s2 in (-1, 0, 1):
            for s3 in (-1, 0, 1):
                df = d + np.array([s1, s2, s3], dtype=np.float64).reshape((3,) + (1,) * (d.ndim - 1))
                out.append(np.tensordot(A, df, axes=(1, 0)))
    return np.stack(out)


def _sphere_mask(geom, X, center_frac, radius):
    D = _min_image_disp(geom, X, center_frac)
    return np.min(np.sum(D * D, axis=1), axis=0) <= radius * radius


def _rod_mask(geom, X, center_frac, radius, axis):
    """Cylinder along canonical lattice vector ``axis`` through the centre."""
    A = geom.lattice_matrix()
    u = A[:, axis] / np.linalg.norm(A[:, axis])
    D = _min_image_disp(geom, X, center_frac)
    along = np.tensordot(u, D, axes=(0, 1))                     # (27, ...)
    perp2 = np.sum(D * D, axis=1) - along ** 2
    return np.min(perp2, axis=0) <= radius * radius


def _ellipsoid_mask(geom, X, center_frac, semi_axes, rot):
    D = _min_image_disp(geom, X, center_frac)                  # (27, 3, ...)
    local = np.einsum("ij,kj...->ki...", rot.T, D)
    q = sum((local[:, i] / semi_axes[i]) ** 2 for i in range(3))
    return np.min(q, axis=0) <= 1.0


def sample_inclusions(geom: Geometry, shapes, eps_in, eps_out=1.0):
    """B_1, B_2, B_3 (each (n3, n2, n1)) for a union of inclusions.

    ``shapes``: list of dicts, kind "sphere" (center, radius), "rod"
    (center, radius, axis given w.r.t. the input vectors) or "ellipsoid"
    (center, semi_axes, rot); centres in fractional coordinates of the input
    vectors.
    """
    out = []
    n1, n2, n3 = geom.n
    slab = max(1, (1 << 16) // (n1 * n2))
    for comp in range(3):
        inside = np.zeros(geom.shape, dtype=bool)
        for k0 in range(0, n3, slab):
            k1 = min(n3, k0 + slab)
            X = yee_points(geom, comp, k0, k1)
            m = np.zeros(X.shape[1:], dtype=bool)
            for sh in shapes:
                c = _canonical_frac(geom, sh["center"])
                if sh["kind"] == "sphere":
                    m |= _sphere_mask(geom, X, c, sh["radius"])
                elif sh["kind"] == "rod":
                    m |= _rod_mask(geom, X, c, sh["radius"], geom.perm.index(sh["axis"]))
                elif sh["kind"] == "ellipsoid":
                    m |= _ellipsoid_mask(geom, X, c, np.asarray(sh["semi_axes"]),
                                         np.asarray(sh["rot"]))
                else:
                    raise ValueError(sh["kind"])
            inside[k0:k1] = m
        out.append(np.where(inside, eps_in, eps_out).astype(np.float64))
    return out


def _input_cartesian(geom: Geometry, vectors, X):
    """Cartesian coordinates, in the frame of the input vectors, of canonical-frame points X
    (3, ...): fractional coordinates w.r.t. the canonical a1, a2, a3, mapped back to the
    input vectors (the structure is placed in fractional coordinates of the lattice)."""
    F = _to_fractional(geom, X)
    Fin = np.empty_like(F)
    for l in range(3):
        Fin[geom.perm[l]] = F[l]
    return np.tensordot(np.asarray(vectors, dtype=np.float64).T, Fin, axes=(1, 0))


def gyroid_value(X):
    """The gyroid's approximating function sin X cos Y + sin Y cos Z + sin Z cos X,
    (X, Y, Z) = 2 pi (x, y, z), at Cartesian points (3, ...) in units of the cubic cell."""
    x, y, z = (2.0 * math.pi * X[i] for i in range(3))
    return np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)


def sample_level_set(geom: Geometry, vectors, fn, level, eps_in, eps_out=1.0):
    """B_1, B_2, B_3 with eps_in at the Yee points where fn(X) > level, X Cartesian in the
    frame of the input vectors, and eps_out elsewhere."""
    out = []
    n1, n2, n3 = geom.n
    slab = max(1, (1 << 18) // (n1 * n2))
    for comp in range(3):
        B = np.empty(geom.shape, dtype=np.float64)
        for k0 in range(0, n3, slab):
            k1 = min(n3, k0 + slab)
            X = _input_cartesian(geom, vectors, yee_points(geom, comp, k0, k1))
            B[k0:k1] = np.where(fn(X) > level, eps_in, eps_out)
        out.append(B)
    return out


def supercell(vectors, n, reps):
    """Primitive vectors (rows N_l a_l) and grid (N_l n_l) of the supercell of reps =
    (N_1, N_2, N_3) primitive cells.  Grid sizes and reps follow the canonical axes,
    so the helper serves lattices whose canonical order is the input order in both
    cells (e.g. simple cubic, N_1 >= N_2 >= N_3)."""
    V = np.asarray(vectors, dtype=np.float64)
    return V * np.asarray(reps, dtype=np.float64)[:, None], tuple(int(a) * int(b) for a, b in zip(n, reps))


def tile_eps(B, reps, empty_cells=(), eps_out=1.0):
    """The primitive-cell B_1, B_2, B_3 (each (n3, n2, n1)) repeated reps = (N_1, N_2, N_3)
    times; each primitive cell (i, j, k) in ``empty_cells`` is set to eps_out (a vacancy:
    the inclusions of that cell removed)."""
    N1, N2, N3 = reps
    out = []
    for b in B:
        n3, n2, n1 = b.shape
        t = np.tile(b, (N3, N2, N1))
        for (i, j, k) in empty_cells:
            t[k * n3:(k + 1) * n3, j * n2:(j + 1) * n2, i * n1:(i + 1) * n1] = eps_out
        out.append(t)
    return out


def smooth_field_eps(n, seed, sigma_vox=3.0, contrast=12.0, steep=8.0):
    """eps on grid nodes: 1 + contrast * sigmoid(steep * g), g a Gaussian-filtered
    (sigma in voxels, periodic) unit-variance white-noise field; then B_l at
    the Yee edge midpoints as the mean of the edge's two end nodes (periodic in
    the index box).  Returns (eps_nodes, [B1, B2, B3])."""
    n1, n2, n3 = n
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n3, n2, n1))
    kz = np.fft.fftfreq(n3)[:, None, None]
    ky = np.fft.fftfreq(n2)[None, :, None]
    kx = np.fft.fftfreq(n1)[None, None, :]
    filt = np.exp(-2.0 * (math.pi * sigma_vox) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    g = (g - g.mean()) / g.std()
    eps = 1.0 + contrast / (1.0 + np.exp(-steep * g))
    B1 = 0.5 * (eps + np.roll(eps, -1, axis=2))
    B2 = 0.5 * (eps + np.roll(eps, -1, axis=1))
    B3 = 0.5 * (eps + np.roll(eps, -1, axis=0))
    return eps, [B1, B2, B3]


def random_inclusions(seed, vectors, count_range=(3, 6), radius_frac=(0.1, 0.25)):
    """3-6 spheres or rods (chosen by the seed), radii U(0.1, 0.25) x shortest |a_l|."""
    rng = np.random.default_rng(seed)
    shortest = float(min(np.linalg.norm(v) for v in vectors))
    count = int(rng.integers(count_range[0], count_range[1] + 1))
    shapes = []
    for _ in range(count):
        kind = "sphere" if rng.random() < 0.5 else "rod"
        r = float(rng.uniform(*radius_frac)) * shortest
        c = rng.random(3)
        if kind == "sphere":
            shapes.append(dict(kind="sphere", center=c, radius=r))
        else:
            shapes.append(dict(kind="rod", center=c, radius=r, axis=int(rng.integers(0, 3))))
    return shapes


def random_ellipsoids(seed, count=8, semi=(0.08, 0.2)):
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(count):
        qv = rng.standard_normal(4)
        qv /= np.linalg.norm(qv)
        w, x, y, z = qv
        rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        shapes.append(dict(kind="ellipsoid", center=rng.random(3),
                           semi_axes=rng.uniform(*semi, size=3), rot=rot))
    return shapes


def bz_path_reduced(points_total=60):
    """Piecewise-linear path Gamma -> (1/2,0,0) -> (1/2,1/2,0) -> (1/2,1/2,1/2) -> Gamma in
    reduced reciprocal coordinates, equal point counts per segment, Gamma once."""
    corners = np.array([[0, 0, 0], [0.5, 0, 0], [0.5, 0.5, 0], [0.5, 0.5, 0.5], [0, 0, 0]],
                       dtype=np.float64)
    seg = points_total // 4
    pts = []
    for s in range(4):
        for t in range(seg):
            pts.append(corners[s] + (corners[s + 1] - corners[s]) * t / seg)
    return np.array(pts)


def random_reduced_kpoints(seed, count, min_norm=0.05):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        c = rng.uniform(-0.5, 0.5, size=3)
        if np.linalg.norm(c) >= min_norm:
            out.append(c)
    return np.array(out)


def random_block(seed, n, m, dtype=np.complex128):
    """m seeded complex normal vectors of length 2n (A_r coordinates), shape (m, 2n)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((m, 2 * n)) + 1j * rng.standard_normal((m, 2 * n))
    return x.astype(dtype)


# ---------------------------------------------------------------------------
# The workloads.
# ---------------------------------------------------------------------------

WORKLOADS = {
    "sc16": dict(
        desc="simple cubic a=1, 16^3, eps=13 sphere r=0.25 centred, K=(pi)(0.5,0.1,0.2), "
             "10 bands, complex128, residual 1e-10",
        vectors=simple_cubic(), n=(16, 16, 16),
        bloch=[np.pi * np.array([0.5, 0.1, 0.2])],
        shapes=[dict(kind="sphere", center=np.array([0.5, 0.5, 0.5]), radius=0.25)],
        eps_in=13.0, nev=10, tol=1e-10, precision="fp64"),
    "fcc64": dict(
        desc="FCC primitive (a/2)(0,1,1),(a/2)(1,0,1),(a/2)(1,1,0), 64^3, eps=13 spheres "
             "r=0.325*sqrt(3)/4 at diamond sites (0,0,0),(1/4,1/4,1/4), 10 bands at one k, "
             "complex64 apply, FP64 Rayleigh-Ritz and refinement to residual 1e-8",
        vectors=fcc(), n=(64, 64, 64),
        reduced_k=[np.array([0.3, 0.2, 0.1])],
        shapes=[dict(kind="sphere", center=np.zeros(3), radius=0.325 * math.sqrt(3) / 4),
                dict(kind="sphere", center=np.full(3, 0.25), radius=0.325 * math.sqrt(3) / 4)],
        eps_in=13.0, nev=10, tol=1e-8, precision="mixed"),
    "bcc96": dict(desc="BCC 96^3, seeded eps=12 rods/spheres, 60-point BZ path",
                  vectors=bcc(), n=(96, 96, 96), path=60, seed=301, eps_in=12.0,
                  nev=10, tol=1e-8, precision="mixed"),
    "hex96": dict(desc="hexagonal c/a=1.6, 96x96x80, seeded eps=12 rods/spheres, 60-point path",
                  vectors=hexagonal(), n=(96, 96, 80), path=60, seed=302, eps_in=12.0,
                  nev=10, tol=1e-8, precision="mixed"),
    "mono80": dict(desc="base-centred monoclinic beta=105 deg, 80x96x64, seeded eps=12 "
                        "rods/spheres, 60-point path",
                   vectors=base_centred_monoclinic(), n=(80, 96, 64), path=60, seed=303,
                   eps_in=12.0, nev=10, tol=1e-8, precision="mixed"),
    "sc48grad": dict(desc="simple cubic 48^3, eps = 1 + 12 sigmoid(8 g), 8 k-points, "
                          "objective (lambda6-lambda5)/lambda5",
                     vectors=simple_cubic(), n=(48, 48, 48), kseed=404, nk=8, seed=401,
                     nev=6, tol=1e-8, precision="mixed"),
    "gyroid96": dict(desc="BCC a=1, 96^3, gyroid sin X cos Y + sin Y cos Z + sin Z cos X > 1.1 "
                          "filled with eps (13; the sweep takes 3..30), 10 bands",
                     vectors=bcc(), n=(96, 96, 96), level=1.1, eps_in=13.0,
                     eps_sweep=(3.0, 5.0, 8.0, 13.0, 18.0, 24.0, 30.0),
                     reduced_k=[np.array([0.5, 0.5, 0.0]), np.array([0.25, 0.25, 0.25])],
                     nev=10, tol=1e-8, precision="mixed"),
    "scvac": dict(desc="simple cubic supercell of 2 x 2 x 2 cells (64^3), eps=13 sphere r=0.25 "
                       "per cell, one cell's sphere removed (a vacancy), 10 bands",
                  vectors=simple_cubic(), n=(32, 32, 32), reps=(2, 2, 2), vacancy=[(0, 0, 0)],
                  shapes=[dict(kind="sphere", center=np.array([0.5, 0.5, 0.5]), radius=0.25)],
                  bloch=[np.pi * np.array([0.5, 0.1, 0.2])],
                  eps_in=13.0, nev=10, tol=1e-8, precision="mixed"),
    "tri192": dict(desc="triclinic |a|=1,1.1,1.25, angles 80/85/95 deg, 192^3, 8 seeded "
                        "ellipsoids eps=13, 20 bands at 4 k-points",
                   vectors=triclinic(1.0, 1.1, 1.25, 80.0, 85.0, 95.0), n=(192, 192, 192),
                   kseed=505, nk=4, seed=501, eps_in=13.0, nev=20, tol=1e-8,
                   precision="mixed"),
}


def bloch_vectors(name):
    """List of Cartesian Bloch vectors 2 pi k for a workload."""
    w = WORKLOADS[name]
    if "bloch" in w:
        return [np.asarray(b, dtype=np.float64) for b in w["bloch"]]
    if "reduced_k" in w:
        return [bloch_from_reduced(w["vectors"], c) for c in w["reduced_k"]]
    if "path" in w:
        return [bloch_from_reduced(w["vectors"], c) for c in bz_path_reduced(w["path"])]
    return [bloch_from_reduced(w["vectors"], c)
            for c in random_reduced_kpoints(w["kseed"], w["nk"])]


def eps_for(name, geom: Geometry, eps_in=None):
    """B_1, B_2, B_3 for a workload on the supplied grid geometry (for the supercell
    workload: the geometry of its primitive cell; the result is the tiled supercell).
    ``eps_in`` overrides the workload's inclusion permittivity (the eps sweep)."""
    w = WORKLOADS[name]
    e_in = w.get("eps_in") if eps_in is None else eps_in
    if name == "sc48grad":
        return smooth_field_eps(geom.n, w["seed"])[1]
    if "level" in w:
        return sample_level_set(geom, w["vectors"], gyroid_value, w["level"], e_in)
    if "reps" in w:
        return tile_eps(sample_inclusions(geom, w["shapes"], e_in), w["reps"], w["vacancy"])
    if "shapes" in w:
        shapes = w["shapes"]
    elif name == "tri192":
        shapes = random_ellipsoids(w["seed"])
    else:
        shapes = random_inclusions(w["seed"], w["vectors"])
    return sample_inclusions(geom, shapes, e_in)
