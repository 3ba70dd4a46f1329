"""GPU parity of the A_r apply and the lift against the CPU oracle (through the C ABI).

Tolerances (max-norm, relative to the largest |entry| of the oracle result):
  complex128: 1e-11 (FFT round-off ~ log2(n) eps64 with margin);
  complex64 : 2e-5  (FFT round-off ~ log2(n) eps32 ~ 1e-6, twist/Lambda/Pi in float,
              with margin); the mixed-precision eigenvalue tolerance is 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.lattice import make_lattice, with_kappa
from oracle.nfsep import apply_Ar, lift, bases, basis_margin, G_TOL
from oracle.spectral import lambdas
from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 2e-5

CASES = [
    ("sc16", (16, 16, 16)),
    ("sc16", (5, 6, 4)),         # ragged: n1 below the 16-wide x tile
    ("fcc64", (12, 10, 6)),      # radix 3 and 5
    ("bcc96", (24, 24, 24)),     # obtuse case, rho = (1,1,1)
    ("hex96", (20, 12, 10)),     # reordered vectors, radix 5
    ("mono80", (20, 24, 16)),
    ("tri192", (18, 15, 8)),     # triclinic, ragged x tiles
    ("fcc64", (2, 2, 2)),        # smallest grid
    # lengths with fixed-length complex64 passes
    ("tri192", (32, 32, 48)),    # XY 32x32, Z 48
    ("mono80", (48, 48, 32)),    # XY 48x48, Z 32
    ("hex96", (20, 32, 16)),     # Z 16 with a ragged x tile, generic XY
    ("bcc96", (80, 96, 16)),     # XY 80x96
    ("tri192", (128, 128, 4)),   # plane too large for shared memory: split y / x / y passes
]


MARGIN = {"c128": 1e-9, "c64": 1e-5}   # distance of every frequency from the basis switch


def _setup(name, n, seed=0, kred=None, margin=1e-5):
    """Lattice, context and eps; with a random k, the first seed whose frequencies all keep
    ``margin`` from the reference-vector switch (both sides then take the same branch)."""
    w = W.WORKLOADS[name]
    for s in range(seed, seed + 50):
        rng = np.random.default_rng(s)
        K = W.bloch_from_reduced(w["vectors"], rng.uniform(-0.5, 0.5, 3) if kred is None else kred)
        lat = make_lattice(w["vectors"], n, K)
        if kred is not None or basis_margin(lat) > margin:
            break
    else:
        raise AssertionError("no Bloch vector clear of the basis switch")
    ctx = fame.Context(w["vectors"], n, K)
    B = [1.0 + 12.0 * (rng.random(lat.shape) < 0.3) for _ in range(3)]
    ctx.set_eps(*B)
    invB = np.stack([1.0 / b for b in B])
    return lat, ctx, invB, rng


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1806_10284_gb300 import build
    build.build()
    fame.load()


@pytest.mark.parametrize("name,n", CASES)
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_apply_matches_oracle(name, n, prec):
    lat, ctx, invB, rng = _setup(name, n, margin=MARGIN[prec])
    assert basis_margin(lat) > MARGIN[prec]
    m = 3
    y = rng.standard_normal((m, 2 * lat.n)) + 1j * rng.standard_normal((m, 2 * lat.n))
    dt = torch.complex128 if prec == "c128" else torch.complex64
    got = ctx.apply(torch.as_tensor(y, dtype=dt, device="cuda")).cpu().numpy()
    for j in range(m):
        ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < (TOL64 if prec == "c128" else TOL32), (name, n, prec, j)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_apply_gamma_point(prec):
    """2 pi k = 0: the zero-frequency coordinates map to zero (Sigma_r = 0 there)."""
    lat, ctx, invB, rng = _setup("fcc64", (8, 8, 8), kred=np.zeros(3))
    y = rng.standard_normal((1, 2 * lat.n)) + 1j * rng.standard_normal((1, 2 * lat.n))
    dt = torch.complex128 if prec == "c128" else torch.complex64
    got = ctx.apply(torch.as_tensor(y, dtype=dt, device="cuda")).cpu().numpy()[0]
    ref = apply_Ar(lat, y[0].reshape((2,) + lat.shape), invB).ravel()
    assert _rel(got, ref) < (TOL64 if prec == "c128" else TOL32)
    assert abs(got[0]) == 0.0 and abs(got[lat.n]) == 0.0


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [(8, 8, 8),        # generic passes
                               (16, 16, 16),     # fixed-length Z 16 and XY 16x16 (complex64)
                               (64, 64, 16)])    # fixed-length XY 64x64, 512-thread form
def test_apply_basis_switch_points(n, prec):
    """Simple cubic at Gamma: Lambda parallel to (1,1,1) on the diagonal p = q = r, where
    the paper's range basis is undefined; both sides take the alternate reference vector
    there (the decision is taken in FP64 and shared by the complex64 kernels)."""
    lat, ctx, invB, rng = _setup("sc16", n, kred=np.zeros(3))
    L = np.stack(lambdas(lat))
    Lq = np.sum(np.abs(L) ** 2, axis=0)
    g = 3.0 * Lq - np.abs(L.sum(axis=0)) ** 2
    assert np.count_nonzero((Lq > 0) & (g < G_TOL * 3.0 * Lq)) > 0       # alternate reference vector in use
    if n[0] == n[1] == n[2]:
        assert np.count_nonzero((Lq > 0) & (g <= 1e-12 * Lq)) >= n[0] - 1  # exact degeneracies present
    y = rng.standard_normal((2, 2 * lat.n)) + 1j * rng.standard_normal((2, 2 * lat.n))
    dt = torch.complex128 if prec == "c128" else torch.complex64
    got = ctx.apply(torch.as_tensor(y, dtype=dt, device="cuda")).cpu().numpy()
    for j in range(2):
        ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < (TOL64 if prec == "c128" else TOL32)


@pytest.mark.parametrize("name,n", [("fcc64", (16, 16, 16)), ("bcc96", (24, 24, 24)),
                                    ("tri192", (32, 32, 48))])
def test_apply_complex64_without_basis_margin(name, n):
    """Complex64 applies at Bloch vectors chosen with no distance from the basis switch
    (frequencies may sit on either side of it, arbitrarily close)."""
    lat, ctx, invB, rng = _setup(name, n, seed=17, margin=0.0)
    y = rng.standard_normal((2, 2 * lat.n)) + 1j * rng.standard_normal((2, 2 * lat.n))
    got = ctx.apply(torch.as_tensor(y, dtype=torch.complex64, device="cuda")).cpu().numpy()
    for j in range(2):
        ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < TOL32


@pytest.mark.parametrize("m", [1, 7, 40])
def test_apply_block_sizes(m):
    lat, ctx, invB, rng = _setup("hex96", (10, 12, 6), seed=m)
    y = rng.standard_normal((m, 2 * lat.n)) + 1j * rng.standard_normal((m, 2 * lat.n))
    got = ctx.apply(torch.as_tensor(y, device="cuda")).cpu().numpy()
    for j in sorted({0, m // 2, m - 1}):
        ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < TOL64


@pytest.mark.parametrize("m", [1, 7, 40])
def test_apply_block_sizes_complex64(m):
    """Several vectors per block in the fixed-length Z passes."""
    lat, ctx, invB, rng = _setup("fcc64", (16, 16, 32), seed=m)
    y = rng.standard_normal((m, 2 * lat.n)) + 1j * rng.standard_normal((m, 2 * lat.n))
    got = ctx.apply(torch.as_tensor(y, dtype=torch.complex64, device="cuda")).cpu().numpy()
    for j in sorted({0, m // 2, m - 1}):
        ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < TOL32


@pytest.mark.parametrize("n", [(12, 10, 8), (16, 16, 16)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_lift_matches_oracle(prec, n):
    lat, ctx, invB, rng = _setup("tri192", n, seed=3)
    y = rng.standard_normal((2, 2 * lat.n)) + 1j * rng.standard_normal((2, 2 * lat.n))
    dt = torch.complex128 if prec == "c128" else torch.complex64
    got = ctx.lift(torch.as_tensor(y, dtype=dt, device="cuda")).cpu().numpy()
    for j in range(2):
        ref = lift(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < (TOL64 if prec == "c128" else TOL32)


def test_plan_matches_oracle_on_device():
    for name in ("fcc64", "bcc96", "hex96", "mono80", "tri192"):
        w = W.WORKLOADS[name]
        K = W.bloch_vectors(name)[0]
        ctx = fame.Context(w["vectors"], w["n"], K)
        lat = make_lattice(w["vectors"], w["n"], K)
        p = ctx.plan()
        assert p["s"] == (lat.s1, lat.s2, lat.s3) and p["perm"] == tuple(lat.perm)
        np.testing.assert_allclose(p["kappa"], lat.kappa, atol=1e-13)


def test_set_k_rebuilds_twists():
    lat, ctx, invB, rng = _setup("mono80", (10, 12, 8), seed=5)
    w = W.WORKLOADS["mono80"]
    K2 = W.bloch_from_reduced(w["vectors"], [0.1, 0.4, -0.3])
    ctx.set_k(K2)
    lat2 = make_lattice(w["vectors"], (10, 12, 8), K2)
    y = rng.standard_normal((1, 2 * lat.n)) + 1j * rng.standard_normal((1, 2 * lat.n))
    got = ctx.apply(torch.as_tensor(y, device="cuda")).cpu().numpy()[0]
    ref = apply_Ar(lat2, y[0].reshape((2,) + lat.shape), invB).ravel()
    assert _rel(got, ref) < TOL64


@pytest.mark.parametrize("name,m", [("fcc64", 16), ("bcc96", 16), ("hex96", 16), ("mono80", 16),
                                    ("tri192", 4)])
def test_homogeneous_closed_form_full_size(name, m):
    """B = c: A_r y = (Lambda_q / c) y at the workload's full grid (192^3 takes the split
    y / x / y passes), m vectors per block."""
    w = W.WORKLOADS[name]
    K = W.bloch_vectors(name)[0]
    lat = make_lattice(w["vectors"], w["n"], K)
    ctx = fame.Context(w["vectors"], w["n"], K)
    c = 6.0
    ones = np.full(lat.n, c)
    ctx.set_eps(ones, ones, ones)
    Lq = (bases(lat)[3] ** 2).ravel()
    lam = np.concatenate([Lq, Lq]) / c
    g = torch.Generator(device="cuda").manual_seed(0)
    y = torch.randn((m, 2 * lat.n), dtype=torch.complex128, device="cuda", generator=g)
    lam_t = torch.as_tensor(lam, device="cuda")
    for dt, tol in ((torch.complex128, TOL64), (torch.complex64, TOL32)):
        yy = y.to(dt)
        got = ctx.apply(yy)
        ref = lam_t[None, :] * yy.to(torch.complex128)
        err = float((got.to(torch.complex128) - ref).abs().max() / ref.abs().max())
        assert err < tol, (name, dt, err)


def test_full_size_sampled_vectors():
    """FCC 64^3, block of 16 in the bench's launch configuration: two of the 16 outputs
    compared element by element with the oracle."""
    w = W.WORKLOADS["fcc64"]
    K = W.bloch_vectors("fcc64")[0]
    lat = make_lattice(w["vectors"], w["n"], K)
    ctx = fame.Context(w["vectors"], w["n"], K)
    geom = fame.geometry_of(fame.plan_lattice(w["vectors"], w["n"], K))
    B = W.eps_for("fcc64", geom)
    ctx.set_eps(*B)
    invB = np.stack([1.0 / b for b in B])
    rng = np.random.default_rng(11)
    y = (rng.standard_normal((16, 2 * lat.n)) + 1j * rng.standard_normal((16, 2 * lat.n)))
    for dt, tol in ((torch.complex64, TOL32), (torch.complex128, TOL64)):
        got = ctx.apply(torch.as_tensor(y, dtype=dt, device="cuda")).cpu().numpy()
        for j in (0, 13):
            ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
            assert _rel(got[j], ref) < tol


def test_api_errors():
    w = W.WORKLOADS["sc16"]
    ctx = fame.Context(w["vectors"], (8, 8, 8), np.zeros(3))
    y = torch.zeros((1, 2 * 512), dtype=torch.complex64, device="cuda")
    with pytest.raises(fame.FameError) as e:
        ctx.apply(y)                                      # eps not set
    assert e.value.status == 6
    ones = np.ones(512)
    with pytest.raises(fame.FameError) as e:
        ctx.set_eps(ones, ones, -ones)
    assert e.value.status == 1
    ctx.set_eps(ones, ones, ones)
    with pytest.raises(fame.FameError) as e:
        ctx.apply(y, out=y)
    assert e.value.status == 1
    with pytest.raises(fame.FameError) as e:
        ctx.grad(1, [1.0])                               # no eigenpairs yet
    assert e.value.status == 6


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_every_apply_plan_matches_oracle(prec):
    """Each available kernel family of the Z and XY passes, and several block sizes,
    gives the oracle's A_r y (fame_set_apply_plan)."""
    lat, ctx, invB, rng = _setup("sc16", (16, 16, 16), seed=2, margin=MARGIN[prec])
    dtype = fame.FAME_C128 if prec == "c128" else fame.FAME_C64
    dt = torch.complex128 if prec == "c128" else torch.complex64
    m = 3
    y = rng.standard_normal((m, 2 * lat.n)) + 1j * rng.standard_normal((m, 2 * lat.n))
    refs = [apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel() for j in range(m)]
    yt = torch.as_tensor(y, dtype=dt, device="cuda")
    tried = 0
    for z in (1, 2, 3, 4):
        for xy in (1, 2, 3, 4, 5):
            for vpc in (1, 2):
                try:
                    ctx.set_apply_plan(dtype, z, xy, vpc)
                except fame.FameError:
                    continue            # family not available for this grid / precision
                got = ctx.apply(yt).cpu().numpy()
                for j in range(m):
                    assert _rel(got[j], refs[j]) < (TOL64 if prec == "c128" else TOL32), (z, xy, vpc, j)
                tried += 1
    assert tried >= (24 if prec == "c64" else 9)
    ctx.set_apply_plan(dtype)


@pytest.mark.parametrize("name,n", [("fcc64", (64, 64, 16)),   # XY 64x64, Z 16
                                    ("mono80", (80, 96, 16)),  # XY 80x96
                                    ("bcc96", (96, 96, 8)),    # XY 96x96, generic Z
                                    ("bcc96", (16, 16, 32)),   # Z 32
                                    ("mono80", (16, 16, 48)),  # Z 48
                                    ("tri192", (16, 16, 64)),  # Z 64
                                    ("sc16", (16, 16, 80)),    # Z 80
                                    ("hex96", (16, 16, 96))])  # Z 96
def test_fixed_length_variants_match_oracle(name, n):
    """The 256- and 512-thread fixed-length XY pass and the fixed-length Z passes with
    and without next-vector prefetch give the oracle's A_r y, with block sizes that
    leave a partial last block of vectors."""
    lat, ctx, invB, rng = _setup(name, n, seed=4)
    m = 5
    y = rng.standard_normal((m, 2 * lat.n)) + 1j * rng.standard_normal((m, 2 * lat.n))
    refs = [apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel() for j in range(m)]
    yt = torch.as_tensor(y, dtype=torch.complex64, device="cuda")
    zs = (1, 4) if n[2] != 8 else (0,)     # no fixed-length Z pass of length 8
    tried = 0
    for z in zs:
        for xy in (1, 5):
            for vpc in (1, 2, 4):
                try:
                    ctx.set_apply_plan(fame.FAME_C64, z, xy, vpc)
                except fame.FameError:
                    continue
                got = ctx.apply(yt).cpu().numpy()
                for j in range(m):
                    assert _rel(got[j], refs[j]) < TOL32, (z, xy, vpc, j)
                tried += 1
    wide = n[0] * n[1] >= 4096             # the 512-thread XY form exists
    assert tried == 3 * len(zs) * (2 if wide else 1)
    ctx.set_apply_plan(fame.FAME_C64)


@pytest.mark.parametrize("name,n", [("fcc64", (16, 16, 16)),     # radix 2 lengths
                                    ("tri192", (24, 20, 12)),   # triclinic twists, radix 3 and 5
                                    ("mono80", (20, 24, 16)),
                                    ("bcc96", (48, 48, 32)),    # a 48 x 48 plane per block
                                    ("hex96", (96, 96, 8))])     # 96 x 96 planes: y / x / y passes
def test_double_float_apply_and_lift_match_oracle(name, n):
    """FAME_C128_DF: complex128 vectors transformed in double-float arithmetic on the FP32
    units.  Its A_r y and lift agree with the oracle's FP64 results and with the FP64
    kernels to 1e-12 of the largest entry (double-float rounds at about 2^-47), and the
    profiler shows the double-float passes ran (no fallback to FP64)."""
    lat, ctx, invB, rng = _setup(name, n, seed=8, margin=MARGIN["c128"])
    m = 3
    y = rng.standard_normal((m, 2 * lat.n)) + 1j * rng.standard_normal((m, 2 * lat.n))
    yt = torch.as_tensor(y, dtype=torch.complex128, device="cuda")
    fame.profile(True)
    got = ctx.apply(yt, double_float=True).cpu().numpy()
    x = ctx.lift(yt, double_float=True).cpu().numpy()
    torch.cuda.synchronize()
    fame.profile(False)
    kinds = fame.profile_read()
    assert {"zin_df_c128", "xy_df_c128", "zout_df_c128"} <= set(kinds), sorted(kinds)
    nat = ctx.apply(yt).cpu().numpy()
    for j in range(m):
        ref = apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()
        assert _rel(got[j], ref) < 1e-12, (j, _rel(got[j], ref))
        assert _rel(got[j], nat[j]) < 1e-12
        assert _rel(x[j], lift(lat, y[j].reshape((2,) + lat.shape), invB).ravel()) < 1e-12
    ctx.close()


def test_autotune_and_plan_cache(tmp_path):
    lat, ctx, invB, rng = _setup("fcc64", (32, 32, 48), seed=1)
    cache = str(tmp_path / "plans.json")
    first = ctx.autotune(6, fame.FAME_C64, cache=cache)
    assert not first["cached"] and first["ms"] > 0
    assert first["z_kernel"] in (1, 2, 3, 4) and first["xy_kernel"] in (1, 2, 3, 4, 5)
    y = rng.standard_normal((2, 2 * lat.n)) + 1j * rng.standard_normal((2, 2 * lat.n))
    got = ctx.apply(torch.as_tensor(y, dtype=torch.complex64, device="cuda")).cpu().numpy()
    for j in range(2):
        assert _rel(got[j], apply_Ar(lat, y[j].reshape((2,) + lat.shape), invB).ravel()) < TOL32
    ctx.set_apply_plan(fame.FAME_C64)
    again = ctx.autotune(6, fame.FAME_C64, cache=cache)
    assert again["cached"] and ctx.apply_plan(fame.FAME_C64)["z_kernel"] == first["z_kernel"]
    with pytest.raises(fame.FameError):
        ctx.set_apply_plan(fame.FAME_C128, z_kernel=1)       # fixed-length passes are complex64 only
