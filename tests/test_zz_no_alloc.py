"""The A_r apply through the entry point that allocates no device memory
(fame_apply_Ar_static, workspace in a static device array).

Some callers cannot allocate device memory at the point where they need the
operator: code that runs under a memory budget owned by a framework's caching
allocator, or a latency-bound loop in which a cudaMalloc (which may synchronise
the device) is not acceptable.  These tests check, through the C ABI, that the
static entry point
  * allocates nothing: the device's free memory is the same before and after
    repeated calls on a fresh context (after one warm-up call that loads the
    kernels),
  * computes A_r y: against the CPU oracle on a small grid, and against the
    ordinary fame_apply_Ar on two calls in a row (the workspace keeps the last
    call's contents, which the next call must not depend on).
Collected last (file name) so that it also runs after every other test has used
the library; it needs no state from them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.lattice import make_lattice
from oracle.nfsep import apply_Ar, basis_margin
from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.complex64: 2e-5, torch.complex128: 1e-11}
LIMIT = 32 << 20    # FAME_STATIC_WORKSPACE_BYTES


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1806_10284_gb300 import build
    build.build()
    fame.load()


def _ctx(name, n, seed, margin=1e-5):
    """Context with a random Bloch vector whose frequencies keep ``margin`` from the
    reference-vector switch of the range basis, and a random two-valued eps."""
    w = W.WORKLOADS[name]
    for s in range(seed, seed + 50):
        rng = np.random.default_rng(s)
        K = W.bloch_from_reduced(w["vectors"], rng.uniform(-0.5, 0.5, 3))
        lat = make_lattice(w["vectors"], n, K)
        if basis_margin(lat) > margin:
            break
    ctx = fame.Context(w["vectors"], n, K)
    B = [1.0 + 12.0 * (rng.random(lat.shape) < 0.3) for _ in range(3)]
    ctx.set_eps(*B)
    return ctx, lat, np.stack([1.0 / b for b in B]), rng


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _block(rng, m, N, dt):
    y = rng.standard_normal((m, 2 * N)) + 1j * rng.standard_normal((m, 2 * N))
    return y, torch.as_tensor(y, dtype=dt, device="cuda")


@pytest.mark.parametrize("dt", [torch.complex64, torch.complex128])
def test_static_apply_allocates_nothing_and_matches_oracle(dt):
    ctx, lat, invB, rng = _ctx("tri192", (18, 15, 8), seed=21)
    m = 3
    y_np, y = _block(rng, m, ctx.N, dt)
    out = torch.empty_like(y)
    ctx.apply_static(y, out)                       # warm-up: loads the kernels
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        ctx.apply_static(y, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "fame_apply_Ar_static changed the device's free memory"
    got = out.cpu().numpy()
    for j in range(m):
        ref = apply_Ar(lat, y_np[j].reshape((2,) + lat.shape), invB).ravel()
        assert float(np.abs(got[j] - ref).max() / np.abs(ref).max()) < TOL[dt], j
    ctx.close()


@pytest.mark.parametrize("dt", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("name,n,m", [("fcc64", (64, 64, 64), 4),    # fixed-length passes
                                      ("hex96", (20, 12, 10), 3)])   # generic passes
def test_static_apply_matches_apply(name, n, m, dt):
    ctx, _, _, rng = _ctx(name, n, seed=11)
    N = ctx.N
    if m * 3 * N * (8 if dt == torch.complex64 else 16) > LIMIT:
        m = LIMIT // (3 * N * (8 if dt == torch.complex64 else 16))
    assert m >= 1
    _, y = _block(rng, m, N, dt)
    out = torch.empty_like(y)
    ctx.apply_static(y, out)                       # warm-up, before the ordinary apply grows its workspace
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outs = []
    for _ in range(2):                             # two calls in a row reuse the same workspace
        o = torch.full_like(y, float("nan"))
        ctx.apply_static(y, o)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = ctx.apply(y)
    for o in outs:
        assert _rel(o, ref) < TOL[dt]
    ctx.close()


def test_static_apply_rejects_oversize():
    ctx, _, _, rng = _ctx("fcc64", (64, 64, 64), seed=12)
    m = LIMIT // (3 * ctx.N * 8) + 1        # one complex64 vector more than fits
    y = torch.zeros((m, 2 * ctx.N), dtype=torch.complex64, device="cuda")
    out = torch.empty_like(y)
    with pytest.raises(fame.FameError, match="exceeds the static maximum"):
        ctx.apply_static(y, out)
    ctx.close()


def test_static_apply_rejects_strided_out():
    ctx, _, _, rng = _ctx("hex96", (20, 12, 10), seed=13)
    _, y = _block(rng, 2, ctx.N, torch.complex64)
    wide = torch.empty((2, 4 * ctx.N), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError, match="contiguous"):
        ctx.apply_static(y, wide[:, ::2])
    ctx.close()
