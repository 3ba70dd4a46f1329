"""The A_r apply through the entry point that allocates no device memory
(fame_apply_Ar_static, workspace in a static device array), against the ordinary
fame_apply_Ar on the same inputs.  Collected last (file name) so that it also runs
after every other test has used the library; it needs no state from them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _ctx(name, n, seed):
    w = W.WORKLOADS[name]
    rng = np.random.default_rng(seed)
    K = W.bloch_from_reduced(w["vectors"], rng.uniform(-0.5, 0.5, 3))
    ctx = fame.Context(w["vectors"], n, K)
    shape = (n[2], n[1], n[0])
    ctx.set_eps(*[1.0 + 12.0 * (rng.random(shape) < 0.3) for _ in range(3)])
    return ctx, rng


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dt", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("name,n,m", [("fcc64", (64, 64, 64), 4),    # fixed-length passes
                                      ("hex96", (20, 12, 10), 3)])   # generic passes
def test_static_apply_matches_apply(name, n, m, dt):
    ctx, rng = _ctx(name, n, seed=11)
    N = ctx.N
    if m * 3 * N * (8 if dt == torch.complex64 else 16) > LIMIT:
        m = LIMIT // (3 * N * (8 if dt == torch.complex64 else 16))
    assert m >= 1
    y = torch.as_tensor(rng.standard_normal((m, 2 * N)) + 1j * rng.standard_normal((m, 2 * N)),
                        dtype=dt, device="cuda")
    ref = ctx.apply(y)
    out = torch.empty_like(y)
    for _ in range(2):                      # two calls in a row reuse the same workspace
        out.zero_()
        ctx.apply_static(y, out)
        torch.cuda.synchronize()
        assert _rel(out, ref) < TOL[dt]
    ctx.close()


def test_static_apply_rejects_oversize():
    ctx, rng = _ctx("fcc64", (64, 64, 64), seed=12)
    m = LIMIT // (3 * ctx.N * 8) + 1        # one complex64 vector more than fits
    y = torch.zeros((m, 2 * ctx.N), dtype=torch.complex64, device="cuda")
    out = torch.empty_like(y)
    with pytest.raises(fame.FameError, match="exceeds the static maximum"):
        ctx.apply_static(y, out)
    ctx.close()
