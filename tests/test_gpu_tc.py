"""The tensor-core block Gram (tcgen05, split-TF32 operands) through the C ABI
(fame_block_gram), against FP64 numpy, the FP32 CUDA-core kernels it replaces, and
the solver; and its bounded waits: a wait that cannot end (a load that the test hook
never issues) gives up, the solver reports FAME_E_TIMEOUT and the context stays
usable.

Tolerance: each entry |G_ij - ref_ij| <= 4e-6 ||U_i|| ||V_j||.  Every real product
carries about 2^-21 relative error from the hi/lo TF32 split, and products are
summed in FP32 over a CTA's rows (a few thousand terms; random rounding grows as
their square root) before the FP64 sum over CTAs: a few 1e-7 of the norm product,
with margin.  The FP32 CUDA-core kernels meet the same bound.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 4e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1806_10284_gb300 import build
    build.build()
    fame.load()


@pytest.fixture(autouse=True)
def _every_shape_on_tensor_cores():
    """The library sends only Grams with a side of at least 64 vectors to the tensor
    cores (narrower ones are faster on the FP32 kernel); the tests here take every
    shape the tensor-core kernel accepts."""
    os.environ["FAME_TC_MIN_WIDTH"] = "1"
    yield
    os.environ.pop("FAME_TC_MIN_WIDTH", None)


def _ctx(n, seed=0):
    w = W.WORKLOADS["tri192"]
    rng = np.random.default_rng(seed)
    ctx = fame.Context(w["vectors"], n, W.bloch_from_reduced(w["vectors"], rng.uniform(-0.5, 0.5, 3)))
    shape = (n[2], n[1], n[0])
    ctx.set_eps(*[1.0 + 12.0 * (rng.random(shape) < 0.3) for _ in range(3)])
    return ctx, rng


def _block(rng, k, N):
    # columns of very different scales, as the eigensolver's [X W P] blocks have
    x = rng.standard_normal((k, 2 * N)) + 1j * rng.standard_normal((k, 2 * N))
    return x * np.logspace(0, -3, k)[:, None]


def _check(G, U, V):
    ref = np.conj(U) @ V.T                      # ref[i, j] = sum conj(U_i) V_j
    got = G.cpu().numpy().T                     # fame: G[j][i]
    scale = np.linalg.norm(U, axis=1)[:, None] * np.linalg.norm(V, axis=1)[None, :]
    return float(np.max(np.abs(got - ref) / scale))


@pytest.mark.parametrize("n", [(16, 16, 12),    # 6144 rows
                               (5, 6, 4),       # 240 rows: one partial chunk per CTA
                               (64, 64, 64)])   # 524288 rows (the FCC 64^3 bench size)
@pytest.mark.parametrize("ku,kv", [(15, 30), (45, 90), (30, 75), (1, 1), (7, 128), (128, 128), (33, 17)])
def test_block_gram_complex64(n, ku, kv):
    ctx, rng = _ctx(n)
    N = ctx.N
    U = _block(rng, ku, N)
    V = _block(rng, kv, N)
    Ut = torch.as_tensor(U, dtype=torch.complex64, device="cuda")
    Vt = torch.as_tensor(V, dtype=torch.complex64, device="cuda")
    U32, V32 = Ut.cpu().numpy().astype(np.complex128), Vt.cpu().numpy().astype(np.complex128)
    err = _check(ctx.block_gram(Ut, Vt), U32, V32)
    assert err < TOL, (n, ku, kv, err)
    os.environ["FAME_NO_TC"] = "1"
    try:
        err32 = _check(ctx.block_gram(Ut, Vt), U32, V32)
    finally:
        del os.environ["FAME_NO_TC"]
    assert err32 < TOL, (n, ku, kv, err32)
    ctx.close()


def test_block_gram_prefix_and_wide_shapes():
    """Shapes outside the tensor-core kernel (more than 128 vectors on a side) take the
    CUDA-core kernels; a block whose leading vectors are the other block's (V = [U | W],
    the layout of the eigensolver's Gram of [X W P] against [X W P | A X ...]) shares
    the staged U tiles."""
    ctx, rng = _ctx((16, 16, 12), seed=3)
    N = ctx.N
    U = _block(rng, 30, N)
    W2 = _block(rng, 45, N)
    big = _block(rng, 140, N)
    Ut = torch.as_tensor(U, dtype=torch.complex64, device="cuda")
    Vt = torch.as_tensor(np.concatenate([U, W2]), dtype=torch.complex64, device="cuda")
    Bt = torch.as_tensor(big, dtype=torch.complex64, device="cuda")
    cast = lambda t: t.cpu().numpy().astype(np.complex128)   # noqa: E731
    assert _check(ctx.block_gram(Ut, Vt), cast(Ut), cast(Vt)) < TOL
    assert _check(ctx.block_gram(Vt, Ut), cast(Vt), cast(Ut)) < TOL
    assert _check(ctx.block_gram(Ut, Bt), cast(Ut), cast(Bt)) < TOL
    ctx.close()


def test_block_gram_complex128():
    ctx, rng = _ctx((12, 10, 8), seed=5)
    U = _block(rng, 9, ctx.N)
    V = _block(rng, 21, ctx.N)
    G = ctx.block_gram(torch.as_tensor(U, device="cuda"), torch.as_tensor(V, device="cuda"))
    assert _check(G, U, V) < 1e-13
    ctx.close()


@pytest.mark.parametrize("flags", [fame.FAME_MIXED, fame.FAME_FP64])
def test_solver_with_and_without_tensor_cores(flags):
    """The same solve with the tensor-core Grams and with the FP32 CUDA-core Grams: both
    converge, and their eigenvalues agree to the solver tolerance."""
    ctx, _ = _ctx((24, 20, 16), seed=9)
    lam_tc, _, it_tc = ctx.eigs(10, tol=1e-10, flags=flags)
    os.environ["FAME_NO_TC"] = "1"
    try:
        lam_fp, _, it_fp = ctx.eigs(10, tol=1e-10, flags=flags)
    finally:
        del os.environ["FAME_NO_TC"]
    np.testing.assert_allclose(lam_tc, lam_fp, rtol=1e-9)
    ctx.close()


def test_tensor_core_wait_gives_up_and_context_stays_usable():
    """The producer of the tensor-core Gram never loads chunk 0 (test hook), so the
    consumers' waits cannot end: each CTA gives up after FAME_WAIT_TIMEOUT_MS, lets
    its other copies and MMAs finish, frees its tensor memory and returns.  The Gram
    comes back as NaN and the eigensolver reports FAME_E_TIMEOUT; afterwards the same
    context solves normally."""
    ctx, rng = _ctx((16, 16, 12), seed=7)
    U = torch.as_tensor(_block(rng, 15, ctx.N), dtype=torch.complex64, device="cuda")
    lam0, _, _ = ctx.eigs(6, tol=1e-9, flags=fame.FAME_MIXED)
    os.environ["FAME_WAIT_TIMEOUT_MS"] = "50"
    os.environ["FAME_TEST_TC_SKIP_CHUNK"] = "0"
    try:
        G = ctx.block_gram(U, U)
        torch.cuda.synchronize()
        assert torch.isnan(G).all()
        with pytest.raises(fame.FameError) as e:
            ctx.eigs(6, tol=1e-9, flags=fame.FAME_MIXED)
        assert e.value.status == 8, str(e.value)
    finally:
        del os.environ["FAME_WAIT_TIMEOUT_MS"]
        del os.environ["FAME_TEST_TC_SKIP_CHUNK"]
    G = ctx.block_gram(U, U)
    assert torch.isfinite(G).all()
    lam1, _, _ = ctx.eigs(6, tol=1e-9, flags=fame.FAME_MIXED)
    np.testing.assert_allclose(lam1, lam0, rtol=1e-8)
    ctx.close()
