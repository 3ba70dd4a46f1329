"""The bounds-checked debug build (libfame_check.so) on the GPU.  It runs in child
processes (a process loads one build of the library): the applies of both precisions
and a mixed eigensolve with the tensor-core Grams report no failed check and give
the normal build's results; and a failed check is recorded, not executed -- a test
hook makes the tensor-core Gram's TMA coordinate check fail for its first chunk, the
copy is not issued, the consumers' bounded waits give up (the Gram comes back NaN)
and fame_bounds_violations reports the kind and the coordinate."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
import numpy as np, torch
sys.path.insert(0, os.environ["FAME_ROOT"])
from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W
fame.load()
out = {"initial": fame.bounds_violations()}
w = W.WORKLOADS["fcc64"]
ctx = fame.Context(w["vectors"], (64, 64, 16), W.bloch_vectors("fcc64")[0])
ctx.set_eps(*W.eps_for("fcc64", ctx.geometry()))
rng = np.random.default_rng(3)
y = rng.standard_normal((5, 2 * ctx.N)) + 1j * rng.standard_normal((5, 2 * ctx.N))
yt = torch.as_tensor(y, device="cuda")
ctx.set_apply_plan(fame.FAME_C64, 1, 5, 2)            # fixed-length Z and XY passes
a64 = ctx.apply(yt.to(torch.complex64)).cpu().numpy()
a128 = ctx.apply(yt).cpu().numpy()
adf = ctx.apply(yt, double_float=True).cpu().numpy()
lam, _, it = ctx.eigs(8, tol=1e-9, flags=fame.FAME_MIXED)
torch.cuda.synchronize()
out["after"] = fame.bounds_violations()
if os.environ.get("PLANT") == "1":
    os.environ["FAME_TC_MIN_WIDTH"] = "1"
    os.environ["FAME_WAIT_TIMEOUT_MS"] = "50"
    os.environ["FAME_TEST_BOUNDS_PLANT"] = "1"
    U = torch.as_tensor(rng.standard_normal((20, 2 * ctx.N)) + 1j * rng.standard_normal((20, 2 * ctx.N)),
                        dtype=torch.complex64, device="cuda")
    G = ctx.block_gram(U, U)
    torch.cuda.synchronize()
    out["planted_nan"] = bool(torch.isnan(G).all())
    out["planted"] = fame.bounds_violations()
    del os.environ["FAME_TEST_BOUNDS_PLANT"]
    G = ctx.block_gram(U, U)
    torch.cuda.synchronize()
    out["after_plant_finite"] = bool(torch.isfinite(G).all())
    out["after_plant"] = fame.bounds_violations()
np.save(os.environ["OUT_NPZ"], np.stack([a64.astype(np.complex128), a128, adf]))
out["lam"] = [float(x) for x in lam]
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def check_lib():
    from paper_1806_10284_gb300 import build
    build.build()
    fame.load()
    return build.build(check_bounds=True)


def _child(tmp_path, plant):
    env = dict(os.environ, FAME_CHECK_BOUNDS="1", FAME_ROOT=ROOT, OUT_NPZ=str(tmp_path / "a.npy"),
               PLANT="1" if plant else "0")
    for k in ("FAME_TEST_BOUNDS_PLANT", "FAME_TC_MIN_WIDTH", "FAME_WAIT_TIMEOUT_MS"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(tmp_path / "a.npy")


def test_checked_build_reports_nothing_and_matches_the_normal_build(check_lib, tmp_path):
    res, arr = _child(tmp_path, plant=False)
    assert res["initial"][0] == 0 and res["after"][0] == 0, res
    w = W.WORKLOADS["fcc64"]
    ctx = fame.Context(w["vectors"], (64, 64, 16), W.bloch_vectors("fcc64")[0])
    ctx.set_eps(*W.eps_for("fcc64", ctx.geometry()))
    rng = np.random.default_rng(3)
    y = rng.standard_normal((5, 2 * ctx.N)) + 1j * rng.standard_normal((5, 2 * ctx.N))
    yt = torch.as_tensor(y, device="cuda")
    ctx.set_apply_plan(fame.FAME_C64, 1, 5, 2)
    ref = [ctx.apply(yt.to(torch.complex64)).cpu().numpy(), ctx.apply(yt).cpu().numpy(),
           ctx.apply(yt, double_float=True).cpu().numpy()]
    lam, _, _ = ctx.eigs(8, tol=1e-9, flags=fame.FAME_MIXED)
    for got, want, tol in zip(arr, ref, (1e-6, 1e-13, 1e-13)):
        assert float(np.abs(got - want).max() / np.abs(want).max()) < tol
    np.testing.assert_allclose(res["lam"], lam, rtol=1e-9)
    ctx.close()


def test_failed_check_is_recorded_not_executed(check_lib, tmp_path):
    res, _ = _child(tmp_path, plant=True)
    count, code, index = res["planted"]
    assert res["planted_nan"] and count >= 1 and code == 1 and index == 0, res
    assert res["after_plant_finite"] and res["after_plant"][0] == 0, res
