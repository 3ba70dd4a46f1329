"""Full-size parity of the workloads shaped like the paper's experiments (Section 6),
through the C ABI, against the CPU oracle.

* Band-path lattices (BCC 96^3, hexagonal 96x96x80, base-centred monoclinic
  80x96x64, seeded eps = 12 rods/spheres), one Bloch vector of each path: the 10
  smallest eigenvalues against the oracle's (tests/golden/<lattice>_eigs.json,
  written by make_band_path_eigs.py from oracle/ alone), 1e-5 relative for the
  mixed path and 1e-10 for the FP64 path; every returned eigenpair re-checked with
  the oracle's own FP64 apply at full size (residual <= 1.05e-8 lambda).
* Triclinic 192^3 (8 seeded ellipsoids, eps = 13), one of its four Bloch vectors:
  all 20 eigenpairs of the mixed solve re-checked with the oracle's apply at full
  size.
* Differentiable band gap (simple cubic 48^3, smooth eps on grid nodes, edge-mean
  B_l): d obj / d eps for obj = sum over the 8 Bloch vectors of
  (lambda_6 - lambda_5) / lambda_5, from the adjoint gradient of FP64 and of mixed
  solves, against central differences (step 1e-4) at 64 seeded node voxels.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle_residuals import oracle_residuals
from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1806_10284_gb300 import build
    build.build()
    fame.load()


def _workload_context(name, bloch):
    w = W.WORKLOADS[name]
    ctx = fame.Context(w["vectors"], w["n"], bloch)
    B = W.eps_for(name, ctx.geometry())
    ctx.set_eps(*B)
    return ctx, np.stack([1.0 / b for b in B])


@pytest.mark.parametrize("flags,rtol,tol", [(fame.FAME_MIXED, 1e-5, 1e-8), (fame.FAME_FP64, 1e-10, 1e-10)])
@pytest.mark.parametrize("name", ["bcc96", "hex96", "mono80"])
def test_band_path_lattice_against_oracle_golden(name, flags, rtol, tol):
    gold = json.load(open(os.path.join(GOLDEN, f"{name}_eigs.json")))
    w = W.WORKLOADS[name]
    K = W.bloch_vectors(name)[gold["path_index"]]
    np.testing.assert_allclose(K, gold["bloch"], rtol=1e-14, atol=1e-14)
    ctx, invB = _workload_context(name, K)
    lam, Y, it = ctx.eigs(10, tol=tol, flags=flags, vectors=True, max_iter=600)
    np.testing.assert_allclose(lam, gold["eigenvalues"], rtol=rtol)
    assert ctx.stats()["max_residual"] <= tol
    res = oracle_residuals(w["vectors"], w["n"], K, invB, lam, Y.cpu().numpy())
    assert np.all(res <= 1.05 * tol + 1e-12), (name, res)
    ctx.close()


def test_triclinic_192_all_bands_oracle_residual():
    name = "tri192"
    w = W.WORKLOADS[name]
    K = W.bloch_vectors(name)[0]
    ctx, invB = _workload_context(name, K)
    lam, Y, it = ctx.eigs(20, tol=1e-8, flags=fame.FAME_MIXED, vectors=True, max_iter=600)
    assert np.all(np.diff(lam) >= 0) and lam[0] > 0
    assert ctx.stats()["max_residual"] <= 1e-8
    Yh = Y.cpu().numpy()
    del Y
    ctx.close()
    res = oracle_residuals(w["vectors"], w["n"], K, invB, lam, Yh, workers=5)
    assert np.all(res <= 1.05e-8), res


def _edges(e):
    return [0.5 * (e + np.roll(e, -1, axis=2)), 0.5 * (e + np.roll(e, -1, axis=1)),
            0.5 * (e + np.roll(e, -1, axis=0))]


def test_config_sc48_band_gap_gradient_64_voxels_8_bloch_vectors():
    """obj = sum_k (lambda_6(k) - lambda_5(k)) / lambda_5(k) over the workload's 8 Bloch
    vectors; the adjoint d obj / d eps at 64 seeded node voxels (chain rule through the
    edge means), from FP64 solves and from mixed solves, against central differences of
    the objective (step 1e-4).  The differences come from FP64 solves that start from the
    previous solve's eigenvectors (FAME_WARM_START) and converge to residual 1e-11.

    Error budget of a central difference: truncation O(h^2) (below 1e-6 relative here)
    plus (|e+| + |e-|) / 2h from the rounding error e of each computed objective.  The
    eigenvalues carry rounding of order 1e-13 lambda whatever the residual: the FP64
    rounding of the transforms (2^-53 times their depth) is amplified by about
    sqrt(||A_r|| / lambda), some 250 at 48^3, through Sigma_r at both ends of A_r.  With
    h = 1e-4 a voxel moves the objective by only about 1e-9, so that term dominates.
    The test samples the rounding as the spread s of the objective at the unperturbed
    eps over five re-solves from other starting blocks, floored at that 1e-13 per
    Bloch vector (five samples can fall well below it); the largest of the 128
    objective errors of the differences is taken as 3 s (about three standard
    deviations), so the budget is 2e-4 relative plus 2 x 3 s / 2h."""
    w = W.WORKLOADS["sc48grad"]
    eps0, _ = W.smooth_field_eps(w["n"], w["seed"])
    Ks = W.bloch_vectors("sc48grad")
    assert len(Ks) == 8
    ctxs = [fame.Context(w["vectors"], w["n"], K) for K in Ks]
    tol = 1e-11

    def solve(ctx, B, flags, warm):
        ctx.set_eps(*B)
        return ctx.eigs(6, tol=tol, max_iter=800, flags=flags | (fame.FAME_WARM_START if warm else 0))[0]

    def objective(B):
        total = 0.0
        for ctx in ctxs:
            lam = solve(ctx, B, fame.FAME_FP64, True)
            total += (lam[5] - lam[4]) / lam[4]
        return total

    B0 = _edges(eps0)

    def adjoint(flags):
        g = np.zeros_like(eps0)
        obj = 0.0
        for ctx in ctxs:
            lam = solve(ctx, B0, flags, False)
            assert (lam[5] - lam[4]) > 1e-6 * lam[4]           # band 5 and 6 not degenerate
            obj += (lam[5] - lam[4]) / lam[4]
            d = np.zeros(6)
            d[5], d[4] = 1.0 / lam[4], -lam[5] / lam[4] ** 2
            gB = ctx.grad(6, d, rel_cluster=1e-8).cpu().numpy().reshape((3,) + eps0.shape)
            g += 0.5 * (gB[0] + np.roll(gB[0], 1, axis=2)) + 0.5 * (gB[1] + np.roll(gB[1], 1, axis=1)) \
                + 0.5 * (gB[2] + np.roll(gB[2], 1, axis=0))
        return g, obj

    g_mixed, _ = adjoint(fame.FAME_MIXED)
    g_fp64, obj0 = adjoint(fame.FAME_FP64)
    rng = np.random.default_rng(w["kseed"] + 1)
    voxels = set()
    while len(voxels) < 64:
        voxels.add(tuple(int(rng.integers(0, s)) for s in eps0.shape))
    voxels = sorted(voxels)
    # rounding of the objective: re-solve the unperturbed problem starting from the
    # eigenvectors of problems perturbed at other voxels
    spread = 0.0
    for v in voxels[:5]:
        e = eps0.copy()
        e[v] += 1e-3
        objective(_edges(e))
        spread = max(spread, abs(objective(B0) - obj0))
    noise = max(spread, 1e-13 * len(ctxs))
    h = 1e-4
    fd = []
    for v in voxels:
        vals = []
        for sgn in (1, -1):
            e = eps0.copy()
            e[v] += sgn * h
            vals.append(objective(_edges(e)))
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    for name, g in (("fp64", g_fp64), ("mixed", g_mixed)):
        gv = np.array([g[v] for v in voxels])
        use = np.abs(gv - fd) / (2e-4 * np.abs(fd) + 3.0 * noise / h)
        rel = np.sort(np.abs(gv - fd) / np.abs(fd))
        print(f"band-gap FD ({name} adjoint): rounding of obj {noise:.2e}, |g - fd| / |fd| median "
              f"{rel[len(rel) // 2]:.2e} max {rel[-1]:.2e}, worst budget use {use.max():.2f}")
        assert use.max() <= 1.0, (name, voxels[int(np.argmax(use))], use.max())
    for ctx in ctxs:
        ctx.close()
