"""The extra workloads on the GPU: the gyroid of Section 6 (BCC lattice) with its
permittivity sweep 3..30, and supercells (Section 7) -- against oracle goldens written
by tests/golden/make_workload_eigs.py, and against facts that hold exactly:

* a supercell with the permittivity repeated has the primitive cell's spectra at
  the folded Bloch vectors, so the library's supercell and primitive-cell solves
  must agree with each other to the solver tolerance;
* raising the permittivity lowers every band (min-max), so the sweep's bands fall
  monotonically; warm starts along the sweep give the cold solves' eigenvalues.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workload_eigs.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1806_10284_gb300 import build
    build.build()
    fame.load()


def _geom(vectors, n, K):
    return fame.geometry_of(fame.plan_lattice(vectors, n, K))


@pytest.mark.parametrize("flags,tol,rtol", [(fame.FAME_FP64, 1e-10, 1e-9), (fame.FAME_MIXED, 1e-8, 1e-7)])
def test_gyroid_against_oracle_golden(flags, tol, rtol):
    g = json.load(open(GOLDEN))
    w = W.WORKLOADS["gyroid96"]
    for case in g["gyroid"]:
        n, K = tuple(case["n"]), np.array(case["bloch"])
        ctx = fame.Context(w["vectors"], n, K)
        ctx.set_eps(*W.eps_for("gyroid96", ctx.geometry(), eps_in=case["eps_in"]))
        lam, _, _ = ctx.eigs(g["nev"], tol=tol, max_iter=800, flags=flags)
        np.testing.assert_allclose(lam, case["eigenvalues"], rtol=rtol, err_msg=str(case["eps_in"]))
        ctx.close()


@pytest.mark.parametrize("flags,tol,rtol", [(fame.FAME_FP64, 1e-10, 1e-9), (fame.FAME_MIXED, 1e-8, 1e-7)])
def test_vacancy_supercell_against_oracle_golden(flags, tol, rtol):
    g = json.load(open(GOLDEN))["vacancy"]
    v = W.WORKLOADS["scvac"]
    K = np.array(g["bloch"])
    Vs, ns = W.supercell(v["vectors"], tuple(g["cell_n"]), v["reps"])
    ctx = fame.Context(Vs, ns, K)
    ctx.set_eps(*W.eps_for("scvac", _geom(v["vectors"], tuple(g["cell_n"]), K)))
    lam, _, _ = ctx.eigs(10, tol=tol, max_iter=800, flags=flags)
    np.testing.assert_allclose(lam, g["eigenvalues"], rtol=rtol)
    ctx.close()


@pytest.mark.parametrize("reps", [(2, 1, 1), (2, 2, 1)])
def test_supercell_folds_onto_primitive_cell(reps):
    """SC 16^3 cell with an eps = 13 sphere: the supercell's 8 smallest eigenvalues at K
    are the 8 smallest of the primitive cell's eigenvalues at the folded Bloch vectors."""
    V, n = W.simple_cubic(), (16, 16, 16)
    K = W.bloch_from_reduced(V, [0.11, 0.23, -0.17])
    sphere = [dict(kind="sphere", center=np.full(3, 0.5), radius=0.25)]
    B = W.sample_inclusions(_geom(V, n, K), sphere, 13.0)
    parts = []
    for j1 in range(reps[0]):
        for j2 in range(reps[1]):
            shift = W.bloch_from_reduced(V, [j1 / reps[0], j2 / reps[1], 0.0])
            ctx = fame.Context(V, n, K + shift)
            ctx.set_eps(*B)
            parts.append(ctx.eigs(8, tol=1e-11, max_iter=800, flags=fame.FAME_FP64)[0])
            ctx.close()
    ref = np.sort(np.concatenate(parts))[:8]
    Vs, ns = W.supercell(V, n, reps)
    ctx = fame.Context(Vs, ns, K)
    ctx.set_eps(*W.tile_eps(B, reps))
    lam64 = ctx.eigs(8, tol=1e-11, max_iter=800, flags=fame.FAME_FP64)[0]
    lam32 = ctx.eigs(8, tol=1e-9, max_iter=800, flags=fame.FAME_MIXED)[0]
    ctx.close()
    np.testing.assert_allclose(lam64, ref, rtol=1e-9)
    np.testing.assert_allclose(lam32, ref, rtol=1e-7)


def test_gyroid_eps_sweep_falls_monotonically_and_warm_starts_agree():
    """BCC gyroid at 48^3, eps 3..30: each band falls as eps grows; the sweep solved with
    each eps starting from the previous eps' eigenvectors gives the cold eigenvalues in
    fewer iterations."""
    w = W.WORKLOADS["gyroid96"]
    n = (48, 48, 48)
    K = W.bloch_from_reduced(w["vectors"], w["reduced_k"][0])
    ctx = fame.Context(w["vectors"], n, K)
    geom = ctx.geometry()
    Bs = [W.eps_for("gyroid96", geom, eps_in=e) for e in w["eps_sweep"]]
    cold, warm, it_cold, it_warm = [], [], 0, 0
    for B in Bs:
        ctx.set_eps(*B)
        lam, _, it = ctx.eigs(10, tol=1e-8, max_iter=800, flags=fame.FAME_MIXED)
        cold.append(lam)
        it_cold += it
    for i, B in enumerate(Bs):
        ctx.set_eps(*B)
        flags = fame.FAME_MIXED | (fame.FAME_WARM_START if i > 0 else 0)
        lam, _, it = ctx.eigs(10, tol=1e-8, max_iter=800, flags=flags)
        warm.append(lam)
        it_warm += it
    ctx.close()
    cold, warm = np.array(cold), np.array(warm)
    np.testing.assert_allclose(warm, cold, rtol=1e-7)
    assert np.all(cold[1:] <= cold[:-1] * (1 + 1e-7))
    assert it_warm < it_cold, (it_warm, it_cold)
