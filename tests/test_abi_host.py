"""CPU tests of the C-ABI library: it loads, exports every symbol include/fame.h declares,
its host lattice plan agrees with the oracle, and host-side errors are reported."""
import os
import re

import numpy as np
import pytest

from oracle.lattice import make_lattice
from paper_1806_10284_gb300 import fame
from paper_1806_10284_gb300 import workloads as W
from small_lattices import random_triclinics

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_10284_gb300 import build
    build.build()
    return fame.load()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "fame.h")).read()
    return sorted(set(re.findall(r"FAME_API\s+[\w\s\*]+?\b(fame_\w+)\s*\(", src)))


def test_header_declares_symbols():
    syms = header_symbols()
    assert "fame_create" in syms and "fame_apply_Ar" in syms and "fame_eigs" in syms
    assert len(syms) >= 15


def test_every_declared_symbol_exported(lib):
    for s in header_symbols():
        assert hasattr(lib, s), s
    assert sorted(fame.exported_symbols()) == header_symbols()


def test_bounds_checked_build_links_and_exports_every_symbol(lib):
    """The debug build with the kernels' bounds checks (-DFAME_CHECK_BOUNDS) compiles,
    links and exports the same C ABI; the normal build reports -1 (no checks)."""
    import ctypes
    from paper_1806_10284_gb300 import build
    path = build.build(check_bounds=True)
    chk = ctypes.CDLL(path)
    for s in header_symbols():
        assert hasattr(chk, s), s
    assert fame.bounds_violations() == (-1, 0, 0)


def test_version_and_counter(lib):
    assert "sm_103a" in fame.version()
    assert fame.launch_count() >= 0


@pytest.mark.parametrize("name", list(W.WORKLOADS))
def test_host_plan_matches_oracle(lib, name):
    w = W.WORKLOADS[name]
    for K in W.bloch_vectors(name)[:3]:
        p = fame.plan_lattice(w["vectors"], w["n"], K)
        lat = make_lattice(w["vectors"], w["n"], K)
        assert p["perm"] == tuple(lat.perm)
        assert p["m"] == (lat.m1, lat.m2, lat.m3)
        assert p["rho"] == (lat.rho1, lat.rho2, lat.rho3)
        assert p["s"] == (lat.s1, lat.s2, lat.s3)
        np.testing.assert_allclose(p["delta"], (lat.dx, lat.dy, lat.dz), rtol=1e-14)
        np.testing.assert_allclose(p["a"], lat.a, atol=1e-14)
        np.testing.assert_allclose(p["kappa"], lat.kappa, atol=1e-13)


def test_host_plan_matches_oracle_random(lib):
    """The same triclinic inputs planned by the library (C++) and the oracle (Python)."""
    rng = np.random.default_rng(3)
    done = 0
    while done < 40:
        v = W.triclinic(1.0, rng.uniform(0.5, 1.3), rng.uniform(0.5, 1.3), *rng.uniform(55, 125, 3))
        n = tuple(int(x) for x in rng.choice([4, 6, 8, 10, 12, 16, 20, 24], 3))
        K = rng.uniform(-4, 4, 3)
        try:
            lat = make_lattice(v, n, K)
        except ValueError:
            with pytest.raises(fame.FameError):
                fame.plan_lattice(v, n, K)
            continue
        p = fame.plan_lattice(v, n, K)
        assert p["m"] == (lat.m1, lat.m2, lat.m3) and p["s"] == (lat.s1, lat.s2, lat.s3)
        assert p["perm"] == tuple(lat.perm)
        np.testing.assert_allclose(p["a"], lat.a, atol=1e-13)
        np.testing.assert_allclose(p["kappa"], lat.kappa, atol=1e-12)
        done += 1


def test_plan_errors(lib):
    sc = np.eye(3)
    with pytest.raises(fame.FameError) as e:
        fame.plan_lattice(sc, (7, 8, 8), np.zeros(3))           # prime factor 7
    assert e.value.status == 3
    with pytest.raises(fame.FameError) as e:
        fame.plan_lattice(sc, (1, 8, 8), np.zeros(3))           # below 2
    assert e.value.status == 3
    with pytest.raises(fame.FameError) as e:
        fame.plan_lattice(np.array([[1.0, 0, 0], [0, 1, 0], [1, 1, 0]]), (8, 8, 8), np.zeros(3))
    assert e.value.status == 2
    with pytest.raises(fame.FameError) as e:
        fame.plan_lattice(sc, (8, 8, 8), np.array([np.nan, 0, 0]))
    assert e.value.status == 1
