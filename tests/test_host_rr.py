"""CPU tests of the host Rayleigh-Ritz solver of the block eigensolver (csrc/rr.cpp),
through a small C++ driver (host_rr_check.cpp) built with the host compiler.

The pencils have known spectra (GA = C^H U diag(lambda) U^H C, GB = C^H C), including
exact and near degeneracies, a tight cluster, a fully flat spectrum and a graded
spectrum with zeros, so each path (Cholesky of GB, and the eigen-decomposition of GB)
is checked against the exact eigenvalues, its residuals and GB-orthonormality."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1806_10284_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("host C++ compiler or CUDA headers not found")
    exe = str(tmp_path_factory.mktemp("rr") / "host_rr_check")
    cmd = [cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", inc, os.path.join(ROOT, "tests", "host_rr_check.cpp"),
           os.path.join(CSRC, "rr.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _run(exe, spectrum, k, m, chol, seed=1, sweeps=None):
    args = [exe, spectrum, str(k), str(m), str(int(chol)), str(seed)] + ([str(sweeps)] if sweeps else [])
    r = subprocess.run(args, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    f = r.stdout.split()
    return dict(theta=float(f[1]), resid=float(f[3]), orth=float(f[5]), got=int(f[7]))


@pytest.mark.parametrize("chol", [True, False])
@pytest.mark.parametrize("spectrum", ["spread", "triples", "pairs9", "pairs13", "cluster", "flat", "graded"])
def test_rayleigh_ritz_known_spectrum(driver, spectrum, chol):
    for seed in (1, 2):
        out = _run(driver, spectrum, 45, 15, chol, seed)
        assert out["got"] == 15
        assert out["theta"] < 1e-12, out
        assert out["resid"] < 1e-12, out
        assert out["orth"] < 1e-11, out


@pytest.mark.parametrize("k,m", [(1, 1), (2, 1), (3, 3), (8, 4), (90, 30)])
def test_rayleigh_ritz_sizes(driver, k, m):
    for chol in (True, False):
        out = _run(driver, "spread", k, m, chol)
        assert out["got"] == m
        assert out["theta"] < 1e-12 and out["resid"] < 1e-12 and out["orth"] < 1e-11, (k, m, chol, out)


@pytest.mark.parametrize("chol", [True, False])
def test_rayleigh_ritz_reports_qr_that_runs_out_of_sweeps(driver, chol):
    """An implicit QR stopped after a few sweeps, far too few to deflate 45 eigenvalues,
    must be reported (got = -2) rather than returned as converged pairs; the same
    pencil converges under the default limit."""
    out = _run(driver, "spread", 45, 15, chol)
    assert out["got"] == 15 and out["theta"] < 1e-12
    out = _run(driver, "spread", 45, 15, chol, sweeps=3)
    assert out["got"] == -2, out
