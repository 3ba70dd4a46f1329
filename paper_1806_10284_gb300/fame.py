"""Thin ctypes binding of the C ABI in include/fame.h (argument marshalling only).

Every numerical step runs in the CUDA library ``_lib/libfame.so``; this module
converts torch tensors / numpy arrays to pointers, streams to handles and
status codes to exceptions.  A missing library raises ``FameError`` at first
use: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfame.so")
# the bounds-checked debug build (build.build(check_bounds=True)); loaded instead of the
# normal library when the environment sets FAME_CHECK_BOUNDS=1
LIB_CHECK_PATH = os.path.join(_HERE, "_lib", "libfame_check.so")

FAME_C64, FAME_C128, FAME_C128_DF = 0, 1, 2
FAME_FP64, FAME_MIXED, FAME_DETERMINISTIC, FAME_WARM_START, FAME_INV_LANCZOS = 1, 2, 4, 8, 16
STATUS = {0: "FAME_OK", 1: "FAME_E_ARG", 2: "FAME_E_LATTICE", 3: "FAME_E_RADIX", 4: "FAME_E_CUDA",
          5: "FAME_E_NOMEM", 6: "FAME_E_STATE", 7: "FAME_E_NOCONV", 8: "FAME_E_TIMEOUT"}

# Every symbol declared in include/fame.h, with its ctypes signature.
_D3 = C.POINTER(C.c_double)
_SIGS = {
    "fame_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _D3, _D3, _D3, C.c_int, C.c_int,
                              C.c_int, _D3]),
    "fame_plan_lattice": (C.c_int, [_D3, _D3, _D3, C.c_int, C.c_int, C.c_int, _D3, C.c_void_p]),
    "fame_get_plan": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fame_set_k": (C.c_int, [C.c_void_p, _D3]),
    "fame_set_eps": (C.c_int, [C.c_void_p, _D3, _D3, _D3, C.c_void_p]),
    "fame_set_eps_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "fame_apply_Ar": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fame_apply_Ar_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fame_lift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fame_set_apply_plan": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fame_get_apply_plan": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fame_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "fame_eigs": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, _D3, C.c_void_p,
                            C.POINTER(C.c_int), C.c_void_p]),
    "fame_get_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fame_grad_eps": (C.c_int, [C.c_void_p, C.c_int, _D3, C.c_double, C.c_void_p, C.c_void_p]),
    "fame_fields": (C.c_int, [C.c_void_p, C.c_void_p, _D3, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                              C.c_void_p]),
    "fame_block_gram": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                  C.c_void_p]),
    "fame_eigs_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_double, C.c_int,
                                    C.c_int, _D3, C.POINTER(C.c_int), C.c_void_p]),
    "fame_profile": (C.c_int, [C.c_int]),
    "fame_profile_read": (C.c_int, [C.c_void_p, C.c_int]),
    "fame_last_error": (C.c_char_p, [C.c_void_p]),
    "fame_destroy": (None, [C.c_void_p]),
    "fame_launch_count": (C.c_ulonglong, []),
    "fame_version": (C.c_char_p, []),
    "fame_bounds_violations": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
}


class FameError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("perm", C.c_int * 3), ("m", C.c_int * 3), ("rho", C.c_int * 3),
                ("s", C.c_int * 3), ("delta", C.c_double * 3), ("a", C.c_double * 9),
                ("kappa", C.c_double * 3)]


class ApplyPlan(C.Structure):
    _fields_ = [("z_kernel", C.c_int), ("xy_kernel", C.c_int), ("vectors_per_block", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iters_mixed", C.c_int), ("iters_fp64", C.c_int), ("applies_c64", C.c_longlong),
                ("applies_c128", C.c_longlong), ("max_residual", C.c_double),
                ("rr_host_ms", C.c_double)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("total_ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


_lib = None
_lock = threading.Lock()


def profile(enable: bool):
    """Start (clearing old records) or stop per-kernel event timing."""
    _check(load().fame_profile(1 if enable else 0), None)


def profile_read():
    """{kernel kind: dict(launches, total_ms, bytes, flops)} since profile(True)."""
    arr = (KernelStat * 64)()
    k = load().fame_profile_read(C.cast(arr, C.c_void_p), 64)
    return {arr[i].name.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms,
                                       bytes=arr[i].bytes, flops=arr[i].flops) for i in range(k)}


def load(path: str = None):
    """Load the library (once).  Raises FameError if it is missing or incomplete.  The
    environment variable FAME_CHECK_BOUNDS=1 selects the bounds-checked build."""
    global _lib
    if path is None:
        path = LIB_CHECK_PATH if os.environ.get("FAME_CHECK_BOUNDS") == "1" else LIB_PATH
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FameError(-1, f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)          # AttributeError if a symbol is missing
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return list(_SIGS)


def _d3(v):
    a = (C.c_double * 3)(*[float(x) for x in np.asarray(v, dtype=np.float64).ravel()[:3]])
    return C.cast(a, _D3), a


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _check(st, ctx=None):
    if st != 0:
        msg = load().fame_last_error(ctx)
        raise FameError(st, msg.decode() if msg else "")


def launch_count() -> int:
    return int(load().fame_launch_count())


def version() -> str:
    return load().fame_version().decode()


def bounds_violations():
    """(count, code, index) of the failed bounds checks since the previous call, cleared
    (the bounds-checked build; count -1 in the normal build)."""
    code, index = C.c_int(0), C.c_longlong(0)
    n = load().fame_bounds_violations(C.byref(code), C.byref(index))
    return int(n), int(code.value), int(index.value)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_out(out, like):
    """A caller-provided output is written through its data pointer in the dense layout:
    it must be contiguous and on the device of the input."""
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    if not out.is_cuda or out.device != like.device:
        raise ValueError("out must be a CUDA tensor on the device of the input")


def _dtype_code(t, double_float=False):
    import torch
    if t.dtype == torch.complex64:
        if double_float:
            raise TypeError("double_float applies to complex128 vectors")
        return FAME_C64
    if t.dtype == torch.complex128:
        return FAME_C128_DF if double_float else FAME_C128
    raise TypeError("vectors must be complex64 or complex128")


def _info_dict(i):
    return dict(n=tuple(i.n), perm=tuple(i.perm), m=tuple(i.m), rho=tuple(i.rho),
                s=tuple(i.s), delta=tuple(i.delta),
                a=np.array(list(i.a)).reshape(3, 3).T, kappa=np.array(list(i.kappa)))


def plan_lattice(vectors, n, bloch):
    """Geometry of fame_create for these arguments, computed on the host (no GPU)."""
    lib = load()
    v = np.asarray(vectors, dtype=np.float64)
    a1, k1 = _d3(v[0])
    a2, k2 = _d3(v[1])
    a3, k3 = _d3(v[2])
    b, k4 = _d3(bloch)
    info = PlanInfo()
    st = lib.fame_plan_lattice(a1, a2, a3, int(n[0]), int(n[1]), int(n[2]), b, C.byref(info))
    _check(st, None)
    return _info_dict(info)


def geometry_of(plan):
    from .workloads import Geometry
    return Geometry(n=plan["n"], s=plan["s"], delta=plan["delta"], perm=plan["perm"])


class Context:
    """One lattice, grid and Bloch vector (fame_create)."""

    def __init__(self, vectors, n, bloch, lattice: int = 14):
        lib = load()
        v = np.asarray(vectors, dtype=np.float64)
        a1, k1 = _d3(v[0])
        a2, k2 = _d3(v[1])
        a3, k3 = _d3(v[2])
        b, k4 = _d3(bloch)
        h = C.c_void_p()
        st = lib.fame_create(C.byref(h), int(lattice), a1, a2, a3, int(n[0]), int(n[1]), int(n[2]), b)
        _check(st, None)
        self._h = h
        info = PlanInfo()
        _check(lib.fame_get_plan(h, C.byref(info)), h)
        self.info = info
        self.n = tuple(info.n)
        self.N = int(np.prod(self.n))

    # -- plan ---------------------------------------------------------------
    def plan(self):
        return _info_dict(self.info)

    def geometry(self):
        return geometry_of(self.plan())

    def set_k(self, bloch):
        b, keep = _d3(bloch)
        _check(load().fame_set_k(self._h, b), self._h)
        info = PlanInfo()
        _check(load().fame_get_plan(self._h, C.byref(info)), self._h)
        self.info = info

    def set_eps(self, B1, B2, B3, stream=None):
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel()) for x in (B1, B2, B3)]
        for a in arrs:
            if a.size != self.N:
                raise ValueError("eps arrays must have n entries")
        ptrs = [a.ctypes.data_as(_D3) for a in arrs]
        _check(load().fame_set_eps(self._h, *ptrs, _stream(stream)), self._h)

    def set_eps_device(self, B, stream=None):
        """B: torch float64 CUDA tensor with 3n entries ([3][n])."""
        import torch
        if B.dtype != torch.float64 or not B.is_cuda or B.numel() != 3 * self.N:
            raise ValueError("B must be a float64 CUDA tensor with 3n entries")
        B = B.contiguous()
        _check(load().fame_set_eps_device(self._h, _ptr(B), _stream(stream)), self._h)

    # -- operator -----------------------------------------------------------
    def apply(self, y, out=None, stream=None, double_float=False):
        """A_r y for a complex CUDA tensor y of shape (m, 2n) (or (2n,)).  With
        double_float a complex128 y is transformed in double-float arithmetic
        (FAME_C128_DF)."""
        import torch
        y = y.contiguous()
        m = y.numel() // (2 * self.N)
        if m * 2 * self.N != y.numel():
            raise ValueError("y must hold m vectors of 2n entries")
        if out is None:
            out = torch.empty_like(y)
        elif out.shape != y.shape or out.dtype != y.dtype:
            raise ValueError("out must have the shape and dtype of y")
        else:
            _check_out(out, y)
        _check(load().fame_apply_Ar(self._h, _ptr(y), _ptr(out), m, _dtype_code(y, double_float),
                                    _stream(stream)), self._h)
        return out

    def apply_static(self, y, out, stream=None):
        """A_r y into a caller-provided ``out`` through the entry point that allocates no
        device memory (workspace limited to FAME_STATIC_WORKSPACE_BYTES)."""
        y = y.contiguous()
        m = y.numel() // (2 * self.N)
        if m * 2 * self.N != y.numel() or out.shape != y.shape or out.dtype != y.dtype:
            raise ValueError("y must hold m vectors of 2n entries and out must match it")
        _check_out(out, y)
        _check(load().fame_apply_Ar_static(self._h, _ptr(y), _ptr(out), m, _dtype_code(y),
                                           _stream(stream)), self._h)
        return out

    def fields(self, y, lam, want_e=True, want_h=True, stream=None):
        """(E, H): complex128 CUDA tensors (m, 3n) of eigenpairs (lam[j], y[j]) (fame_fields);
        E = B^{-1} Q_r Sigma_r y, H = -i sqrt(lam) P_r y.  Either may be skipped (None)."""
        import torch
        y = y.contiguous()
        if y.dtype != torch.complex128:
            raise TypeError("fields are computed from complex128 eigenvectors")
        m = y.numel() // (2 * self.N)
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).ravel())
        if lam.size != m:
            raise ValueError("one eigenvalue per vector")
        E = torch.empty((m, 3 * self.N), dtype=torch.complex128, device=y.device) if want_e else None
        H = torch.empty((m, 3 * self.N), dtype=torch.complex128, device=y.device) if want_h else None
        _check(load().fame_fields(self._h, _ptr(y), lam.ctypes.data_as(_D3), _ptr(E) if E is not None else None,
                                  _ptr(H) if H is not None else None, m, FAME_C128, _stream(stream)), self._h)
        return E, H

    def block_gram(self, U, V, stream=None):
        """G = U^H V (complex128 CUDA tensor [kv][ku], column-major in the C sense: G[j][i] =
        sum conj(U_i) V_j) for U (ku, 2n) and V (kv, 2n) of one complex dtype (fame_block_gram)."""
        import torch
        U = U.contiguous()
        V = V.contiguous()
        if U.dtype != V.dtype or U.shape[-1] != 2 * self.N or V.shape[-1] != 2 * self.N:
            raise ValueError("U and V must be (k, 2n) tensors of one complex dtype")
        ku, kv = U.numel() // (2 * self.N), V.numel() // (2 * self.N)
        G = torch.empty((kv, ku), dtype=torch.complex128, device=U.device)
        _check(load().fame_block_gram(self._h, _ptr(U), ku, _ptr(V), kv, _dtype_code(U), _ptr(G),
                                      _stream(stream)), self._h)
        return G

    # -- apply plans and the autotuner --------------------------------------
    def apply_plan(self, dtype=FAME_C64):
        """{z_kernel, xy_kernel, vectors_per_block} of the apply for dtype (0 = automatic)."""
        p = ApplyPlan()
        _check(load().fame_get_apply_plan(self._h, int(dtype), C.byref(p)), self._h)
        return {f: getattr(p, f) for f, _ in ApplyPlan._fields_}

    def set_apply_plan(self, dtype=FAME_C64, z_kernel=0, xy_kernel=0, vectors_per_block=0):
        p = ApplyPlan(int(z_kernel), int(xy_kernel), int(vectors_per_block))
        _check(load().fame_set_apply_plan(self._h, int(dtype), C.byref(p)), self._h)

    def autotune(self, m, dtype=FAME_C64, cache=None, stream=None):
        """Pick the fastest apply plan for blocks of m vectors (fame_autotune).  With
        ``cache`` (a JSON file path) a plan stored under (n1, n2, n3, precision, m) is
        reused instead of timed, and a newly timed one is stored."""
        import json
        import os
        key = "%dx%dx%d/%s/%d" % (*self.n, "c64" if int(dtype) == FAME_C64 else "c128", int(m))
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                e = table[key]
                self.set_apply_plan(dtype, e["z_kernel"], e["xy_kernel"], e["vectors_per_block"])
                return dict(e, cached=True)
        ms = C.c_double(0.0)
        _check(load().fame_autotune(self._h, int(m), int(dtype), C.byref(ms), _stream(stream)), self._h)
        entry = dict(self.apply_plan(dtype), ms=ms.value)
        if cache:
            table[key] = entry
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(entry, cached=False)

    def lift(self, y, stream=None, double_float=False):
        """x = B^{-1} Q_r Sigma_r y: (m, 2n) -> (m, 3n) complex on the Yee grid (double_float:
        as in apply)."""
        import torch
        y = y.contiguous()
        m = y.numel() // (2 * self.N)
        x = torch.empty((m, 3 * self.N), dtype=y.dtype, device=y.device)
        _check(load().fame_lift(self._h, _ptr(y), _ptr(x), m, _dtype_code(y, double_float), _stream(stream)),
               self._h)
        return x

    # -- eigensolver --------------------------------------------------------
    def eigs(self, nev, tol=1e-8, max_iter=400, flags=FAME_MIXED, vectors=False, stream=None,
             allow_noconv=False):
        import torch
        lam = np.zeros(nev, dtype=np.float64)
        Y = None
        if vectors:
            Y = torch.empty((nev, 2 * self.N), dtype=torch.complex128, device="cuda")
        it = C.c_int(0)
        st = load().fame_eigs(self._h, int(nev), float(tol), int(max_iter), int(flags),
                              lam.ctypes.data_as(_D3), _ptr(Y) if Y is not None else None,
                              C.byref(it), _stream(stream))
        if not (allow_noconv and st == 7):
            _check(st, self._h)
        return lam, Y, int(it.value)

    def stats(self):
        s = SolveStats()
        _check(load().fame_get_stats(self._h, C.byref(s)), self._h)
        return dict(iters_mixed=s.iters_mixed, iters_fp64=s.iters_fp64,
                    applies_c64=s.applies_c64, applies_c128=s.applies_c128,
                    max_residual=s.max_residual, rr_host_ms=s.rr_host_ms)

    def grad(self, nev, dobj_dlambda, rel_cluster=1e-8, stream=None):
        """dB (float64 CUDA tensor [3][n]) for the last eigs call."""
        import torch
        d = np.ascontiguousarray(np.asarray(dobj_dlambda, dtype=np.float64))
        out = torch.empty((3, self.N), dtype=torch.float64, device="cuda")
        _check(load().fame_grad_eps(self._h, int(nev), d.ctypes.data_as(_D3), float(rel_cluster),
                                    _ptr(out), _stream(stream)), self._h)
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.fame_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eigs_batched(contexts, nev, tol=1e-8, max_iter=400, flags=FAME_MIXED, stream=None):
    lib = load()
    arr = (C.c_void_p * len(contexts))(*[c._h.value for c in contexts])
    lam = np.zeros((len(contexts), nev), dtype=np.float64)
    its = (C.c_int * len(contexts))()
    st = lib.fame_eigs_batched(arr, len(contexts), int(nev), float(tol), int(max_iter), int(flags),
                               lam.ctypes.data_as(_D3), its, _stream(stream))
    if st != 0:
        msgs = [lib.fame_last_error(c._h) for c in contexts]
        msg = next((m.decode() for m in msgs if m), None) or (lib.fame_last_error(None) or b"").decode()
        raise FameError(st, msg or "batched solve failed")
    return lam, list(its)


def eig_grad_function():
    """torch.autograd.Function: B (float64 CUDA, [3][n]) -> the nev smallest eigenvalues.

    Forward runs fame_set_eps_device + fame_eigs; backward runs fame_grad_eps
    (Hellmann-Feynman through B^{-1}, cluster-averaged), so any differentiable
    objective of the eigenvalues gets d obj / d B.
    """
    import torch

    class EigGrad(torch.autograd.Function):
        @staticmethod
        def forward(ctx_, B, fctx, nev, tol, flags, rel_cluster):
            fctx.set_eps_device(B.detach())
            lam, _, _ = fctx.eigs(nev, tol=tol, flags=flags)
            ctx_.fctx, ctx_.nev, ctx_.rel = fctx, nev, rel_cluster
            return torch.as_tensor(lam, dtype=torch.float64, device=B.device)

        @staticmethod
        def backward(ctx_, g):
            dB = ctx_.fctx.grad(ctx_.nev, g.detach().cpu().numpy(), ctx_.rel)
            return dB.reshape(-1), None, None, None, None, None

    return EigGrad
