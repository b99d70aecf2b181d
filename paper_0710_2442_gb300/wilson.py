"""Thin ctypes binding of libwilson_gb300 (the C ABI in include/wilson.h).

Argument marshalling only: every operation runs in the library's CUDA
kernels.  Fields are passed as torch tensors (complex128, canonical layout;
CUDA tensors for the stateless calls, CUDA or CPU for handle import/export)
or raw integer addresses.  If the shared library is missing this module
raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libwilson_gb300.so")

WILSON_OK, WILSON_ERR_ARG, WILSON_ERR_CUDA, WILSON_ERR_OOM, WILSON_ERR_NOCONV, WILSON_ERR_TIMEOUT, \
    WILSON_ERR_NUMERIC, WILSON_ERR_UNSUPPORTED = range(8)
WILSON_F64, WILSON_F32, WILSON_F16, WILSON_BF16 = range(4)
WILSON_OP_HOP, WILSON_OP_M, WILSON_OP_SCHUR, WILSON_OP_SCHUR_DAG = range(4)
WILSON_EVEN, WILSON_ODD, WILSON_FULL = range(3)
WILSON_PROBE_FMA_F64, WILSON_PROBE_FMA_F32, WILSON_PROBE_FMA_F32X2 = range(3)
WILSON_DD_ALL, WILSON_DD_INTERIOR, WILSON_DD_FACES = range(3)
PREC = {"f64": WILSON_F64, "f32": WILSON_F32, "f16": WILSON_F16, "bf16": WILSON_BF16}


class WilsonError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wilson status {code}: {msg}")
        self.code = code


class wilson_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("bc_phase", (ctypes.c_double * 2) * 4)]


class wilson_solver_params(ctypes.Structure):
    _fields_ = [("inner", ctypes.c_int), ("recon", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxiter", ctypes.c_int), ("max_restarts", ctypes.c_int), ("delta", ctypes.c_double),
                ("use_initial_guess", ctypes.c_int), ("reliable", ctypes.c_int), ("block_cg", ctypes.c_int)]


class wilson_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("hop_applications", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("inner_seconds", ctypes.c_double), ("outer_f32", ctypes.c_int)]


class wilson_problem(ctypes.Structure):
    _fields_ = [("L", wilson_lattice), ("kappa", ctypes.c_double), ("gauge", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class wilson_batch_info(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("device_seconds", ctypes.c_double), ("iterations", ctypes.c_int),
                ("graph_launches", ctypes.c_int), ("device_loop", ctypes.c_int), ("timed_out", ctypes.c_int),
                ("tiles", ctypes.c_int)]


_lib = None
VP = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double


def _declare(lib):
    P = ctypes.POINTER
    sig = {
        "wilson_dslash": (I, [VP, VP, VP, P(wilson_lattice), D, I, VP]),
        "wilson_dslash_eo": (I, [VP, VP, VP, P(wilson_lattice), I, D, I, VP]),
        "wilson_dslash_eo_noalloc": (I, [VP, VP, VP, P(wilson_lattice), I, D, I, VP]),
        "wilson_cg_solve": (I, [VP, VP, VP, P(wilson_lattice), D, P(wilson_solver_params),
                                P(wilson_solve_stats), VP]),
        "wilson_cg_solve_multi": (I, [VP, VP, VP, I, P(wilson_lattice), D, P(wilson_solver_params),
                                      P(wilson_solve_stats), VP]),
        "wilson_batch_solve": (I, [I, P(wilson_problem), P(wilson_solver_params), P(wilson_solve_stats),
                                   P(wilson_batch_info), VP]),
        "wilson_solver_defaults": (wilson_solver_params, [I]),
        "wilson_gauge_create": (I, [P(VP), VP, P(wilson_lattice), I, I, VP]),
        "wilson_gauge_destroy": (I, [VP]),
        "wilson_spinor_create": (I, [P(VP), P(wilson_lattice), I, I, I]),
        "wilson_spinor_destroy": (I, [VP]),
        "wilson_spinor_bytes": (ctypes.c_longlong, [VP]),
        "wilson_spinor_import": (I, [VP, VP, VP]),
        "wilson_spinor_export": (I, [VP, VP, VP]),
        "wilson_dslash_h": (I, [VP, VP, VP, D, I, VP]),
        "wilson_probe_fma_peak": (I, [I, P(D), VP]),
        "wilson_probe_hop_access": (I, [VP, VP, VP, I, P(D), VP]),
        "wilson_stage_timeouts": (I, [P(ctypes.c_ulonglong), VP]),
        "wilson_dd_halo_bytes": (ctypes.c_longlong, [P(wilson_lattice), I]),
        "wilson_dd_pack": (I, [VP, VP, VP, VP, I, VP]),
        "wilson_dd_hop": (I, [VP, VP, VP, VP, VP, I, I, I, I, VP]),
        "wilson_last_error": (ctypes.c_char_p, []),
        "wilson_version": (I, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0710_2442_gb300.build.build()")
        l = ctypes.CDLL(LIB_PATH)
        _declare(l)
        _lib = l
    return _lib


def _check(rc: int):
    if rc != WILSON_OK:
        raise WilsonError(rc, lib().wilson_last_error().decode(errors="replace"))


def lattice(dims, phases=(1, 1, 1, -1)) -> wilson_lattice:
    L = wilson_lattice()
    for mu in range(4):
        L.dims[mu] = int(dims[mu])
        z = complex(phases[mu])
        L.bc_phase[mu][0] = z.real
        L.bc_phase[mu][1] = z.imag
    return L


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()  # torch tensor


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def wilson_dslash(out, gauge, inp, L: wilson_lattice, kappa: float = 0.0, op: int = WILSON_OP_HOP, stream=None):
    _check(lib().wilson_dslash(_ptr(out), _ptr(gauge), _ptr(inp), ctypes.byref(L), float(kappa), int(op),
                               _stream(stream)))


def wilson_dslash_eo(out, gauge, inp, L: wilson_lattice, out_parity: int, kappa: float = 0.0,
                     op: int = WILSON_OP_HOP, stream=None):
    _check(lib().wilson_dslash_eo(_ptr(out), _ptr(gauge), _ptr(inp), ctypes.byref(L), int(out_parity),
                                  float(kappa), int(op), _stream(stream)))


def wilson_dslash_eo_noalloc(out, gauge, inp, L: wilson_lattice, out_parity: int, kappa: float = 0.0,
                             op: int = WILSON_OP_HOP, stream=None):
    """wilson_dslash_eo without device allocation (fixed 32 MiB scratch array;
    asynchronous; overlapping calls race)."""
    _check(lib().wilson_dslash_eo_noalloc(_ptr(out), _ptr(gauge), _ptr(inp), ctypes.byref(L), int(out_parity),
                                          float(kappa), int(op), _stream(stream)))


def solver_defaults(inner: int) -> wilson_solver_params:
    return lib().wilson_solver_defaults(int(inner))


def wilson_cg_solve(x, gauge, b, L: wilson_lattice, kappa: float, params: wilson_solver_params | None = None,
                    stream=None, check: bool = True) -> dict:
    p = params if params is not None else solver_defaults(WILSON_F16)
    st = wilson_solve_stats()
    rc = lib().wilson_cg_solve(_ptr(x), _ptr(gauge), _ptr(b), ctypes.byref(L), float(kappa), ctypes.byref(p),
                               ctypes.byref(st), _stream(stream))
    out = {f: getattr(st, f) for f, _ in wilson_solve_stats._fields_}
    out["rc"] = rc
    if check:
        _check(rc)
    return out


def wilson_cg_solve_multi(x, gauge, b, nrhs: int, L: wilson_lattice, kappa: float,
                          params: wilson_solver_params | None = None, stream=None, check: bool = True):
    """nrhs independent solves sharing one gauge field; x, b: [nrhs, V, 4, 3].
    Returns (rc, [per-rhs stats dicts])."""
    p = params if params is not None else solver_defaults(WILSON_F16)
    st = (wilson_solve_stats * int(nrhs))()
    rc = lib().wilson_cg_solve_multi(_ptr(x), _ptr(gauge), _ptr(b), int(nrhs), ctypes.byref(L), float(kappa),
                                     ctypes.byref(p), st, _stream(stream))
    out = [{f: getattr(st[k], f) for f, _ in wilson_solve_stats._fields_} for k in range(int(nrhs))]
    if check:
        _check(rc)
    return rc, out


def wilson_batch_solve(problems, params: wilson_solver_params | None = None, stream=None, check: bool = True):
    """Independent solves of different lattices in one graph launch.

    problems: list of dicts with keys L (wilson_lattice), kappa, gauge, b, x
    (device tensors in the canonical layout).  Returns (rc, [per-problem
    stats dicts], batch info dict)."""
    n = len(problems)
    arr = (wilson_problem * n)()
    for i, q in enumerate(problems):
        arr[i].L = q["L"]
        arr[i].kappa = float(q["kappa"])
        arr[i].gauge = _ptr(q["gauge"])
        arr[i].b = _ptr(q["b"])
        arr[i].x = _ptr(q["x"])
    p = params if params is not None else solver_defaults(WILSON_F16)
    st = (wilson_solve_stats * n)()
    info = wilson_batch_info()
    rc = lib().wilson_batch_solve(n, arr, ctypes.byref(p), st, ctypes.byref(info), _stream(stream))
    out = [{f: getattr(st[k], f) for f, _ in wilson_solve_stats._fields_} for k in range(n)]
    inf = {f: getattr(info, f) for f, _ in wilson_batch_info._fields_}
    if check:
        _check(rc)
    return rc, out, inf


class Gauge:
    """wilson_gauge handle: links prepared in one precision and storage."""

    def __init__(self, canon, L: wilson_lattice, prec: int, recon: int, stream=None):
        self.h = VP()
        self.L = L
        self.prec = prec
        self.recon = recon
        _check(lib().wilson_gauge_create(ctypes.byref(self.h), _ptr(canon), ctypes.byref(L), int(prec), int(recon),
                                         _stream(stream)))

    def close(self):
        if self.h:
            _check(lib().wilson_gauge_destroy(self.h))
            self.h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Spinor:
    """wilson_spinor handle: one subset (even/odd/full) of nrhs fields."""

    def __init__(self, L: wilson_lattice, subset: int, prec: int, nrhs: int = 1):
        self.h = VP()
        self.L = L
        self.subset = subset
        self.prec = prec
        self.nrhs = nrhs
        _check(lib().wilson_spinor_create(ctypes.byref(self.h), ctypes.byref(L), int(subset), int(nrhs), int(prec)))

    @property
    def nbytes(self) -> int:
        return int(lib().wilson_spinor_bytes(self.h))

    def load(self, canon, stream=None):
        _check(lib().wilson_spinor_import(self.h, _ptr(canon), _stream(stream)))

    def store(self, canon, stream=None):
        _check(lib().wilson_spinor_export(self.h, _ptr(canon), _stream(stream)))

    def close(self):
        if self.h:
            _check(lib().wilson_spinor_destroy(self.h))
            self.h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wilson_dd_halo_bytes(L: wilson_lattice, prec: int) -> int:
    n = lib().wilson_dd_halo_bytes(ctypes.byref(L), int(prec))
    if n < 0:
        raise WilsonError(WILSON_ERR_ARG, lib().wilson_last_error().decode(errors="replace"))
    return int(n)


def wilson_dd_pack(send_prev, send_next, gauge: "Gauge", inp: "Spinor", dagger: int = 0, stream=None):
    _check(lib().wilson_dd_pack(_ptr(send_prev), _ptr(send_next), gauge.h, inp.h, int(dagger), _stream(stream)))


def wilson_dd_hop(out: "Spinor", gauge: "Gauge", inp: "Spinor", recv_next, recv_prev, dagger: int = 0,
                  t_first: int = 1, t_last: int = 1, part: int = 0, stream=None):
    _check(lib().wilson_dd_hop(out.h, gauge.h, inp.h, _ptr(recv_next), _ptr(recv_prev), int(dagger),
                               int(t_first), int(t_last), int(part), _stream(stream)))


def wilson_probe_fma_peak(kind: int, stream=None) -> float:
    """Measured peak GFLOP/s of one FMA kind (WILSON_PROBE_FMA_*)."""
    v = ctypes.c_double(0.0)
    _check(lib().wilson_probe_fma_peak(int(kind), ctypes.byref(v), _stream(stream)))
    return v.value


def wilson_probe_hop_access(out: "Spinor", gauge: "Gauge", inp: "Spinor", reps: int = 50, stream=None) -> float:
    """Seconds per launch of the even-odd hop's memory accesses with trivial
    arithmetic (overwrites out with a checksum, not a spinor)."""
    v = ctypes.c_double(0.0)
    _check(lib().wilson_probe_hop_access(out.h, gauge.h, inp.h, int(reps), ctypes.byref(v), _stream(stream)))
    return v.value


def wilson_stage_timeouts(stream=None) -> int:
    """Bounded waits in the library's kernels that gave up (0 when healthy)."""
    v = ctypes.c_ulonglong(0)
    _check(lib().wilson_stage_timeouts(ctypes.byref(v), _stream(stream)))
    return v.value


def wilson_dslash_h(out: Spinor, gauge: Gauge, inp: Spinor, kappa: float = 0.0, op: int = WILSON_OP_HOP,
                    stream=None):
    _check(lib().wilson_dslash_h(out.h, gauge.h, inp.h, float(kappa), int(op), _stream(stream)))
