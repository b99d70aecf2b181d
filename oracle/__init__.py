"""FP64 CPU oracle for the Wilson hopping term (Eq. 3) and the CG solve.

TEST INFRASTRUCTURE ONLY: the GPU library never imports, links or calls this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code with the GPU path; both sides
only share the seeded input generators.

The arithmetic lives in ``wilson_oracle.c`` (plain C, FP64, OpenMP over
sites); this module compiles it with gcc on first use and wraps it for numpy
arrays in the canonical layout:

* spinor  ``complex128[V, 4, 3]``      (site, spin, colour)
* gauge   ``complex128[V, 4, 3, 3]``   (site, mu = x,y,z,t, row, col)
* half (checkerboard) fields ``complex128[V/2, 4, 3]``: site ``s`` of parity
  ``(x+y+z+t) % 2`` is stored at ``s >> 1``
* site index ``s = x + Lx*(y + Ly*(z + Lz*t))``
* boundary phases ``complex[4]``: the factor a forward hop picks up when it
  wraps from ``x_mu = L_mu - 1`` to ``0`` (the backward hop takes its
  conjugate).

Parity pins: see ``tests/test_oracle_*.py`` (free-field closed form,
gamma_5-hermiticity, gauge covariance, dense brute force, the convention
identity of Eq. 3, CG against a dense LU solve).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libwilson_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp).  Returns the .so path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def declare(lib):
    """Set the ctypes signatures of an oracle library handle."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_gamma.argtypes = [ctypes.c_int, dp]
    lib.oracle_gamma.restype = None
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_get_num_threads.restype = ctypes.c_int
    lib.oracle_dslash.argtypes = [dp, dp, dp, ip, dp, ctypes.c_int]
    lib.oracle_wilson_m.argtypes = [dp, dp, dp, ip, dp, ctypes.c_double]
    lib.oracle_dslash_eo.argtypes = [dp, dp, dp, ip, dp, ctypes.c_int, ctypes.c_int]
    lib.oracle_schur.argtypes = [dp, dp, dp, ip, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.oracle_cg.argtypes = [dp, dp, dp, ip, dp, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int, ip, dp]
    for f in (lib.oracle_dslash, lib.oracle_wilson_m, lib.oracle_dslash_eo,
              lib.oracle_schur, lib.oracle_cg):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = declare(ctypes.CDLL(build()))
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims(dims) -> np.ndarray:
    d = np.ascontiguousarray(dims, dtype=np.int32)
    if d.shape != (4,):
        raise ValueError("dims must have 4 entries (Lx, Ly, Lz, Lt)")
    return d


def _phases(phases) -> np.ndarray:
    if phases is None:
        phases = (1, 1, 1, -1)
    return _c128(np.asarray(phases, dtype=np.complex128).reshape(4))


def _check(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle {what}: bad arguments (rc={rc})")


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def num_threads() -> int:
    return int(_load().oracle_get_num_threads())


def gamma(mu: int) -> np.ndarray:
    """The oracle's gamma matrix: mu = 0..3 for gamma_1..gamma_4, 4 for gamma_5."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().oracle_gamma(int(mu), _dp(out))
    return out


def dslash(gauge, psi, dims, phases=None, conv: int = 1) -> np.ndarray:
    """Full-lattice hopping term D_h psi (Eq. 3).  conv=+1: (1-gamma) forward,
    conv=-1: (1+gamma) forward as printed in Eq. 3."""
    d = _dims(dims)
    V = int(np.prod(d))
    U = _c128(gauge).reshape(V, 4, 3, 3)
    x = _c128(psi).reshape(V, 4, 3)
    out = np.empty_like(x)
    ph = _phases(phases)
    _check(_load().oracle_dslash(_dp(out), _dp(U), _dp(x), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 _dp(ph), int(conv)), "dslash")
    return out


def wilson_m(gauge, psi, dims, kappa: float, phases=None) -> np.ndarray:
    """Full Wilson operator M psi = psi - kappa D_h psi."""
    d = _dims(dims)
    V = int(np.prod(d))
    U = _c128(gauge).reshape(V, 4, 3, 3)
    x = _c128(psi).reshape(V, 4, 3)
    out = np.empty_like(x)
    ph = _phases(phases)
    _check(_load().oracle_wilson_m(_dp(out), _dp(U), _dp(x), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   _dp(ph), float(kappa)), "wilson_m")
    return out


def dslash_eo(gauge, psi_half, dims, out_parity: int, phases=None, conv: int = 1) -> np.ndarray:
    """D_{p,1-p}: hop from the (1-p) half field to the p half field."""
    d = _dims(dims)
    V = int(np.prod(d))
    U = _c128(gauge).reshape(V, 4, 3, 3)
    x = _c128(psi_half).reshape(V // 2, 4, 3)
    out = np.empty_like(x)
    ph = _phases(phases)
    _check(_load().oracle_dslash_eo(_dp(out), _dp(U), _dp(x), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    _dp(ph), int(out_parity), int(conv)), "dslash_eo")
    return out


def schur(gauge, psi_half, dims, kappa: float, parity: int = 0, dagger: bool = False,
          phases=None) -> np.ndarray:
    """Mhat_p = 1 - kappa^2 D_{p,1-p} D_{1-p,p} (dagger: gamma_5 Mhat gamma_5)."""
    d = _dims(dims)
    V = int(np.prod(d))
    U = _c128(gauge).reshape(V, 4, 3, 3)
    x = _c128(psi_half).reshape(V // 2, 4, 3)
    out = np.empty_like(x)
    ph = _phases(phases)
    _check(_load().oracle_schur(_dp(out), _dp(U), _dp(x), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                _dp(ph), float(kappa), int(parity), int(bool(dagger))), "schur")
    return out


def cg_solve(gauge, b, dims, kappa: float, tol: float = 1e-10, maxiter: int = 100000,
             phases=None):
    """Solve M x = b (full lattice) through the even Schur complement with CGNR.

    Returns (x, info) with info = {converged, iterations, schur_applications,
    true_rel_resid}."""
    d = _dims(dims)
    V = int(np.prod(d))
    U = _c128(gauge).reshape(V, 4, 3, 3)
    bb = _c128(b).reshape(V, 4, 3)
    x = np.empty_like(bb)
    ph = _phases(phases)
    info = np.zeros(2, dtype=np.int32)
    res = np.zeros(1, dtype=np.float64)
    rc = _load().oracle_cg(_dp(x), _dp(U), _dp(bb), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           _dp(ph), float(kappa), float(tol), int(maxiter),
                           info.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(res))
    _check(rc, "cg")
    return x, {"converged": rc == 0, "iterations": int(info[0]),
               "schur_applications": int(info[1]), "true_rel_resid": float(res[0])}
