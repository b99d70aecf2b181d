"""The C ABI library builds for sm_103a, loads, exports every symbol that
include/*.h declares, and rejects invalid arguments on the host (no GPU
needed: validation happens before any device call)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(wilson_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(w):
    lib = ctypes.CDLL(w.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version(w):
    assert w.lib().wilson_version() >= 100


def _status(w, fn):
    try:
        fn()
    except w.WilsonError as e:
        return e.code
    return 0


@pytest.mark.parametrize("dims", [(4, 4, 3, 4), (0, 4, 4, 4), (4, 4, 4, 1)])
def test_bad_dims_rejected(w, dims):
    L = w.lattice(dims)
    buf = np.zeros(16, dtype=np.complex128)
    assert _status(w, lambda: w.wilson_dslash(buf.ctypes.data + 0, buf, buf.ctypes.data + 64, L, 0.1)) \
        == w.WILSON_ERR_ARG


def test_bad_phase_null_and_alias_rejected(w):
    buf = np.zeros(64, dtype=np.complex128)
    L = w.lattice((4, 4, 4, 4), phases=(1, 1, 1, 2.0))
    assert _status(w, lambda: w.wilson_dslash(buf, buf, buf.ctypes.data + 256, L, 0.1)) == w.WILSON_ERR_ARG
    L = w.lattice((4, 4, 4, 4))
    assert _status(w, lambda: w.wilson_dslash(0, buf, buf, L, 0.1)) == w.WILSON_ERR_ARG
    assert _status(w, lambda: w.wilson_dslash(buf, buf, buf, L, 0.1)) == w.WILSON_ERR_ARG
    assert _status(w, lambda: w.wilson_dslash(buf.ctypes.data + 8, buf, buf.ctypes.data + 256, L, 0.1)) \
        == w.WILSON_ERR_ARG  # misaligned
    assert _status(w, lambda: w.wilson_dslash(buf, buf, buf.ctypes.data + 256, L, float("nan"))) \
        == w.WILSON_ERR_ARG
    assert _status(w, lambda: w.wilson_dslash_eo(buf, buf, buf.ctypes.data + 256, L, 2)) == w.WILSON_ERR_ARG
    assert _status(w, lambda: w.wilson_dslash_eo(buf, buf, buf.ctypes.data + 256, L, 0, 0.1, w.WILSON_OP_M)) \
        == w.WILSON_ERR_ARG


def test_probe_arguments_rejected(w):
    """The probes check their arguments before any device call."""
    import ctypes
    v = ctypes.c_double(0.0)
    lib = w.lib()
    assert lib.wilson_probe_hop_access(None, None, None, 3, ctypes.byref(v), None) == w.WILSON_ERR_ARG
    assert lib.wilson_probe_fma_peak(7, ctypes.byref(v), None) == w.WILSON_ERR_ARG
    assert lib.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F64, None, None) == w.WILSON_ERR_ARG
    assert lib.wilson_stage_timeouts(None, None) == w.WILSON_ERR_ARG


def test_last_error_message(w):
    buf = np.zeros(64, dtype=np.complex128)
    L = w.lattice((4, 4, 3, 4))
    with pytest.raises(w.WilsonError, match="even"):
        w.wilson_dslash(buf, buf, buf.ctypes.data + 256, L, 0.1)


def test_no_device_is_an_error_not_a_fallback(w):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    buf = np.zeros(64, dtype=np.complex128)
    L = w.lattice((2, 2, 2, 2))
    assert _status(w, lambda: w.wilson_dslash(buf, buf, buf.ctypes.data + 256, L, 0.1)) == w.WILSON_ERR_CUDA


def test_solver_defaults(w):
    p = w.solver_defaults(w.WILSON_F16)
    assert p.inner == w.WILSON_F16 and p.recon == 12 and p.tol == 1e-10 and p.reliable == 1
    assert p.block_cg == 0
    p = w.solver_defaults(w.WILSON_F64)
    assert p.recon == 18


def test_block_cg_rhs_limit(w):
    """Block CG carries at most 16 right-hand sides; more is an argument error
    raised before any device call."""
    buf = np.zeros(64, dtype=np.complex128)
    L = w.lattice((2, 2, 2, 2))
    p = w.solver_defaults(w.WILSON_F16)
    p.block_cg = 1
    call = lambda: w.wilson_cg_solve_multi(buf, buf.ctypes.data + 256, buf.ctypes.data + 512, 17, L, 0.1, p,
                                           check=False)[0]
    assert call() == w.WILSON_ERR_ARG
    assert "16" in w.lib().wilson_last_error().decode()


def test_batch_and_multi_rhs_arguments_rejected(w):
    """Batched and multi-RHS solves validate their arguments before any
    device call: an empty batch, an FP64 or 18-real inner operator, an odd
    extent, x aliasing b, and right-hand-side counts outside 1..64."""
    buf = np.zeros(4096, dtype=np.complex128)
    base = buf.ctypes.data
    L = w.lattice((4, 4, 4, 4))

    def prob(dims=(4, 4, 4, 4), b_off=512, x_off=1024):
        return dict(L=w.lattice(dims), kappa=0.12, gauge=base, b=base + b_off, x=base + x_off)

    def batch(probs, inner=w.WILSON_F16, recon=12):
        p = w.solver_defaults(inner)
        p.recon = recon
        return w.wilson_batch_solve(probs, p, check=False)[0]

    assert batch([]) == w.WILSON_ERR_ARG
    assert batch([prob()], inner=w.WILSON_F64) == w.WILSON_ERR_ARG
    assert batch([prob()], recon=18) == w.WILSON_ERR_ARG
    assert batch([prob(), prob(dims=(4, 4, 3, 4))]) == w.WILSON_ERR_ARG
    assert batch([prob(b_off=512, x_off=512)]) == w.WILSON_ERR_ARG
    p = w.solver_defaults(w.WILSON_F16)
    for nrhs in (0, 65):
        rc, _ = w.wilson_cg_solve_multi(base + 1024, base, base + 512, nrhs, L, 0.12, p, check=False)
        assert rc == w.WILSON_ERR_ARG


def test_environment_variables_documented():
    """The header's environment section lists exactly the variables the
    library reads (getenv, or the autotuner's flag helper)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    header = open(os.path.join(root, "include", "wilson.h")).read()
    section = header[header.index(" * Environment"):header.index(" */", header.index(" * Environment"))]
    documented = set(re.findall(r"\b(WILSON_[A-Z_]+)=", section))
    csrc = os.path.join(root, "paper_0710_2442_gb300", "csrc")
    read = set()
    for name in os.listdir(csrc):
        if name.endswith((".cu", ".cuh", ".h")):
            text = open(os.path.join(csrc, name)).read()
            read |= set(re.findall(r'(?:getenv|env_flag)\("(WILSON_[A-Z_]+)"', text))
    assert documented == read, (sorted(documented - read), sorted(read - documented))
