"""wilson_dslash_eo_noalloc: the even-odd operator without device allocation.

It exists for callers that cannot let the library allocate device memory:
hosts whose allocator owns the whole device, and loops that must never
block in an allocator.  Checked through the C ABI against wilson_dslash_eo,
the allocating entry point with the same semantics, at the FP64 tolerance
(1e-13 relative L2), on two calls in a row (the second sees the first call's
leftovers in the shared scratch array), at the largest lattice the array
holds, and with the device's free memory unchanged across a call.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

from conftest import assert_parity
from gpu_helpers import dev, empty_like_dev, host
from paper_0710_2442_gb300 import inputs

pytestmark = pytest.mark.gpu

PHASES = (np.exp(0.4j), 1.0, np.exp(-2.2j), -1.0)


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


def reference(w, U, src, L, parity, kappa, op):
    out = empty_like_dev(src)
    w.wilson_dslash_eo(out, U, src, L, parity, kappa, op)
    return host(out)


def test_noalloc_matches_allocating_call_twice(w):
    import torch
    dims = (12, 12, 12, 12)  # V/2 = 10368: near the scratch's range, several blocks
    L = w.lattice(dims, PHASES)
    U = dev(inputs.gauge_field(dims, "random", seed=301))
    Vh = inputs.volume(dims) // 2
    calls = [(dev(inputs.gaussian_spinor(Vh, seed=302)), 1, 0.0, w.WILSON_OP_HOP),
             (dev(inputs.gaussian_spinor(Vh, seed=303)), 0, 0.1350, w.WILSON_OP_SCHUR)]
    for src, parity, kappa, op in calls:
        out = empty_like_dev(np.zeros((Vh, 4, 3)))
        w.wilson_dslash_eo_noalloc(out, U, src, L, parity, kappa, op)
        torch.cuda.synchronize()
        got = host(out)
        want = reference(w, U, src, L, parity, kappa, op)
        assert_parity(got, want, 1e-13)


def test_noalloc_small_lattice_and_dagger(w):
    import torch
    dims = (4, 4, 4, 8)
    L = w.lattice(dims, PHASES)
    U = dev(inputs.gauge_field(dims, "random", seed=304))
    Vh = inputs.volume(dims) // 2
    src = dev(inputs.gaussian_spinor(Vh, seed=305))
    for op in (w.WILSON_OP_SCHUR_DAG, w.WILSON_OP_HOP):
        out = empty_like_dev(np.zeros((Vh, 4, 3)))
        w.wilson_dslash_eo_noalloc(out, U, src, L, 1, 0.125, op)
        torch.cuda.synchronize()
        assert_parity(host(out), reference(w, U, src, L, 1, 0.125, op), 1e-13)


def test_noalloc_rejects_lattice_beyond_scratch(w):
    dims = (16, 16, 16, 16)  # V/2 = 32768 needs ~57 MB of packed fields
    L = w.lattice(dims)
    buf = dev(np.zeros((64, 4, 3)))
    with pytest.raises(w.WilsonError, match="too large") as e:
        w.wilson_dslash_eo_noalloc(buf, buf, dev(np.zeros((64, 4, 3))), L, 0)
    assert e.value.code == w.WILSON_ERR_ARG


def test_noalloc_at_the_scratch_limit(w):
    """12^3 x 22 (V/2 = 19008) is the largest 12^3 x Lt lattice whose packed
    fields fit the 32 MiB array (32,845,824 bytes); 12^3 x 24 needs
    35,831,808 bytes and is rejected before any work."""
    import torch
    dims = (12, 12, 12, 22)
    L = w.lattice(dims, PHASES)
    U = dev(inputs.gauge_field(dims, "random", seed=306))
    Vh = inputs.volume(dims) // 2
    src = dev(inputs.gaussian_spinor(Vh, seed=307))
    for op, parity in ((w.WILSON_OP_SCHUR, 0), (w.WILSON_OP_HOP, 1)):
        out = empty_like_dev(np.zeros((Vh, 4, 3)))
        w.wilson_dslash_eo_noalloc(out, U, src, L, parity, 0.1350, op)
        torch.cuda.synchronize()
        assert_parity(host(out), reference(w, U, src, L, parity, 0.1350, op), 1e-13)
    big = w.lattice((12, 12, 12, 24))
    buf = dev(np.zeros((64, 4, 3)))
    with pytest.raises(w.WilsonError, match="too large") as e:
        w.wilson_dslash_eo_noalloc(buf, buf, dev(np.zeros((64, 4, 3))), big, 0)
    assert e.value.code == w.WILSON_ERR_ARG


def test_noalloc_leaves_device_memory_unchanged(w):
    """After a first call (which loads the kernels' code), further calls
    change neither the device's free memory nor torch's allocator."""
    import torch
    dims = (8, 8, 8, 8)
    L = w.lattice(dims, PHASES)
    U = dev(inputs.gauge_field(dims, "random", seed=308))
    Vh = inputs.volume(dims) // 2
    src = dev(inputs.gaussian_spinor(Vh, seed=309))
    out = empty_like_dev(np.zeros((Vh, 4, 3)))
    w.wilson_dslash_eo_noalloc(out, U, src, L, 0, 0.125, w.WILSON_OP_SCHUR_DAG)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        w.wilson_dslash_eo_noalloc(out, U, src, L, 0, 0.125, w.WILSON_OP_SCHUR_DAG)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert_parity(host(out), reference(w, U, src, L, 0, 0.125, w.WILSON_OP_SCHUR_DAG), 1e-13)
