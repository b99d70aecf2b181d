"""The measurement probes on the GPU: the FMA peak kernels and the even-odd
hop's access-pattern kernel (Sec. 5, after Table 1: the paper's benchmark of
Eq. 3's memory-access pattern against T_mem).

The access probe makes the hop's loads and stores with the arithmetic taken
out, so it must run no slower than the hop itself on a lattice larger than
L2, write only its output field (the input and the links still give the
oracle's hop afterwards), and reject handles that the hop would reject.
"""
import numpy as np
import pytest

from conftest import assert_parity
from gpu_helpers import dev, empty_like_dev, host
from paper_0710_2442_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3}


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


def test_fma_peaks(w):
    f64 = w.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F64)
    f32 = w.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F32)
    f32x2 = w.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F32X2)
    assert all(np.isfinite(v) and v > 0 for v in (f64, f32, f32x2))
    # GB300 runs FP64 at a small fraction of its FP32 rate
    assert f64 < f32
    assert 0.5 * f32 < f32x2 < 4.0 * f32


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("f32", 12), ("f32", 18), ("f16", 12),
                                        ("bf16", 18)])
def test_access_probe_leaves_inputs_intact(w, oracle_mod, prec, recon):
    dims = (6, 4, 6, 10)
    phases = (np.exp(0.4j), 1.0, np.exp(-2.2j), -1.0)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=301)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=302)
    L = w.lattice(dims, phases)
    P = w.PREC[prec]
    g = w.Gauge(U, L, P, recon)
    a = w.Spinor(L, w.WILSON_EVEN, P)
    b = w.Spinor(L, w.WILSON_ODD, P)
    a.load(dev(src))
    t = w.wilson_probe_hop_access(b, g, a, reps=3)
    assert np.isfinite(t) and 0 < t < 1.0
    w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP)
    out = empty_like_dev(src)
    b.store(out)
    assert_parity(host(out), oracle_mod.dslash_eo(U, src, dims, 1, phases), TOL[prec])
    for h in (g, a, b):
        h.close()


def test_access_probe_rejects_bad_handles(w):
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=303)
    L = w.lattice(dims)
    g = w.Gauge(U, L, w.WILSON_F32, 12)
    even = w.Spinor(L, w.WILSON_EVEN, w.WILSON_F32)
    even2 = w.Spinor(L, w.WILSON_EVEN, w.WILSON_F32)
    odd16 = w.Spinor(L, w.WILSON_ODD, w.WILSON_F16)
    odd = w.Spinor(L, w.WILSON_ODD, w.WILSON_F32)
    bad = [(even2, g, even, 3), (odd16, g, even, 3), (odd, g, even, 0)]
    for out, gg, inp, reps in bad:
        with pytest.raises(w.WilsonError):
            w.wilson_probe_hop_access(out, gg, inp, reps=reps)
    for h in (g, even, even2, odd16, odd):
        h.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_access_probe_no_slower_than_the_hop(w, prec):
    """On 32^3 x 64 (fields larger than L2) the probe's time is at most the
    tuned hop's: the same DRAM accesses with less work between them."""
    import torch
    dims = (32, 32, 32, 64)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=2452)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=31)
    L = w.lattice(dims)
    P = w.PREC[prec]
    g = w.Gauge(U, L, P, 12)
    a = w.Spinor(L, w.WILSON_EVEN, P)
    b = w.Spinor(L, w.WILSON_ODD, P)
    a.load(dev(src))
    stream = torch.cuda.current_stream()
    for _ in range(5):
        w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_hop = e0.elapsed_time(e1) / 1e3 / 20
    t_probe = w.wilson_probe_hop_access(b, g, a, reps=20, stream=stream)
    assert t_probe <= 1.02 * t_hop, (t_probe, t_hop)
    for h in (g, a, b):
        h.close()
