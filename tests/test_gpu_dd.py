"""The t-decomposed even-odd hop on one GPU: the lattice split into 1, 2 or 4
sub-lattices, face buffers packed by wilson_dd_pack, moved by device copies
(the loopback exchange), applied by wilson_dd_hop, and the gathered result
compared element by element with the oracle's D_{p,1-p} on the whole lattice
(FP64 1e-13, FP32 1e-6), with complex boundary phases, both output parities
and the dagger projectors."""
import numpy as np
import pytest

from conftest import assert_parity
from gpu_helpers import dev, host
from paper_0710_2442_gb300 import inputs
from paper_0710_2442_gb300.dd import TSplit, exchange_loopback

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6}
PHASES = (np.exp(0.4j), 1.0, np.exp(-2.2j), np.exp(2.9j))


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


def dd_apply(w, U, src, dims, n, prec, recon, out_parity, dagger, phases, split=False):
    """split: the interior t-slices are applied before the exchange (with no
    face buffers), the two face slices after it."""
    import torch
    sp = TSplit(dims, n)
    L = w.lattice(sp.local_dims, phases)
    P = w.PREC[prec]
    pin = 1 - out_parity
    hb = w.wilson_dd_halo_bytes(L, P)
    gauges = [w.Gauge(u, L, P, recon) for u in sp.split_gauge(U)]
    ins = [w.Spinor(L, pin, P) for _ in range(n)]
    outs = [w.Spinor(L, out_parity, P) for _ in range(n)]
    for s_, part in zip(ins, sp.split_half(src)):
        s_.load(dev(part))
    buf = lambda: [torch.empty(hb, dtype=torch.uint8, device="cuda") for _ in range(n)]
    send_prev, send_next, recv_next, recv_prev = buf(), buf(), buf(), buf()
    for r in range(n):
        w.wilson_dd_pack(send_prev[r], send_next[r], gauges[r], ins[r], dagger)
    if split:
        for r in range(n):
            w.wilson_dd_hop(outs[r], gauges[r], ins[r], None, None, dagger, sp.first(r), sp.last(r),
                            w.WILSON_DD_INTERIOR)
    exchange_loopback(sp, send_prev, send_next, recv_next, recv_prev)
    for r in range(n):
        w.wilson_dd_hop(outs[r], gauges[r], ins[r], recv_next[r], recv_prev[r], dagger, sp.first(r), sp.last(r),
                        w.WILSON_DD_FACES if split else w.WILSON_DD_ALL)
    parts = []
    for o in outs:
        t = torch.full((sp.Lr * sp.Vs // 2, 4, 3), float("nan"), dtype=torch.complex128, device="cuda")
        o.store(t)
        parts.append(host(t))
    for h in gauges + ins + outs:
        h.close()
    return sp.gather_half(parts)


@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f64", 12), ("f32", 18)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dd_hop_matches_oracle(w, oracle_mod, n, prec, recon, out_parity):
    dims = (4, 6, 4, 8)
    U = inputs.gauge_field(dims, "random", seed=401)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=402)
    got = dd_apply(w, U, src, dims, n, prec, recon, out_parity, 0, PHASES)
    want = oracle_mod.dslash_eo(U, src, dims, out_parity, PHASES)
    assert_parity(got, want, TOL[prec])


@pytest.mark.parametrize("n", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dd_hop_dagger(w, oracle_mod, n, prec):
    """The dagger projectors (the hop of g5 D g5, Eq. 3 as printed)."""
    dims = (6, 4, 2, 4)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=403)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=404)
    got = dd_apply(w, U, src, dims, n, prec, 12 if prec == "f32" else 18, 1, 1, PHASES)
    want = oracle_mod.dslash_eo(U, src, dims, 1, PHASES, conv=-1)
    assert_parity(got, want, TOL[prec])


@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12)])
def test_dd_interior_then_faces(w, oracle_mod, n, prec, recon):
    """The interior t-slices (no face buffers) before the exchange and the
    face slices after it give the whole operator; with Lr = 2 (n = 4) the
    interior is empty."""
    dims = (4, 6, 4, 8)
    U = inputs.gauge_field(dims, "random", seed=406)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=407)
    for out_parity in (0, 1):
        got = dd_apply(w, U, src, dims, n, prec, recon, out_parity, 0, PHASES, split=True)
        assert_parity(got, oracle_mod.dslash_eo(U, src, dims, out_parity, PHASES), TOL[prec])


def test_dd_halo_bytes_and_argument_checks(w):
    import torch
    L = w.lattice((4, 4, 4, 4))
    # Vs/2 = 32 face sites, stride rounded up to 64
    assert w.wilson_dd_halo_bytes(L, w.WILSON_F64) == 96 * 64
    assert w.wilson_dd_halo_bytes(L, w.WILSON_F32) == 48 * 64
    with pytest.raises(w.WilsonError):
        w.wilson_dd_halo_bytes(L, w.WILSON_F16)
    g = w.Gauge(inputs.gauge_field((4, 4, 4, 4), "weak", eps=0.3, seed=405), L, w.WILSON_F32, 12)
    a = w.Spinor(L, 0, w.WILSON_F32)
    b = w.Spinor(L, 0, w.WILSON_F32)
    buf = torch.empty(48 * 64, dtype=torch.uint8, device="cuda")
    buf2 = torch.empty(48 * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(w.WilsonError):  # out has the input's parity
        w.wilson_dd_hop(b, g, a, buf, buf2)
    with pytest.raises(w.WilsonError):  # one buffer for both faces
        w.wilson_dd_pack(buf, buf, g, a)
    c = w.Spinor(L, 1, w.WILSON_F32)
    with pytest.raises(w.WilsonError):  # the faces need their buffers
        w.wilson_dd_hop(c, g, a, None, None, 0, 1, 1, w.WILSON_DD_FACES)
    with pytest.raises(w.WilsonError):  # unknown part
        w.wilson_dd_hop(c, g, a, buf, buf2, 0, 1, 1, 3)
    c.close()
    for h in (g, a, b):
        h.close()
