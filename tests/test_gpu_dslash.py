"""Parity of the CUDA hopping term against the FP64 CPU oracle, element by
element, through the C ABI.

Tolerances (relative L2 over the whole output): 1e-13 for FP64 fields,
1e-6 for FP32, 5e-3 for FP16 / BF16 storage; every component must also lie
within 10x that tolerance times the RMS modulus of the oracle's output.  Sizes span several 128-site
blocks with a ragged tail (Vh not a multiple of the block size) plus the
8^4 random-SU(3) lattice of the FP64 workload and the 32^3 x 64 weak-field
lattice of the FP32 even-odd workload.
"""
import numpy as np
import pytest

from conftest import assert_parity, parity_merge, parity_split
from gpu_helpers import dev, empty_like_dev, handle_hop, host
from paper_0710_2442_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3}
CPLX_PHASES = (np.exp(0.4j), 1.0, np.exp(-2.2j), -1.0)
SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 6, 10), (8, 6, 4, 10), (8, 8, 8, 8), (4, 2, 2, 2)]


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("op", ["hop", "m"])
def test_f64_full_dslash(w, oracle_mod, dims, op):
    U = inputs.gauge_field(dims, "random", seed=101)
    psi = inputs.gaussian_spinor(dims, seed=102)
    kappa = 0.125
    L = w.lattice(dims, CPLX_PHASES)
    out = empty_like_dev(psi)
    w.wilson_dslash(out, dev(U), dev(psi), L, kappa, w.WILSON_OP_HOP if op == "hop" else w.WILSON_OP_M)
    got = host(out)
    want = oracle_mod.dslash(U, psi, dims, CPLX_PHASES) if op == "hop" else \
        oracle_mod.wilson_m(U, psi, dims, kappa, CPLX_PHASES)
    assert_parity(got, want, TOL["f64"])


def test_f64_config_8x8x8x8_default_phases(w, oracle_mod):
    cfg = inputs.WORKLOADS["dslash_f64_8^4"]
    dims = cfg["dims"]
    U = inputs.gauge_field(dims, cfg["gauge"], seed=cfg["gauge_seed"])
    psi = inputs.gaussian_spinor(dims, seed=cfg["spinor_seed"])
    L = w.lattice(dims)
    for op in (w.WILSON_OP_M, w.WILSON_OP_HOP):
        out = empty_like_dev(psi)
        w.wilson_dslash(out, dev(U), dev(psi), L, cfg["kappa"], op)
        want = oracle_mod.wilson_m(U, psi, dims, cfg["kappa"]) if op == w.WILSON_OP_M else \
            oracle_mod.dslash(U, psi, dims)
        assert_parity(host(out), want, TOL["f64"])


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("out_parity", [0, 1])
def test_f64_eo_hop(w, oracle_mod, dims, out_parity):
    U = inputs.gauge_field(dims, "random", seed=103)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=104)
    L = w.lattice(dims, CPLX_PHASES)
    out = empty_like_dev(src)
    w.wilson_dslash_eo(out, dev(U), dev(src), L, out_parity, 0.0, w.WILSON_OP_HOP)
    want = oracle_mod.dslash_eo(U, src, dims, out_parity, CPLX_PHASES)
    assert_parity(host(out), want, TOL["f64"])


def test_stateless_calls_do_not_synchronise(w, oracle_mod):
    """wilson_dslash_eo and wilson_dslash return before their stream has run
    them: two calls are queued behind a GPU busy-wait of about half a second,
    the stream is still busy when both have returned, and once it has run
    them both results match the oracle.  A first pair of calls outside the
    check tunes the launch configurations (that pass synchronises)."""
    import torch
    dims = (8, 6, 4, 10)
    U = inputs.gauge_field(dims, "random", seed=131)
    Vh = inputs.volume(dims) // 2
    src_h = inputs.gaussian_spinor(Vh, seed=132)
    src_f = inputs.gaussian_spinor(inputs.volume(dims), seed=133)
    L = w.lattice(dims, CPLX_PHASES)
    Ud, sh, sf = dev(U), dev(src_h), dev(src_f)
    out_h, out_f = empty_like_dev(src_h), empty_like_dev(src_f)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(2):
            w.wilson_dslash_eo(out_h, Ud, sh, L, 1, 0.135, w.WILSON_OP_SCHUR, stream)
            w.wilson_dslash(out_f, Ud, sf, L, 0.135, w.WILSON_OP_M, stream)
        stream.synchronize()
        out_h.fill_(float("nan"))
        out_f.fill_(float("nan"))
        torch.cuda._sleep(1_000_000_000)  # about 0.5 s of GPU time at 2 GHz
        w.wilson_dslash_eo(out_h, Ud, sh, L, 1, 0.135, w.WILSON_OP_SCHUR, stream)
        w.wilson_dslash(out_f, Ud, sf, L, 0.135, w.WILSON_OP_M, stream)
        still_busy = not stream.query()
        stream.synchronize()
    assert still_busy, "a stateless call waited for its stream"
    assert_parity(host(out_h), oracle_mod.schur(U, src_h, dims, 0.135, 1, False, CPLX_PHASES), TOL["f64"])
    assert_parity(host(out_f), oracle_mod.wilson_m(U, src_f, dims, 0.135, CPLX_PHASES), TOL["f64"])


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10), (2, 2, 2, 4)])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("dag", [False, True])
def test_f64_schur(w, oracle_mod, dims, parity, dag):
    U = inputs.gauge_field(dims, "random", seed=105)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=106)
    kappa = 0.135
    L = w.lattice(dims, CPLX_PHASES)
    out = empty_like_dev(src)
    w.wilson_dslash_eo(out, dev(U), dev(src), L, parity, kappa,
                       w.WILSON_OP_SCHUR_DAG if dag else w.WILSON_OP_SCHUR)
    want = oracle_mod.schur(U, src, dims, kappa, parity, dag, CPLX_PHASES)
    assert_parity(host(out), want, TOL["f64"])


LOWP = [("f64", 18), ("f64", 12), ("f32", 12), ("f32", 18), ("f16", 12), ("bf16", 12), ("f16", 18), ("bf16", 18)]


@pytest.mark.parametrize("prec,recon", LOWP)
@pytest.mark.parametrize("dims", [(6, 4, 6, 10), (8, 6, 4, 10), (4, 4, 4, 4)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_handle_eo_hop(w, oracle_mod, prec, recon, dims, out_parity):
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=107)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=108)
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], recon, 1 - out_parity, out_parity,
                     w.WILSON_OP_HOP)
    want = oracle_mod.dslash_eo(U, src, dims, out_parity, CPLX_PHASES)
    assert_parity(got, want, TOL[prec])


@pytest.mark.parametrize("prec,recon", LOWP)
@pytest.mark.parametrize("op", ["hop", "m"])
def test_handle_full(w, oracle_mod, prec, recon, op):
    dims = (6, 4, 6, 10)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=109)
    psi = inputs.gaussian_spinor(dims, seed=110)
    kappa = 0.1350
    got = handle_hop(w, U, psi, dims, CPLX_PHASES, w.PREC[prec], recon, w.WILSON_FULL, w.WILSON_FULL,
                     w.WILSON_OP_HOP if op == "hop" else w.WILSON_OP_M, kappa)
    want = oracle_mod.dslash(U, psi, dims, CPLX_PHASES) if op == "hop" else \
        oracle_mod.wilson_m(U, psi, dims, kappa, CPLX_PHASES)
    assert_parity(got, want, TOL[prec])


def test_handle_multi_rhs_fields(w, oracle_mod):
    """nrhs fields in one handle: each is applied independently."""
    dims = (4, 4, 4, 6)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=111)
    Vh = inputs.volume(dims) // 2
    src = inputs.gaussian_spinor(Vh, seed=112, nrhs=3)
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.WILSON_F32, 12, 1, 0, w.WILSON_OP_HOP, nrhs=3)
    for k in range(3):
        want = oracle_mod.dslash_eo(U, src[k], dims, 0, CPLX_PHASES)
        assert_parity(got[k], want, TOL["f32"])


@pytest.fixture(scope="module")
def workload_32x32x32x64(oracle_mod):
    """The 32^3 x 64 even-odd workload's fields and the oracle's output."""
    cfg = inputs.WORKLOADS["dslash_eo_f32_32^3x64"]
    dims = cfg["dims"]
    U = inputs.gauge_field(dims, cfg["gauge"], eps=cfg["eps"], seed=cfg["gauge_seed"])
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=cfg["spinor_seed"]).astype(np.complex64)
    src = src.astype(np.complex128)  # the workload's spinor is complex64 data
    return dims, U, src, oracle_mod.dslash_eo(U, src, dims, 1)


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_eo_workload_32x32x32x64(w, workload_32x32x32x64, prec):
    """The even-odd workload at full size (Vh = 1,048,576), whole output
    compared with the oracle element by element, in the launch configuration
    the autotuner picks (the one the bench times), for the F32 headline
    storage and for the F16 / BF16 storage of the inner solver."""
    dims, U, src, want = workload_32x32x32x64
    got = handle_hop(w, U, src, dims, inputs.DEFAULT_PHASES, w.PREC[prec], 12, 0, 1, w.WILSON_OP_HOP)
    assert_parity(got, want, TOL[prec])


def test_nan_sentinels_overwritten(w):
    """Every output site is written (outputs start as NaN)."""
    dims = (6, 4, 6, 10)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=113)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=114)
    for prec in ("f32", "f16"):
        got = handle_hop(w, U, src, dims, inputs.DEFAULT_PHASES, w.PREC[prec], 12, 0, 1, w.WILSON_OP_HOP)
        assert np.all(np.isfinite(got))


def test_zero_field_f16_scale(w):
    """A zero spinor has scale 0 and stays exactly zero through F16 storage."""
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=115)
    src = np.zeros((inputs.volume(dims) // 2, 4, 3), dtype=np.complex128)
    got = handle_hop(w, U, src, dims, inputs.DEFAULT_PHASES, w.WILSON_F16, 12, 0, 1, w.WILSON_OP_HOP)
    assert np.all(got == 0)


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f16", 12)])
@pytest.mark.parametrize("dag", [False, True])
def test_handle_schur(w, oracle_mod, prec, recon, dag):
    dims = (6, 4, 6, 10)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=116)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=117, nrhs=2)
    kappa = 0.1350
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], recon, 0, 0,
                     w.WILSON_OP_SCHUR_DAG if dag else w.WILSON_OP_SCHUR, kappa, nrhs=2)
    for k in range(2):
        want = oracle_mod.schur(U, src[k], dims, kappa, 0, dag, CPLX_PHASES)
        assert_parity(got[k], want, TOL[prec])


# Every kernel variant (register budgets 0-2 of the scalar stencil, 3-5 of the
# paired-FP32 stencil, 12-14 two or four sites per thread, 15-17 the F16
# projection on packed halves, 20-22 F16 with the neighbour data copied ahead
# into shared memory, 23-25 the scalar and paired stencils with L2 prefetches
# of the site's links and neighbours; a variant that does not fit a precision
# runs variant 3)
# against the oracle, pinned through WILSON_HOP_VARIANT so that the
# autotuner's choice does not decide which code is tested.
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 12, 13, 14, 15, 16, 17, 20, 21, 22, 23, 24, 25])
@pytest.mark.parametrize("prec,recon", [("f32", 12), ("f16", 12), ("bf16", 12), ("f32", 18), ("f16", 18)])
def test_every_variant_eo_and_schur(w, oracle_mod, monkeypatch, variant, prec, recon):
    monkeypatch.setenv("WILSON_HOP_VARIANT", str(variant))
    monkeypatch.setenv("WILSON_HOP_BLOCK", str((64, 128, 256)[variant % 3]))
    dims = (6, 4, 6, 10)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=118)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=119, nrhs=2)
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], recon, 1, 0, w.WILSON_OP_HOP, nrhs=2)
    for k in range(2):
        assert_parity(got[k], oracle_mod.dslash_eo(U, src[k], dims, 0, CPLX_PHASES), TOL[prec])
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], recon, 1, 1, w.WILSON_OP_SCHUR_DAG, 0.1350,
                     nrhs=2)
    for k in range(2):
        assert_parity(got[k], oracle_mod.schur(U, src[k], dims, 0.1350, 1, True, CPLX_PHASES), TOL[prec])
    psi = inputs.gaussian_spinor(dims, seed=120)
    got = handle_hop(w, U, psi, dims, CPLX_PHASES, w.PREC[prec], recon, w.WILSON_FULL, w.WILSON_FULL,
                     w.WILSON_OP_M, 0.1350)
    assert_parity(got, oracle_mod.wilson_m(U, psi, dims, 0.1350, CPLX_PHASES), TOL[prec])


@pytest.mark.parametrize("variant", [0, 3, 12, 14, 16, 21, 23, 25])
def test_variant_solver(w, oracle_mod, monkeypatch, variant):
    """The mixed-precision solve on each stencil family."""
    monkeypatch.setenv("WILSON_HOP_VARIANT", str(variant))
    dims = (4, 4, 4, 8)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=121)
    b = inputs.gaussian_spinor(dims, seed=122)
    x = dev(np.zeros_like(b))
    st = w.wilson_cg_solve(x, dev(U), dev(b), w.lattice(dims), 0.135, w.solver_defaults(w.WILSON_F16))
    r = b - oracle_mod.wilson_m(U, host(x), dims, 0.135)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.1e-10


# The t-slab streaming kernel (variant 26): tiles of a 3-d slice swept along
# t, the neighbouring input slices staged in shared memory by bulk copies, on
# lattices whose slices the tile divides: one and several tiles and t-chunks,
# Lt = 2 (the ring of slices wraps around the lattice), 64/128/256-site
# tiles.  No bounded wait may give up.
SLAB_CASES = [((8, 4, 4, 6), 64), ((8, 8, 4, 16), 64), ((4, 4, 8, 2), 64), ((16, 8, 8, 10), 128),
              ((16, 8, 8, 10), 256), ((8, 8, 8, 8), 256)]


@pytest.mark.parametrize("dims,block", SLAB_CASES)
@pytest.mark.parametrize("prec,recon", [("f32", 12), ("f16", 12), ("bf16", 12), ("f32", 18), ("f16", 18)])
def test_slab_variant(w, oracle_mod, monkeypatch, dims, block, prec, recon):
    monkeypatch.setenv("WILSON_HOP_VARIANT", "26")
    monkeypatch.setenv("WILSON_HOP_BLOCK", str(block))
    before = w.wilson_stage_timeouts()
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=131)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=132)
    for out_parity in (0, 1):
        got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], recon, 1 - out_parity, out_parity,
                         w.WILSON_OP_HOP)
        assert_parity(got, oracle_mod.dslash_eo(U, src, dims, out_parity, CPLX_PHASES), TOL[prec])
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], recon, 0, 0, w.WILSON_OP_SCHUR_DAG, 0.1350)
    assert_parity(got, oracle_mod.schur(U, src, dims, 0.1350, 0, True, CPLX_PHASES), TOL[prec])
    assert w.wilson_stage_timeouts() == before


def test_slab_solver(w, oracle_mod, monkeypatch):
    """The mixed-precision solve with its non-reducing hops on the t-slab kernel."""
    monkeypatch.setenv("WILSON_HOP_VARIANT", "26")
    monkeypatch.setenv("WILSON_HOP_BLOCK", "64")
    dims = (8, 4, 4, 8)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=133)
    b = inputs.gaussian_spinor(dims, seed=134)
    x = dev(np.zeros_like(b))
    w.wilson_cg_solve(x, dev(U), dev(b), w.lattice(dims), 0.135, w.solver_defaults(w.WILSON_F16))
    r = b - oracle_mod.wilson_m(U, host(x), dims, 0.135)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.1e-10


def test_slab_wait_gives_up(w, oracle_mod, monkeypatch):
    """Failure detection without a fault: with WILSON_TEST_STAGE_TIMEOUT=1 the
    staged slices are armed but never copied, so the kernel's bounded waits
    give up.  The kernel stores NaN at the sites it could not compute and
    returns, the library counts the timeouts, and the next launch on the same
    context computes the oracle's hop."""
    monkeypatch.setenv("WILSON_HOP_VARIANT", "26")
    monkeypatch.setenv("WILSON_HOP_BLOCK", "64")
    dims = (4, 4, 8, 2)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=135)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=136)
    before = w.wilson_stage_timeouts()
    monkeypatch.setenv("WILSON_TEST_STAGE_TIMEOUT", "1")
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.WILSON_F32, 12, 1, 0, w.WILSON_OP_HOP)
    assert np.isnan(got).any()
    assert w.wilson_stage_timeouts() > before
    monkeypatch.delenv("WILSON_TEST_STAGE_TIMEOUT")
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.WILSON_F32, 12, 1, 0, w.WILSON_OP_HOP)
    assert_parity(got, oracle_mod.dslash_eo(U, src, dims, 0, CPLX_PHASES), TOL["f32"])


# The register-blocked multi-RHS variants (NB = 2, 2, 3, 4 right-hand sides
# per thread; 18, 19: NB = 2 with the F16 packed projection; 27, 28: the F16
# pipeline with two right-hand sides per thread), the link-staged one (10:
# links in shared memory, a loop over the right-hand sides), pinned
# through WILSON_HOP_VARIANT, on 12 right-hand
# sides (a multiple of every NB) over a lattice with a ragged last block.
@pytest.mark.parametrize("variant", [6, 7, 8, 9, 10, 18, 19, 27, 28])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_blocked_multi_rhs_variants(w, oracle_mod, monkeypatch, variant, prec):
    monkeypatch.setenv("WILSON_HOP_VARIANT", str(variant))
    monkeypatch.setenv("WILSON_HOP_BLOCK", str((64, 128, 256)[variant % 3]))
    dims = (6, 4, 6, 10)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=123)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=124, nrhs=12)
    src[5] *= 1e-3  # right-hand sides of different magnitudes (F16 per-site scales)
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], 12, 1, 0, w.WILSON_OP_HOP, nrhs=12)
    for k in range(12):
        assert_parity(got[k], oracle_mod.dslash_eo(U, src[k], dims, 0, CPLX_PHASES), TOL[prec])
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], 12, 1, 1, w.WILSON_OP_SCHUR_DAG, 0.1350,
                     nrhs=12)
    for k in range(12):
        assert_parity(got[k], oracle_mod.schur(U, src[k], dims, 0.1350, 1, True, CPLX_PHASES), TOL[prec])
    psi = inputs.gaussian_spinor(dims, seed=125, nrhs=12)
    got = handle_hop(w, U, psi, dims, CPLX_PHASES, w.PREC[prec], 12, w.WILSON_FULL, w.WILSON_FULL,
                     w.WILSON_OP_M, 0.1350, nrhs=12)
    for k in range(12):
        assert_parity(got[k], oracle_mod.wilson_m(U, psi[k], dims, 0.1350, CPLX_PHASES), TOL[prec])


# The tensor-core multi-RHS kernel (variant 11: one warp per site, up to 16
# right-hand sides as the rows of mma.sync m16n8k16), pinned through
# WILSON_HOP_VARIANT: 2, 12 and 17 right-hand sides (17 = a full group of 16
# plus a group of one), right-hand sides of very different magnitudes, a
# ragged last warp tile (Vh = 720 = 22.5 tiles of 32 sites), complex boundary
# phases, and the three launch forms (even-odd hop, the Schur operator's
# xpay hop with the dagger projectors, the full-lattice M).
@pytest.mark.parametrize("nrhs", [2, 12, 17])
@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("block", [64, 256])
def test_tensor_core_multi_rhs_variant(w, oracle_mod, monkeypatch, nrhs, prec, block):
    monkeypatch.setenv("WILSON_HOP_VARIANT", "11")
    monkeypatch.setenv("WILSON_HOP_BLOCK", str(block))
    dims = (6, 4, 6, 10)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=128)
    src = inputs.gaussian_spinor(inputs.volume(dims) // 2, seed=129, nrhs=nrhs)
    src[nrhs - 1] *= 1e-3
    src[0] *= 40.0
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], 12, 1, 0, w.WILSON_OP_HOP, nrhs=nrhs)
    for k in range(nrhs):
        assert_parity(got[k], oracle_mod.dslash_eo(U, src[k], dims, 0, CPLX_PHASES), TOL[prec], f"rhs {k}")
    got = handle_hop(w, U, src, dims, CPLX_PHASES, w.PREC[prec], 12, 1, 1, w.WILSON_OP_SCHUR_DAG, 0.1350,
                     nrhs=nrhs)
    for k in range(nrhs):
        assert_parity(got[k], oracle_mod.schur(U, src[k], dims, 0.1350, 1, True, CPLX_PHASES), TOL[prec],
                      f"rhs {k}")
    psi = inputs.gaussian_spinor(dims, seed=130, nrhs=nrhs)
    got = handle_hop(w, U, psi, dims, CPLX_PHASES, w.PREC[prec], 12, w.WILSON_FULL, w.WILSON_FULL,
                     w.WILSON_OP_M, 0.1350, nrhs=nrhs)
    for k in range(nrhs):
        assert_parity(got[k], oracle_mod.wilson_m(U, psi[k], dims, 0.1350, CPLX_PHASES), TOL[prec], f"rhs {k}")


@pytest.mark.parametrize("variant", [6, 8, 9, 10, 11, 18, 27])
def test_blocked_variant_lockstep_solve(w, oracle_mod, monkeypatch, variant):
    """The lockstep multi-RHS solve on a blocked kernel: right-hand sides that
    finish early (a zero source at once) are skipped inside their group while
    the others go on, and every per-RHS reduction stays separate."""
    monkeypatch.setenv("WILSON_HOP_VARIANT", str(variant))
    dims = (4, 4, 4, 8)
    kappa = 0.1350
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=126)
    b = inputs.gaussian_spinor(dims, seed=127, nrhs=12)
    b[2] = 0
    b[7] *= 1e-6
    b[10] = inputs.point_sources(dims, site=3)[4]
    x = dev(np.zeros_like(b))
    rc, st = w.wilson_cg_solve_multi(x, dev(U), dev(b), 12, w.lattice(dims), kappa,
                                     w.solver_defaults(w.WILSON_F16))
    xs = host(x)
    assert rc == 0 and np.all(xs[2] == 0)
    for k in range(12):
        if k == 2:
            continue
        r = b[k] - oracle_mod.wilson_m(U, xs[k], dims, kappa)
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.1e-10


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_import_export_host_memory(w, oracle_mod, prec):
    """Spinor import and export through device memory, page-locked host
    memory (asynchronous copies on the library's copy streams) and pageable
    host memory (staged, synchronous) give the same fields: bit-exact for
    FP64 handles, and the same hop result whichever way the field came in."""
    import torch
    dims = (6, 4, 6, 10)
    Vh = inputs.volume(dims) // 2
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=132)
    src = inputs.gaussian_spinor(Vh, seed=133, nrhs=2)
    L = w.lattice(dims, CPLX_PHASES)
    g = w.Gauge(U, L, w.PREC[prec], 18 if prec == "f64" else 12)
    sources = {"device": dev(src), "pinned": torch.from_numpy(src.copy()).pin_memory(),
               "pageable": np.ascontiguousarray(src)}
    outs = {}
    for name, s_in in sources.items():
        a = w.Spinor(L, w.WILSON_ODD, w.PREC[prec], 2)
        b = w.Spinor(L, w.WILSON_EVEN, w.PREC[prec], 2)
        a.load(s_in)
        w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP)
        back = {"device": empty_like_dev(src), "pinned": torch.empty(src.shape, dtype=torch.complex128).pin_memory(),
                "pageable": np.full_like(src, np.nan)}[name]
        a.store(back)
        res = np.full_like(src, np.nan)
        b.store(res)
        torch.cuda.synchronize()  # exports to page-locked memory are asynchronous on the stream
        back = host(back) if name == "device" else (back.numpy() if name == "pinned" else back)
        if prec == "f64":
            assert np.array_equal(back, src), name
        else:
            assert_parity(back, src, TOL[prec], name)
        outs[name] = res
        a.close(); b.close()
    g.close()
    for name in ("pinned", "pageable"):
        assert np.array_equal(outs[name], outs["device"]), name
    for k in range(2):
        assert_parity(outs["device"][k], oracle_mod.dslash_eo(U, src[k], dims, 0, CPLX_PHASES), TOL[prec])
