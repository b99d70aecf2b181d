"""The batched solve of many uneven lattices in one graph launch, checked
problem by problem against the FP64 oracle's Wilson matrix (true residual
<= 1e-10) and against single solves of the same problems."""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_helpers import dev, host
from paper_0710_2442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


MIX = [((4, 4, 4, 4), 0.2, 0.125), ((4, 4, 4, 8), 0.3, 0.1350), ((6, 4, 6, 10), 0.4, 0.13),
       ((2, 2, 2, 4), 0.3, 0.128), ((8, 8, 8, 8), 0.25, 0.1355), ((4, 6, 4, 6), 0.35, 0.131)]


def make_batch(w, mix, seed0=400, phases=None):
    probs, host_fields = [], []
    for i, (dims, eps, kappa) in enumerate(mix):
        U = inputs.gauge_field(dims, "weak", eps=eps, seed=seed0 + 2 * i)
        b = inputs.gaussian_spinor(dims, seed=seed0 + 2 * i + 1)
        L = w.lattice(dims, phases if phases is not None else inputs.DEFAULT_PHASES)
        probs.append(dict(L=L, kappa=kappa, gauge=dev(U), b=dev(b), x=dev(np.zeros_like(b))))
        host_fields.append((dims, U, b, kappa))
    return probs, host_fields


def true_resid(oracle_mod, U, x, b, dims, kappa, phases=None):
    return np.linalg.norm(b - oracle_mod.wilson_m(U, x, dims, kappa, phases)) / np.linalg.norm(b)


# WILSON_BATCH_SMALL_VH: problems with at most this many sites per parity run
# the CTA-resident solver; 0 sends every problem through the device loop,
# 400 splits MIX between the two paths, 4096 puts all of MIX on CTAs.
@pytest.mark.parametrize("small_vh", ["0", "400", "4096"])
@pytest.mark.parametrize("inner", ["f16", "bf16", "f32"])
def test_batch_matches_oracle(w, oracle_mod, monkeypatch, inner, small_vh):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", small_vh)
    probs, hf = make_batch(w, MIX)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.PREC[inner]))
    assert rc == 0 and not info["timed_out"]
    assert info["graph_launches"] >= 1
    assert (info["tiles"] > 0) == (small_vh != "4096")  # all of MIX fits the CTA path at 4096
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        x = host(q["x"])
        assert s["status"] == 0 and s["true_rel_resid"] <= 1e-10
        assert true_resid(oracle_mod, U, x, b, dims, kappa) <= 1.1e-10
        assert 0 <= s["seconds"] <= info["device_seconds"] + 1e-6


# WILSON_BATCH_HOP pins the inner hop of the device loop: the pipelined
# F16 / BF16 stencil (variant 22, 64- and 128-thread blocks, 256-site tiles
# walked by 4 or 2 sites per thread) and the paired stencil, on MIX through
# the loop.
@pytest.mark.parametrize("hop,inner", [("22:64", "f16"), ("22:128", "f16"), ("4:128", "f16"), ("22:64", "bf16")])
def test_batch_inner_hop_variants(w, oracle_mod, monkeypatch, hop, inner):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "0")
    monkeypatch.setenv("WILSON_BATCH_HOP", hop)
    probs, hf = make_batch(w, MIX)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.PREC[inner]))
    assert rc == 0 and not info["timed_out"] and info["tiles"] > 0
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert s["status"] == 0
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10


# WILSON_BATCH_TILE pins the tile size of every class (the autotuner's
# candidates): 128, 256 and 512 sites, on MIX (half volumes 32 to 512 sites:
# single, partial and many tiles per problem) through the device loop.
@pytest.mark.parametrize("tile", ["128", "256", "512"])
def test_batch_tile_sizes(w, oracle_mod, monkeypatch, tile):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "0")
    monkeypatch.setenv("WILSON_BATCH_TILE", tile)
    probs, hf = make_batch(w, MIX, seed0=440)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    assert rc == 0 and not info["timed_out"]
    want_tiles = sum(-(-inputs.volume(dims) // 2 // int(tile)) for dims, _, _, _ in hf)
    assert info["tiles"] == want_tiles
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert s["status"] == 0
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10


@pytest.mark.parametrize("small_vh", ["0", "4096"])
def test_batch_initial_guess(w, oracle_mod, monkeypatch, small_vh):
    """use_initial_guess: every problem starts from a nonzero iterate (its
    first FP64 correction applies the operator to it) and still reaches the
    1e-10 true residual; the problems without the flag start from zero."""
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", small_vh)
    probs, hf = make_batch(w, MIX, seed0=460)
    for i, (q, (dims, _, b, _)) in enumerate(zip(probs, hf)):
        q["x"] = dev(0.3 * inputs.gaussian_spinor(dims, seed=480 + i))
    p = w.solver_defaults(w.WILSON_F16)
    p.use_initial_guess = 1
    rc, st, info = w.wilson_batch_solve(probs, p)
    assert rc == 0 and not info["timed_out"]
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert s["status"] == 0
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10


@pytest.mark.parametrize("small_vh", ["0", "4096"])
def test_batch_equals_single_solves(w, monkeypatch, small_vh):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", small_vh)
    probs, hf = make_batch(w, MIX[:4], seed0=420)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    for q, (dims, U, b, kappa) in zip(probs, hf):
        xs = dev(np.zeros_like(b))
        w.wilson_cg_solve(xs, dev(U), dev(b), w.lattice(dims), kappa, w.solver_defaults(w.WILSON_F16))
        # both reach 1e-10; the solutions agree to the conditioning of M times that
        assert rel_l2(host(q["x"]), host(xs)) <= 1e-7


@pytest.mark.parametrize("small_vh", ["0", "400"])
def test_batch_complex_phases(w, oracle_mod, monkeypatch, small_vh):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", small_vh)
    ph = (np.exp(0.3j), 1.0, np.exp(-1.2j), -1.0)
    probs, hf = make_batch(w, MIX[:3], seed0=440, phases=ph)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    for q, (dims, U, b, kappa) in zip(probs, hf):
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa, ph) <= 1.1e-10


@pytest.mark.parametrize("small_vh", ["0", "4096"])
def test_batch_noconv_and_numeric_are_per_problem(w, oracle_mod, monkeypatch, small_vh):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", small_vh)
    probs, hf = make_batch(w, MIX[:3], seed0=460)
    bad = host(probs[1]["b"])
    bad[3, 2, 1] = np.nan
    probs[1]["b"] = dev(bad)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16), check=False)
    assert rc == w.WILSON_ERR_NUMERIC
    assert st[1]["status"] == w.WILSON_ERR_NUMERIC
    for k in (0, 2):
        dims, U, b, kappa = hf[k]
        assert st[k]["status"] == 0
        assert true_resid(oracle_mod, U, host(probs[k]["x"]), b, dims, kappa) <= 1.1e-10
    p = w.solver_defaults(w.WILSON_F16)
    p.maxiter = 4
    probs, hf = make_batch(w, MIX[:2], seed0=470)
    rc, st, info = w.wilson_batch_solve(probs, p, check=False)
    assert rc == w.WILSON_ERR_NOCONV and all(s["status"] == w.WILSON_ERR_NOCONV for s in st)


# WILSON_BATCH_CLASSES caps the number of device loops (one per class of
# lattice sizes); WILSON_BATCH_HOST_LOOP=1 replaces the device-side loop by
# host-replayed graphs of eight iterations.
@pytest.mark.parametrize("classes,host_loop", [("1", "0"), ("2", "0"), ("8", "0"), ("8", "1")])
def test_batch_classes_and_host_loop(w, oracle_mod, monkeypatch, classes, host_loop):
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "0")
    monkeypatch.setenv("WILSON_BATCH_CLASSES", classes)
    monkeypatch.setenv("WILSON_BATCH_HOST_LOOP", host_loop)
    probs, hf = make_batch(w, MIX, seed0=500)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    assert rc == 0 and not info["timed_out"]
    assert info["device_loop"] == (host_loop == "0")
    if host_loop == "0":
        assert info["graph_launches"] == 1
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert s["status"] == 0
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10


def test_loop_limit_runs_out_and_context_stays_usable(w, oracle_mod, monkeypatch):
    """The device-side loop has a hard iteration cap; when it runs out the
    unfinished problems report WILSON_ERR_TIMEOUT and the next call works."""
    probs, hf = make_batch(w, MIX[:3], seed0=480)
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "0")  # the loop cap governs the loop path
    monkeypatch.setenv("WILSON_BATCH_MAX_LOOP", "6")
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16), check=False)
    assert info["timed_out"] == 1 and info["iterations"] == 6
    assert rc == w.WILSON_ERR_TIMEOUT
    assert all(s["status"] == w.WILSON_ERR_TIMEOUT for s in st)
    monkeypatch.delenv("WILSON_BATCH_MAX_LOOP")
    for q in probs:
        q["x"].zero_()
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    assert rc == 0 and info["timed_out"] == 0
    for q, (dims, U, b, kappa) in zip(probs, hf):
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10


def test_small_path_budget_runs_out(w, monkeypatch):
    """The CTA-resident solver checks the wall-clock budget too."""
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "4096")
    monkeypatch.setenv("WILSON_BATCH_BUDGET_MS", "1")
    probs, hf = make_batch(w, [((8, 8, 8, 8), 0.3, 0.1355)] * 2, seed0=490)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16), check=False)
    assert rc in (w.WILSON_ERR_TIMEOUT, w.WILSON_OK)
    assert all(s["status"] in (w.WILSON_ERR_TIMEOUT, w.WILSON_OK) for s in st)


@pytest.mark.parametrize("small_vh", ["0", "4096"])
def test_batch_single_and_degenerate_problems(w, oracle_mod, monkeypatch, small_vh):
    """A batch of one problem, and a batch holding a kappa = 0 problem (M = 1,
    x = b) and a zero source (x stays 0) beside a regular one, on the loop
    path and on the CTA-resident path."""
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", small_vh)
    probs, hf = make_batch(w, [((4, 4, 4, 8), 0.3, 0.13)], seed0=510)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    dims, U, b, kappa = hf[0]
    assert rc == 0 and true_resid(oracle_mod, U, host(probs[0]["x"]), b, dims, kappa) <= 1.1e-10
    probs, hf = make_batch(w, [((4, 4, 4, 4), 0.3, 0.0), ((6, 4, 6, 10), 0.3, 0.13), ((4, 4, 4, 8), 0.3, 0.125)],
                           seed0=520)
    probs[2]["b"].zero_()
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.WILSON_F16))
    assert rc == 0 and all(s["status"] == 0 for s in st)
    assert rel_l2(host(probs[0]["x"]), hf[0][2]) <= 1e-10
    dims, U, b, kappa = hf[1]
    assert true_resid(oracle_mod, U, host(probs[1]["x"]), b, dims, kappa) <= 1.1e-10
    assert np.all(host(probs[2]["x"]) == 0)


@pytest.mark.parametrize("cluster", ["1", "4"])
@pytest.mark.parametrize("inner", ["f16", "f32"])
def test_small_path_block_and_cluster(w, oracle_mod, monkeypatch, cluster, inner):
    """The CTA-resident solves on one thread block per problem and on a
    cluster of four blocks (cluster barriers, sums through distributed shared
    memory) both reach the target against the oracle."""
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "4096")
    monkeypatch.setenv("WILSON_BATCH_SMALL_CLUSTER", cluster)
    probs, hf = make_batch(w, MIX, seed0=530)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.PREC[inner]))
    assert rc == 0 and info["tiles"] == 0
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert s["status"] == 0
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10


@pytest.mark.parametrize("inner", ["f16", "bf16"])
def test_batch_fp32_outer_residuals(w, oracle_mod, monkeypatch, inner):
    """The early corrections of the device-loop problems compute their
    residual with FP32 fields and links; every problem still reaches the
    1e-10 true residual by the oracle's FP64 M.  A target of 1e-6 uses only
    FP64 residuals."""
    monkeypatch.setenv("WILSON_BATCH_SMALL_VH", "0")
    probs, hf = make_batch(w, MIX, seed0=500)
    rc, st, info = w.wilson_batch_solve(probs, w.solver_defaults(w.PREC[inner]))
    assert rc == 0 and not info["timed_out"]
    assert all(s["outer_f32"] >= 1 and s["outer_f32"] < s["outer_iters"] for s in st)
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-10
    probs, hf = make_batch(w, MIX, seed0=500)
    p = w.solver_defaults(w.PREC[inner])
    p.tol = 1e-6
    rc, st, info = w.wilson_batch_solve(probs, p)
    assert rc == 0 and all(s["outer_f32"] == 0 for s in st)
    for q, (dims, U, b, kappa), s in zip(probs, hf, st):
        assert true_resid(oracle_mod, U, host(q["x"]), b, dims, kappa) <= 1.1e-6
