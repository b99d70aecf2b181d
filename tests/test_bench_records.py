"""The bench's parity record: relative L2 and largest-component error of the
library's first hop application against the oracle's output."""
import numpy as np

import bench


def test_parity_record_values():
    rng = np.random.default_rng(7)
    want = rng.standard_normal((512, 4, 3)) + 1j * rng.standard_normal((512, 4, 3))
    rec = bench.parity_record("f32", want.copy(), want)
    assert rec["rel_l2"] == 0.0 and rec["max_component_error_over_rms"] == 0.0
    assert rec["tolerance_rel_l2"] == 1e-6 and rec["sites"] == 512
    got = want.copy()
    rms = np.sqrt(np.mean(np.abs(want) ** 2))
    got[3, 1, 2] += 0.5 * rms  # one real component off by half the RMS modulus
    rec = bench.parity_record("f16", got, want)
    assert abs(rec["max_component_error_over_rms"] - 0.5) < 1e-12
    assert abs(rec["rel_l2"] - 0.5 * rms / np.linalg.norm(want)) < 1e-12
    assert rec["tolerance_rel_l2"] == 5e-3


def test_oracle_solution_check_record(oracle_mod):
    """The CPU leg's check of solver results: an oracle CG solution on a 4^4
    lattice has a true residual below its tolerance, and a planted error in
    the solution is reported."""
    from paper_0710_2442_gb300 import inputs
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=11)
    b = inputs.gaussian_spinor(dims, seed=12)
    x, _ = oracle_mod.cg_solve(U, b, dims, 0.12, tol=1e-10)
    good, bad = {}, {}
    bench.SOLUTIONS.append((good, "oracle", [(U, b, x, dims, 0.12)], x))
    xb = x.copy()
    xb[5, 1, 2] += 1e-3 * np.linalg.norm(x)
    bench.SOLUTIONS.append((bad, "oracle", [(lambda: U, lambda: b, xb, dims, 0.12)]))
    bench.oracle_solution_checks()
    assert not bench.SOLUTIONS
    assert good["oracle"]["true_rel_resid_max"] <= 1e-10
    assert good["oracle"]["rel_diff_vs_fp64_gpu_solution"] == 0.0
    assert bad["oracle"]["true_rel_resid_max"] > 1e-4


def test_access_pattern_record_arithmetic():
    """The access-pattern record: T_mem is the compulsory bytes at the copy
    bandwidth, and the two ratios compare the probe with T_mem and the hop
    with the probe (the headline's figures: 604 MB, 6791.7 GB/s)."""
    byts = 576 * 1048576
    rec = bench.access_record(byts, 88.0e-6, 89.9e-6, 6791.7)
    assert abs(rec["t_mem_us"] - byts / 6791.7e9 * 1e6) < 0.01
    assert abs(rec["access_over_t_mem"] - 88.0 / rec["t_mem_us"]) < 2e-3
    assert abs(rec["hop_over_access"] - 89.9 / 88.0) < 1e-3
    assert abs(rec["frac"] - byts / 88.0e-6 / 1e9 / 6791.7) < 1e-4
    assert rec["us"] == 88.0 and rec["hop_us"] == 89.9
