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
