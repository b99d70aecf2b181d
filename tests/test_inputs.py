"""The seeded generators produce what their recipes promise."""
import numpy as np

from paper_0710_2442_gb300 import inputs


def test_random_su3_unitary_det_one():
    U = inputs.random_su3(np.random.default_rng(0), 2000)
    eye = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.transpose(U, (0, 2, 1))) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-14


def test_weak_field_su3_close_to_one():
    for eps in (0.2, 0.3, 0.4):
        U = inputs.weak_field_su3(np.random.default_rng(1), 5000, eps)
        assert np.max(np.abs(U @ np.conj(np.transpose(U, (0, 2, 1))) - np.eye(3))) < 1e-14
        assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-14
        # <Re tr U / 3> ~ 1 - eps^2 <tr H^2> / 6 with <tr H^2> = 4 (h_a ~ N(0,1), tr(l_a l_b)/4 = d_ab/2)
        u0 = np.mean(np.trace(U, axis1=1, axis2=2).real) / 3
        assert abs(u0 - (1 - eps ** 2 * 4 / 6)) < 0.05 * eps ** 2


def test_generators_deterministic():
    a = inputs.gauge_field((2, 2, 2, 2), "weak", eps=0.3, seed=5)
    b = inputs.gauge_field((2, 2, 2, 2), "weak", eps=0.3, seed=5)
    assert np.array_equal(a, b)
    assert np.array_equal(inputs.gaussian_spinor(16, seed=3), inputs.gaussian_spinor(16, seed=3))


def test_batch_mix():
    probs = inputs.batch_problems()
    assert len(probs) == 64
    sites = sum(inputs.volume(p["dims"]) for p in probs)
    assert sites == 4689920
    for p in probs:
        assert 0.2 <= p["eps"] <= 0.4 and 0.125 <= p["kappa"] <= 0.1355
