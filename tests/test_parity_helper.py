"""The element bound of the parity helper catches an error confined to one
site, which the global relative L2 norm lets through on a large output."""
import numpy as np
import pytest

from conftest import assert_parity, rel_l2


def test_single_site_error_caught():
    rng = np.random.default_rng(3)
    want = rng.standard_normal((65536, 4, 3)) + 1j * rng.standard_normal((65536, 4, 3))
    got = want.copy()
    rms = np.sqrt(np.mean(np.abs(want) ** 2))
    got[40000, 2, 1] += 0.3 * rms  # one component of one site off by 0.3 RMS
    assert rel_l2(got, want) < 5e-3  # invisible to the norm at the F16 tolerance
    with pytest.raises(AssertionError, match="largest component"):
        assert_parity(got, want, 5e-3)


def test_storage_rounding_accepted():
    rng = np.random.default_rng(4)
    want = rng.standard_normal((4096, 4, 3)) + 1j * rng.standard_normal((4096, 4, 3))
    got = want.astype(np.complex64).astype(np.complex128)
    assert_parity(got, want, 1e-6)
    with pytest.raises(AssertionError, match="rel L2"):
        assert_parity(got * 1.001, want, 1e-6)
