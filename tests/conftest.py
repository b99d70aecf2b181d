import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests need a device: skip them cleanly where there is none.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


# ---------------------------------------------------------------------------
# test-side helpers (layout bookkeeping only)
# ---------------------------------------------------------------------------
def parity_split(field: np.ndarray, dims):
    """Full canonical field -> (even half, odd half), half index s >> 1."""
    from paper_0710_2442_gb300.inputs import site_parity
    par = site_parity(dims)
    V = par.size
    idx = np.arange(V)
    halves = []
    for p in (0, 1):
        h = np.zeros((V // 2,) + field.shape[1:], dtype=field.dtype)
        sel = par == p
        h[idx[sel] >> 1] = field[sel]
        halves.append(h)
    return halves[0], halves[1]


def parity_merge(even: np.ndarray, odd: np.ndarray, dims):
    from paper_0710_2442_gb300.inputs import site_parity
    par = site_parity(dims)
    V = par.size
    idx = np.arange(V)
    out = np.zeros((V,) + even.shape[1:], dtype=even.dtype)
    out[par == 0] = even[idx[par == 0] >> 1]
    out[par == 1] = odd[idx[par == 1] >> 1]
    return out


def rel_l2(a, b) -> float:
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
