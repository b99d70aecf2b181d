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


def assert_parity(got, want, tol, msg="", elem=10.0):
    """Parity of an operator output with the oracle's.

    Two bounds: the relative L2 error over the whole output is at most tol,
    and every real and imaginary component differs by at most elem * tol
    times the RMS modulus of the oracle's output.  The second catches
    errors confined to a few sites, which the global norm dilutes on large
    lattices (one wrong site of 10^6 moves it by 1e-3).  Reduced-precision
    storage alone (per-site scaled halves, IEEE F16 or BF16, inputs, links
    and output) gives a largest component error of 1.3e-3 (F16) and 1.0e-2
    (BF16) of the RMS on lattices up to 16^4, against a bound of 5e-2;
    a dropped or sign-flipped neighbour term moves a component by about
    0.3 of the RMS.
    """
    g = np.asarray(got).ravel()
    w = np.asarray(want).ravel()
    r = rel_l2(g, w)
    assert r <= tol, f"{msg} rel L2 {r:.3e} > {tol:.1e}"
    rms = float(np.sqrt(np.mean(np.abs(w) ** 2))) if w.size else 0.0
    d = g - w
    worst = float(np.max(np.maximum(np.abs(d.real), np.abs(d.imag)))) if d.size else 0.0
    bound = elem * tol * (rms if rms > 0 else 1.0)
    assert worst <= bound, f"{msg} largest component error {worst:.3e} > {bound:.3e}"


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
