"""Pins of the oracle by identities of the Wilson hopping term (Eq. 3).

* gamma_5-hermiticity: <x, D y> = <gamma_5 D gamma_5 x, y> on random SU(3)
  links with complex boundary phases (catches a missing conjugation, a wrong
  link on the backward hop, or a backward phase that is not conjugated);
* gauge covariance: U'_{x,mu} = W_x U_{x,mu} W^dag_{x+mu}, psi' = W psi
  gives D[U'] psi' = W D[U] psi (catches a transposed or misplaced link);
* the convention identity: Eq. 3 as printed equals gamma_5 D gamma_5 of the
  "(1-gamma) forward" form;
* linearity and M = 1 - kappa D_h;
* even-odd blocks: the checkerboarded hop equals the full hop on a field
  embedded by the test's own parity split.
"""
import numpy as np
import pytest

from conftest import parity_merge, parity_split, rel_l2
from paper_0710_2442_gb300 import inputs

DIMS = [(4, 4, 4, 4), (2, 2, 2, 2), (4, 2, 6, 8), (6, 4, 2, 4)]
PHASES = (np.exp(0.4j), 1.0, np.exp(-2.2j), -1.0)


def g5(psi, oracle_mod):
    return np.einsum("ab,sbc->sac", oracle_mod.gamma(4), psi)


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


@pytest.mark.parametrize("dims", DIMS)
def test_gamma5_hermiticity(oracle_mod, dims):
    U = inputs.gauge_field(dims, "random", seed=1)
    x = inputs.gaussian_spinor(dims, seed=2)
    y = inputs.gaussian_spinor(dims, seed=3)
    lhs = vdot(x, oracle_mod.dslash(U, y, dims, PHASES))
    rhs = vdot(g5(oracle_mod.dslash(U, g5(x, oracle_mod), dims, PHASES), oracle_mod), y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("dims", DIMS)
def test_gauge_covariance(oracle_mod, dims):
    V = inputs.volume(dims)
    U = inputs.gauge_field(dims, "random", seed=4)
    psi = inputs.gaussian_spinor(dims, seed=5)
    W = inputs.random_gauge_transform(np.random.default_rng(6), V)
    coords = inputs.site_coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        c = coords.copy()
        c[:, mu] = (c[:, mu] + 1) % dims[mu]
        fwd = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * (c[:, 2] + dims[2] * c[:, 3]))
        Up[:, mu] = W @ U[:, mu] @ np.conj(np.transpose(W[fwd], (0, 2, 1)))
    psip = np.einsum("sij,saj->sai", W, psi)
    lhs = oracle_mod.dslash(Up, psip, dims, PHASES)
    rhs = np.einsum("sij,saj->sai", W, oracle_mod.dslash(U, psi, dims, PHASES))
    assert rel_l2(lhs, rhs) < 1e-13


@pytest.mark.parametrize("dims", DIMS[:2])
def test_convention_identity(oracle_mod, dims):
    U = inputs.gauge_field(dims, "random", seed=8)
    psi = inputs.gaussian_spinor(dims, seed=9)
    printed = oracle_mod.dslash(U, psi, dims, PHASES, conv=-1)
    ours = g5(oracle_mod.dslash(U, g5(psi, oracle_mod), dims, PHASES, conv=1), oracle_mod)
    assert rel_l2(printed, ours) < 1e-14
    # and the two conventions really differ
    assert rel_l2(printed, oracle_mod.dslash(U, psi, dims, PHASES, conv=1)) > 0.1


def test_linearity_and_wilson_m(oracle_mod):
    dims = (4, 4, 2, 6)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=10)
    a = inputs.gaussian_spinor(dims, seed=11)
    b = inputs.gaussian_spinor(dims, seed=12)
    ca, cb = 0.7 - 1.3j, -2.1 + 0.2j
    lhs = oracle_mod.dslash(U, ca * a + cb * b, dims, PHASES)
    rhs = ca * oracle_mod.dslash(U, a, dims, PHASES) + cb * oracle_mod.dslash(U, b, dims, PHASES)
    assert rel_l2(lhs, rhs) < 1e-14
    kappa = 0.1350
    m = oracle_mod.wilson_m(U, a, dims, kappa, PHASES)
    assert rel_l2(m, a - kappa * oracle_mod.dslash(U, a, dims, PHASES)) < 1e-15


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (4, 6, 2, 8)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_eo_blocks_equal_restricted_full_hop(oracle_mod, dims, out_parity):
    U = inputs.gauge_field(dims, "random", seed=13)
    psi = inputs.gaussian_spinor(dims, seed=14)
    e, o = parity_split(psi, dims)
    src = o if out_parity == 0 else e
    zero = np.zeros_like(src)
    full_in = parity_merge(zero, src, dims) if out_parity == 0 else parity_merge(src, zero, dims)
    full_out = oracle_mod.dslash(U, full_in, dims, PHASES)
    want = parity_split(full_out, dims)[out_parity]
    got = oracle_mod.dslash_eo(U, src, dims, out_parity, PHASES)
    assert rel_l2(got, want) < 1e-15


def test_eo_gamma5_adjoint_blocks(oracle_mod):
    """D_eo^dag = gamma_5 D_oe gamma_5."""
    dims = (4, 2, 4, 6)
    U = inputs.gauge_field(dims, "random", seed=15)
    Vh = inputs.volume(dims) // 2
    x = inputs.gaussian_spinor(Vh, seed=16)
    y = inputs.gaussian_spinor(Vh, seed=17)
    lhs = vdot(x, oracle_mod.dslash_eo(U, y, dims, 0, PHASES))             # <x_e, D_eo y_o>
    rhs = vdot(g5(oracle_mod.dslash_eo(U, g5(x, oracle_mod), dims, 1, PHASES), oracle_mod), y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_odd_extent_rejected_for_eo(oracle_mod):
    dims = (4, 4, 3, 4)
    U = inputs.gauge_field(dims, "unit")
    with pytest.raises(ValueError):
        oracle_mod.dslash_eo(U, np.zeros((inputs.volume(dims) // 2, 4, 3)), dims, 0)
