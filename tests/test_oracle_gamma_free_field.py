"""Pins of the oracle's gamma table and of the hopping term on a free field.

* The gamma table must be the DeGrand-Rossi basis (golden fixture from the
  literature) and satisfy the Euclidean Clifford algebra.
* Free field (all links = 1): a plane wave psi_x = exp(i p.x) u with
  p_mu = (2 pi n_mu + theta_mu) / L_mu (theta_mu the boundary twist) is an
  eigenvector of the hopping term with
      D_h psi = sum_mu (2 cos p_mu - 2 i c gamma_mu sin p_mu) psi
  (c = +1 for the "(1-gamma) forward" convention, c = -1 for Eq. 3 as
  printed).  The 12x12 matrix of D_h on the 12 plane waves of one momentum
  has eigenvalues 2 sum cos p_mu +- 2 i sqrt(sum sin^2 p_mu), each 6-fold;
  that statement does not depend on the gamma basis.
"""
import os

import numpy as np
import pytest

from conftest import rel_l2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "degrand_rossi_gamma.txt")


def load_dr_table():
    g = np.zeros((5, 4, 4), dtype=np.complex128)
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, vals = line.split(":")
            name, row = head.split()
            mu = int(name[1:]) - 1
            g[mu, int(row)] = [complex(v) for v in vals.split()]
    return g


def test_gamma_table_is_degrand_rossi(oracle_mod):
    dr = load_dr_table()
    for mu in range(5):
        assert np.array_equal(oracle_mod.gamma(mu), dr[mu]), f"gamma_{mu + 1} differs from the DeGrand-Rossi table"


def test_clifford_algebra(oracle_mod):
    g = [oracle_mod.gamma(mu) for mu in range(5)]
    eye = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2 * eye * (mu == nu), atol=0)
        assert np.allclose(g[4] @ g[mu] + g[mu] @ g[4], 0, atol=0)
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]), atol=0)


def plane_wave(dims, p, u):
    from paper_0710_2442_gb300.inputs import site_coords
    c = site_coords(dims)
    phase = np.exp(1j * (c @ np.asarray(p)))
    return phase[:, None, None] * u[None, :, :]


def unit_gauge(dims):
    from paper_0710_2442_gb300.inputs import gauge_field
    return gauge_field(dims, kind="unit")


CASES = [
    ((8, 8, 8, 8), (1, 1, 1, -1)),
    ((2, 2, 2, 2), (1, 1, 1, -1)),
    ((4, 6, 2, 8), (np.exp(0.3j), np.exp(-1.1j), 1, -1)),
    ((6, 4, 4, 10), (np.exp(2.0j), 1j, np.exp(0.7j), np.exp(-2.9j))),
]


@pytest.mark.parametrize("dims,phases", CASES)
@pytest.mark.parametrize("conv", [1, -1])
def test_free_field_plane_wave_pointwise(oracle_mod, dims, phases, conv):
    rng = np.random.default_rng(7)
    U = unit_gauge(dims)
    g = load_dr_table()  # the basis both sides use, from the literature
    theta = np.angle(np.asarray(phases, dtype=np.complex128))
    for trial in range(3):
        n = np.array([rng.integers(0, L) for L in dims])
        p = (2 * np.pi * n + theta) / np.asarray(dims)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = plane_wave(dims, p, u)
        got = oracle_mod.dslash(U, psi, dims, phases, conv=conv)
        K = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * conv * np.sin(p[m]) * g[m] for m in range(4))
        want = plane_wave(dims, p, K @ u)
        assert rel_l2(got, want) < 1e-13


@pytest.mark.parametrize("dims,phases", CASES)
def test_free_field_spectrum_basis_independent(oracle_mod, dims, phases):
    rng = np.random.default_rng(11)
    U = unit_gauge(dims)
    theta = np.angle(np.asarray(phases, dtype=np.complex128))
    V = int(np.prod(dims))
    for trial in range(4):
        n = np.array([rng.integers(0, L) for L in dims])
        p = (2 * np.pi * n + theta) / np.asarray(dims)
        cols = []
        for k in range(12):
            u = np.zeros((4, 3), dtype=np.complex128)
            u[k // 3, k % 3] = 1
            psi = plane_wave(dims, p, u)
            out = oracle_mod.dslash(U, psi, dims, phases)
            # project back onto the 12 plane waves of momentum p
            cols.append((np.conj(plane_wave(dims, p, np.ones((4, 3)))) * out).sum(axis=0).ravel() / V)
        K = np.array(cols).T
        ev = np.linalg.eigvals(K)
        c = 2 * np.cos(p).sum()
        s = 2 * np.sqrt((np.sin(p) ** 2).sum())
        ev = ev[np.argsort(ev.imag, kind="stable")]
        want = np.array([c - 1j * s] * 6 + [c + 1j * s] * 6)
        assert np.allclose(ev, want, atol=1e-12), (ev, want)


def test_wilson_m_free_field_eigenvalues(oracle_mod):
    """Eigenvalues of M = 1 - kappa D_h on a plane wave: 1 - 2 kappa sum cos
    p -+ 2 i kappa sqrt(sum sin^2 p)."""
    dims = (4, 4, 4, 6)
    phases = (1, 1, 1, -1)
    U = unit_gauge(dims)
    kappa = 0.13
    theta = np.angle(np.asarray(phases, dtype=np.complex128))
    p = (2 * np.pi * np.array([1, 2, 3, 1]) + theta) / np.asarray(dims)
    g = load_dr_table()
    u = np.arange(12).reshape(4, 3) + 1j
    psi = plane_wave(dims, p, u)
    got = oracle_mod.wilson_m(U, psi, dims, kappa, phases)
    K = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * g[m] for m in range(4))
    want = plane_wave(dims, p, (np.eye(4) - kappa * K) @ u)
    assert rel_l2(got, want) < 1e-14
