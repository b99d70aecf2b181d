"""Brute-force pins on tiny lattices: the Wilson matrix assembled entry by
entry by an independent loop, the even-odd Schur complement by dense block
algebra, and the CG solve against a dense LU solve.

The dense matrix below is written from Eq. 3 (with the (1-gamma) forward
convention and M = 1 - kappa D_h) using the literature gamma table and the
test's own neighbour bookkeeping; it shares nothing with the oracle but the
input fields.
"""
import numpy as np
import pytest

from conftest import parity_merge, parity_split, rel_l2
from paper_0710_2442_gb300 import inputs
from test_oracle_gamma_free_field import load_dr_table

PHASES = (np.exp(0.9j), 1.0, -1.0, np.exp(-0.5j))


def dense_wilson(U, dims, kappa, phases):
    g = load_dr_table()
    V = inputs.volume(dims)
    N = 12 * V
    M = np.eye(N, dtype=np.complex128)
    I4 = np.eye(4)
    Lx, Ly, Lz, Lt = dims
    for t in range(Lt):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    c = [x, y, z, t]
                    s = x + Lx * (y + Ly * (z + Lz * t))
                    for mu in range(4):
                        cf = list(c)
                        cb = list(c)
                        cf[mu] = (c[mu] + 1) % dims[mu]
                        cb[mu] = (c[mu] - 1) % dims[mu]
                        sf = cf[0] + Lx * (cf[1] + Ly * (cf[2] + Lz * cf[3]))
                        sb = cb[0] + Lx * (cb[1] + Ly * (cb[2] + Lz * cb[3]))
                        ef = phases[mu] if c[mu] == dims[mu] - 1 else 1.0
                        eb = np.conj(phases[mu]) if c[mu] == 0 else 1.0
                        fwd = ef * np.kron(I4 - g[mu], U[s, mu])
                        bwd = eb * np.kron(I4 + g[mu], U[sb, mu].conj().T)
                        M[12 * s:12 * s + 12, 12 * sf:12 * sf + 12] -= kappa * fwd
                        M[12 * s:12 * s + 12, 12 * sb:12 * sb + 12] -= kappa * bwd
    return M


def oracle_columns(fn, n):
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1
        cols.append(np.asarray(fn(e)).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (4, 2, 2, 2)])
def test_dense_matrix_matches_stencil(oracle_mod, dims):
    U = inputs.gauge_field(dims, "random", seed=21)
    kappa = 0.124
    V = inputs.volume(dims)
    M = dense_wilson(U, dims, kappa, PHASES)
    Mo = oracle_columns(lambda e: oracle_mod.wilson_m(U, e.reshape(V, 4, 3), dims, kappa, PHASES), 12 * V)
    assert np.max(np.abs(M - Mo)) < 1e-14


def test_dense_free_field_spectrum_2x2x2x4(oracle_mod):
    """All eigenvalues of the free Wilson matrix on 2x2x2x4 with an
    antiperiodic t direction: 1 - 2 kappa sum cos p -+ 2 i kappa sqrt(sum sin^2 p)."""
    dims = (2, 2, 2, 4)
    phases = (1, 1, 1, -1)
    kappa = 0.11
    U = inputs.gauge_field(dims, "unit")
    V = inputs.volume(dims)
    M = oracle_columns(lambda e: oracle_mod.wilson_m(U, e.reshape(V, 4, 3), dims, kappa, phases), 12 * V)
    want = []
    for nx in range(2):
        for ny in range(2):
            for nz in range(2):
                for nt in range(4):
                    p = np.array([np.pi * nx, np.pi * ny, np.pi * nz, (2 * np.pi * nt + np.pi) / 4])
                    c = 1 - 2 * kappa * np.cos(p).sum()
                    s = 2 * kappa * np.sqrt((np.sin(p) ** 2).sum())
                    want += [c + 1j * s] * 6 + [c - 1j * s] * 6
    ev = np.linalg.eigvals(M)
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    assert sorted(map(key, ev)) == sorted(map(key, np.array(want)))


def test_schur_complement_dense(oracle_mod):
    dims = (2, 2, 2, 4)
    U = inputs.gauge_field(dims, "random", seed=22)
    kappa = 0.13
    V = inputs.volume(dims)
    Vh = V // 2
    M = dense_wilson(U, dims, kappa, PHASES)
    # permutation: canonical site order -> (even half, odd half)
    par = inputs.site_parity(dims)
    idx = np.arange(V)
    order = np.concatenate([idx[par == 0][np.argsort(idx[par == 0] >> 1)],
                            idx[par == 1][np.argsort(idx[par == 1] >> 1)]])
    perm = (12 * order[:, None] + np.arange(12)[None, :]).ravel()
    Mp = M[np.ix_(perm, perm)]
    n = 12 * Vh
    Mee, Meo, Moe, Moo = Mp[:n, :n], Mp[:n, n:], Mp[n:, :n], Mp[n:, n:]
    assert np.allclose(Mee, np.eye(n)) and np.allclose(Moo, np.eye(n))
    S = Mee - Meo @ np.linalg.solve(Moo, Moe)
    So = oracle_columns(lambda e: oracle_mod.schur(U, e.reshape(Vh, 4, 3), dims, kappa, 0, False, PHASES), n)
    assert np.max(np.abs(S - So)) < 1e-14
    Sd = oracle_columns(lambda e: oracle_mod.schur(U, e.reshape(Vh, 4, 3), dims, kappa, 0, True, PHASES), n)
    assert np.max(np.abs(S.conj().T - Sd)) < 1e-14
    # odd-parity Schur complement too
    S1 = Moo - Moe @ np.linalg.solve(Mee, Meo)
    So1 = oracle_columns(lambda e: oracle_mod.schur(U, e.reshape(Vh, 4, 3), dims, kappa, 1, False, PHASES), n)
    assert np.max(np.abs(S1 - So1)) < 1e-14


@pytest.mark.parametrize("dims,kind,kappa", [((2, 2, 2, 4), "random", 0.124), ((4, 2, 2, 4), "weak", 0.135),
                                             ((2, 2, 2, 2), "random", 0.12)])
def test_cg_matches_dense_lu(oracle_mod, dims, kind, kappa):
    U = inputs.gauge_field(dims, kind, eps=0.3, seed=23)
    V = inputs.volume(dims)
    b = inputs.gaussian_spinor(dims, seed=24)
    M = dense_wilson(U, dims, kappa, PHASES)
    x_lu = np.linalg.solve(M, b.ravel())
    sv = np.linalg.svd(M, compute_uv=False)
    cond = sv[0] / sv[-1]
    x, info = oracle_mod.cg_solve(U, b, dims, kappa, tol=1e-10, phases=PHASES)
    assert info["converged"]
    assert info["true_rel_resid"] <= 1e-10
    # independent residual from the dense matrix
    assert np.linalg.norm(b.ravel() - M @ x.ravel()) <= 1e-10 * np.linalg.norm(b)
    assert rel_l2(x, x_lu) <= cond * 1e-10


def test_cg_zero_source(oracle_mod):
    dims = (2, 2, 2, 2)
    U = inputs.gauge_field(dims, "random", seed=25)
    x, info = oracle_mod.cg_solve(U, np.zeros((16, 4, 3)), dims, 0.12)
    assert info["converged"] and np.all(x == 0)


def test_cg_maxiter_reported(oracle_mod):
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, "weak", eps=0.3, seed=26)
    b = inputs.gaussian_spinor(dims, seed=27)
    x, info = oracle_mod.cg_solve(U, b, dims, 0.135, tol=1e-10, maxiter=3)
    assert not info["converged"] and info["iterations"] == 3
