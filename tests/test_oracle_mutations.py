"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), builds it, swaps it in, and runs a fixed set of
the pins from the other oracle tests: at least one of them must fail.  The
unmodified source must pass all of them.
"""
import contextlib
import ctypes
import os
import subprocess

import pytest

import test_oracle_dense as dense
import test_oracle_gamma_free_field as ff
import test_oracle_identities as ident

MUTATIONS = {
    "backward link not conjugated": ("dagger ? conj(U[3 * j + i]) : U[3 * i + j]", "dagger ? U[3 * j + i] : U[3 * i + j]"),
    "backward link not transposed": ("dagger ? conj(U[3 * j + i]) : U[3 * i + j]", "dagger ? conj(U[3 * i + j]) : U[3 * i + j]"),
    "forward link transposed": ("dagger ? conj(U[3 * j + i]) : U[3 * i + j]", "dagger ? conj(U[3 * j + i]) : U[3 * j + i]"),
    "backward phase not conjugated": ("(c[mu] == 0) ? conj(phase[mu]) : 1.0", "(c[mu] == 0) ? phase[mu] : 1.0"),
    "forward phase on the wrong boundary": ("(c[mu] == L[mu] - 1) ? phase[mu] : 1.0", "(c[mu] == 0) ? phase[mu] : 1.0"),
    "backward link taken at x": ("U + LINK_CPLX * (4 * sb + mu), mu, -conv", "U + LINK_CPLX * (4 * s + mu), mu, -conv"),
    "backward projector sign": ("mu, -conv, 1, eta_b", "mu, conv, 1, eta_b"),
    "gamma_2 entry sign": ("G[1][0][3] = -1;", "G[1][0][3] = 1;"),
    "gamma_3 entry sign": ("G[2][1][3] = -iu;", "G[2][1][3] = iu;"),
    "t direction dropped": ("    for (int mu = 0; mu < 4; mu++) {\n        int cf[4]", "    for (int mu = 0; mu < 3; mu++) {\n        int cf[4]"),
    "wilson M sign": ("out[i] = in[i] - kappa * out[i];", "out[i] = in[i] + kappa * out[i];"),
    "schur kappa not squared": ("res[i] = src[i] - kappa * kappa * res[i];", "res[i] = src[i] - kappa * res[i];"),
    "bhat sign": ("bh[i] = be[i] + kappa * bh[i];", "bh[i] = be[i] - kappa * bh[i];"),
    "odd reconstruction sign": ("q[i] = bo[i] + kappa * q[i];", "q[i] = bo[i] - kappa * q[i];"),
    "eo extraction parity": ("if (parity_of(c) == par) memcpy(half + SPINOR_CPLX * (s >> 1)", "if (parity_of(c) != par) memcpy(half + SPINOR_CPLX * (s >> 1)"),
}


def pins(o, stop_at_first=False):
    """Run the pin set against oracle module o; returns the failing checks
    (all of them, or only the first with stop_at_first)."""
    checks = [
        lambda: ff.test_free_field_plane_wave_pointwise(o, *ff.CASES[2], 1),
        lambda: ff.test_free_field_spectrum_basis_independent(o, *ff.CASES[3]),
        lambda: ff.test_gamma_table_is_degrand_rossi(o),
        lambda: ident.test_gamma5_hermiticity(o, (4, 2, 6, 8)),
        lambda: ident.test_gauge_covariance(o, (4, 2, 6, 8)),
        lambda: ident.test_linearity_and_wilson_m(o),
        lambda: ident.test_eo_blocks_equal_restricted_full_hop(o, (4, 6, 2, 8), 0),
        lambda: dense.test_dense_matrix_matches_stencil(o, (2, 2, 2, 4)),
        lambda: dense.test_schur_complement_dense(o),
        lambda: dense.test_cg_matches_dense_lu(o, (2, 2, 2, 4), "random", 0.124),
    ]
    fails = []
    for i, c in enumerate(checks):
        try:
            c()
        except (AssertionError, ValueError):
            fails.append(i)
            if stop_at_first:
                break
    return fails


@contextlib.contextmanager
def swapped(oracle_mod, source, tmp_path):
    src = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    src.write_text(source)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(src), "-lm"],
                   check=True)
    lib = oracle_mod.declare(ctypes.CDLL(str(so)))
    saved = oracle_mod._load()
    oracle_mod._lib = lib
    try:
        yield
    finally:
        oracle_mod._lib = saved


def test_unmodified_source_passes_all_pins(oracle_mod, tmp_path):
    with swapped(oracle_mod, open(oracle_mod._SRC).read(), tmp_path):
        assert pins(oracle_mod) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name):
    old, new = MUTATIONS[name]
    text = open(oracle_mod._SRC).read()
    assert text.count(old) == 1, f"mutation anchor not unique: {name}"
    with swapped(oracle_mod, text.replace(old, new), tmp_path):
        assert pins(oracle_mod, stop_at_first=True), f"no pin caught: {name}"
