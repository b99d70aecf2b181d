"""Flop and byte constants of the hopping term, used for every reported rate.

Flops: 1320 per output site (Sec. 5: sign flips and complex conjugations are
not counted).  Per hop: spin projection 6 complex adds (12 flops), two 3x3
complex matrix-vector products (2 x 66 flops), accumulation into the 4-spinor
12 complex adds (24 flops): 168 flops, times 8 hops, minus the 24 flops of the
first hop, which needs no accumulation.

Bytes: the compulsory ("algorithmic") traffic of one application counts every
input spinor, link and output spinor once.  In double precision this is the
model behind the paper's T_mem row of Table 1 (192 B in + 4 x 144 B links +
192 B out per site for the full operator); the even-odd operator reads 8 links
per output site because the links of both parities are read once per half
sweep.
"""
from __future__ import annotations

FLOPS_PER_SITE = 1320
HOP_FLOPS = 12 + 2 * 66 + 24       # 168
MULADDS_PER_SITE_MIN = 840         # Sec. 5, lower bound on multiply-adds

# bytes of one spinor / one link by storage format
SPINOR_BYTES = {"f64": 24 * 8, "f32": 24 * 4, "f16": 24 * 2 + 4, "bf16": 24 * 2 + 4}
LINK_BYTES = {("f64", 18): 18 * 8, ("f64", 12): 12 * 8, ("f32", 18): 18 * 4, ("f32", 12): 12 * 4,
              ("f16", 12): 12 * 2, ("bf16", 12): 12 * 2, ("f16", 18): 18 * 2, ("bf16", 18): 18 * 2}
HALF_SPINOR_BYTES_F64 = 12 * 8     # a projected half spinor in double precision


def compulsory_bytes_per_site(prec: str, recon: int, eo: bool, nrhs: int = 1) -> int:
    """Algorithmic bytes per output site of one hopping-term application."""
    links = 8 if eo else 4
    return 2 * nrhs * SPINOR_BYTES[prec] + links * LINK_BYTES[(prec, recon)]


def naive_bytes_per_site(prec: str, recon: int) -> int:
    """All operands of one site as Sec. 5 lists them: 9 spinors (8 neighbours
    + the result) and 8 links."""
    return 9 * SPINOR_BYTES[prec] + 8 * LINK_BYTES[(prec, recon)]


def cell_table1(sites_per_spe, sites_per_cell, a_ext, clock_hz=3.2e9, n_spe=8,
                beta_mem=25.6e9, beta_ext=6.0e9, t_peak_site=330, t_fp_site=420):
    """The Eq. 1 / Eq. 2 estimates of Table 1 (in SPE cycles) from the byte
    and flop constants above: returns dict(T_peak, T_FP, T_mem, T_ext)."""
    out = {
        "T_peak": t_peak_site * sites_per_spe,
        "T_FP": t_fp_site * sites_per_spe,
        "T_ext": n_spe * a_ext * HALF_SPINOR_BYTES_F64 / beta_ext * clock_hz,
    }
    if sites_per_cell is not None:
        out["T_mem"] = sites_per_cell * compulsory_bytes_per_site("f64", 18, eo=False) / beta_mem * clock_hz
    return out


def cg_inner_bytes_per_site(inner: str, recon: int = 12) -> int:
    """Algorithmic bytes per even site of one inner CG iteration of the
    solver, counted over its six launches: two Schur operators (four hops;
    the second hop of each also reads the xpay field), the x/s update (x and s
    read and written in the accumulation precision, p and q read, and for
    F16/BF16 the copy of s in storage precision written), and p = r + beta p."""
    S = SPINOR_BYTES[inner]
    L = LINK_BYTES[(inner, recon)]
    X = SPINOR_BYTES["f64" if inner == "f64" else "f32"]
    schur = (2 * S + 8 * L) + (3 * S + 8 * L)
    xs = 4 * X + 2 * S + (S if inner in ("f16", "bf16") else 0)
    p_update = 3 * S
    return 2 * schur + xs + p_update
