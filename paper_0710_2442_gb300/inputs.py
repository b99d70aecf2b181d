"""Seeded synthetic inputs: gauge fields, spinor sources and workload presets.

This module is shared by the oracle side (tests, CPU baseline) and the GPU
side (tests, bench).  It draws random numbers and builds fields in the
canonical layout; it holds none of the Wilson operator's arithmetic.

Canonical layout (complex128):
  spinor  [V, 4, 3]        site, spin, colour
  gauge   [V, 4, 3, 3]     site, mu (x, y, z, t), row, col
  site index s = x + Lx*(y + Ly*(z + Lz*t))

Field recipes (the workloads the paper's Sec. 5 kernel is run on; the paper
itself fixes none of them):
  * random SU(3): complex Gaussian 3x3, rows orthonormalised by Gram-Schmidt,
    then multiplied by exp(-i arg(det)/3) with arg in (-pi, pi] so det = 1.
  * weak field: U = exp(i eps H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0,1)
    and lambda_a the Gell-Mann matrices; exp by a batched matrix exponential,
    then the same projection onto SU(3).
  * Gaussian spinor: real and imaginary parts i.i.d. N(0, 1).
"""
from __future__ import annotations

import numpy as np

DEFAULT_PHASES = (1.0 + 0j, 1.0 + 0j, 1.0 + 0j, -1.0 + 0j)  # periodic x,y,z; antiperiodic t
SEED_BASE = 2442


def volume(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def site_coords(dims) -> np.ndarray:
    """int64[V, 4] coordinates (x, y, z, t) of every site in canonical order."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1).astype(np.int64)


def site_parity(dims) -> np.ndarray:
    """int8[V]: (x+y+z+t) mod 2 of every site in canonical order."""
    return (site_coords(dims).sum(axis=1) & 1).astype(np.int8)


def make_rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# SU(3)
# --------------------------------------------------------------------------
def project_su3(m: np.ndarray) -> np.ndarray:
    """Gram-Schmidt the rows of each 3x3 matrix, then remove the det phase."""
    m = np.array(m, dtype=np.complex128, copy=True)
    r0 = m[:, 0, :]
    r0 /= np.linalg.norm(r0, axis=1, keepdims=True)
    r1 = m[:, 1, :]
    r2 = m[:, 2, :]
    for _ in range(2):  # Gram-Schmidt twice keeps orthogonality at rounding level
        r1 -= np.sum(np.conj(r0) * r1, axis=1, keepdims=True) * r0
    r1 /= np.linalg.norm(r1, axis=1, keepdims=True)
    for _ in range(2):
        r2 -= np.sum(np.conj(r0) * r2, axis=1, keepdims=True) * r0
        r2 -= np.sum(np.conj(r1) * r2, axis=1, keepdims=True) * r1
    r2 /= np.linalg.norm(r2, axis=1, keepdims=True)
    phi = np.angle(np.linalg.det(m))
    m *= np.exp(-1j * phi / 3.0)[:, None, None]
    return m


def random_su3(rng, n: int) -> np.ndarray:
    rng = make_rng(rng)
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    return project_su3(z)


def gell_mann() -> np.ndarray:
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def _project_su3_torch(u):
    """project_su3 on a torch complex128 tensor [n, 3, 3] (multi-threaded)."""
    import torch
    r0 = u[:, 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=1, keepdim=True)
    r1 = u[:, 1, :]
    r2 = u[:, 2, :]
    for _ in range(2):
        r1 = r1 - (r0.conj() * r1).sum(dim=1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=1, keepdim=True)
    for _ in range(2):
        r2 = r2 - (r0.conj() * r2).sum(dim=1, keepdim=True) * r0
        r2 = r2 - (r1.conj() * r2).sum(dim=1, keepdim=True) * r1
    r2 = r2 / torch.linalg.vector_norm(r2, dim=1, keepdim=True)
    m = torch.stack([r0, r1, r2], dim=1)
    det = torch.linalg.det(m)
    return m * torch.exp(-1j * torch.angle(det) / 3.0)[:, None, None]


def weak_field_su3(rng, n: int, eps, chunk: int = 1 << 20) -> np.ndarray:
    """exp(i eps H) with H = sum_a h_a lambda_a / 2; eps scalar or per-matrix.

    The coefficients h_a are drawn with numpy (seeded); the exponential is a
    batched matrix exponential (torch, CPU), followed by the SU(3) projection."""
    import torch
    rng = make_rng(rng)
    lam = torch.from_numpy(gell_mann() / 2.0)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    eps_arr = np.broadcast_to(np.asarray(eps, dtype=np.float64), (n,))
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        h = torch.from_numpy(rng.standard_normal((b - a, 8))).to(torch.complex128)
        H = torch.einsum("na,aij->nij", h, lam)
        e = torch.from_numpy(np.ascontiguousarray(eps_arr[a:b])).to(torch.complex128)
        u = torch.linalg.matrix_exp(1j * e[:, None, None] * H)
        out[a:b] = _project_su3_torch(u).numpy()
    return out


def gauge_field(dims, kind: str = "weak", eps: float = 0.3, seed=SEED_BASE) -> np.ndarray:
    """complex128[V, 4, 3, 3] gauge field: kind in {'weak', 'random', 'unit'}."""
    V = volume(dims)
    if kind == "unit":
        U = np.zeros((V * 4, 3, 3), dtype=np.complex128)
        U[:, 0, 0] = U[:, 1, 1] = U[:, 2, 2] = 1
    elif kind == "random":
        U = random_su3(make_rng(seed), V * 4)
    elif kind == "weak":
        U = weak_field_su3(make_rng(seed), V * 4, eps)
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return U.reshape(V, 4, 3, 3)


def gaussian_spinor(dims_or_nsites, seed=SEED_BASE + 1, nrhs: int | None = None) -> np.ndarray:
    """complex128[n, 4, 3] (or [nrhs, n, 4, 3]) with N(0,1) real and imaginary parts."""
    n = volume(dims_or_nsites) if np.ndim(dims_or_nsites) else int(dims_or_nsites)
    rng = make_rng(seed)
    shape = (n, 4, 3) if nrhs is None else (nrhs, n, 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def point_sources(dims, site: int = 0) -> np.ndarray:
    """complex128[12, V, 4, 3]: one unit source per (spin, colour) at one site."""
    V = volume(dims)
    b = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for k in range(12):
        b[k, site, k // 3, k % 3] = 1.0
    return b


def random_gauge_transform(rng, n: int) -> np.ndarray:
    return random_su3(rng, n)


# --------------------------------------------------------------------------
# workload presets (lattice, fields, kappa, seeds)
# --------------------------------------------------------------------------
WORKLOADS = {
    # full F64 hopping term, random SU(3) links
    "dslash_f64_8^4": dict(dims=(8, 8, 8, 8), gauge="random", eps=None, kappa=0.125,
                           gauge_seed=SEED_BASE, spinor_seed=SEED_BASE + 1),
    # F32 even-odd hopping term, 12-real links, weak field
    "dslash_eo_f32_32^3x64": dict(dims=(32, 32, 32, 64), gauge="weak", eps=0.3, kappa=0.1350,
                                  gauge_seed=SEED_BASE + 10, spinor_seed=SEED_BASE + 11,
                                  applications=100),
    # mixed-precision CG on the even-odd Schur complement
    "cg_mixed_24^3x48": dict(dims=(24, 24, 24, 48), gauge="weak", eps=0.3, kappa=0.1350,
                             gauge_seed=SEED_BASE + 20, spinor_seed=SEED_BASE + 21, tol=1e-10),
    # 12 right-hand sides sharing one gauge field
    "multirhs12_32^3x64": dict(dims=(32, 32, 32, 64), gauge="weak", eps=0.3, kappa=0.1350,
                               gauge_seed=SEED_BASE + 30, spinor_seed=SEED_BASE + 31, nrhs=12),
}

# uneven batch: (dims, count)
BATCH_MIX = (((8, 8, 8, 8), 32), ((12, 12, 12, 12), 16), ((16, 16, 16, 32), 12), ((24, 24, 24, 48), 4))


def batch_problems(seed=SEED_BASE + 40, mix=BATCH_MIX, eps_range=(0.2, 0.4),
                   kappa_range=(0.125, 0.1355)):
    """The uneven batch: a shuffled list of dicts(dims, eps, kappa, gauge_seed, spinor_seed)."""
    rng = make_rng(seed)
    probs = []
    for dims, count in mix:
        for _ in range(count):
            probs.append(dict(dims=tuple(dims)))
    order = rng.permutation(len(probs))
    probs = [probs[i] for i in order]
    for i, p in enumerate(probs):
        p["eps"] = float(rng.uniform(*eps_range))
        p["kappa"] = float(rng.uniform(*kappa_range))
        p["gauge_seed"] = int(seed * 1000 + 2 * i)
        p["spinor_seed"] = int(seed * 1000 + 2 * i + 1)
    return probs
