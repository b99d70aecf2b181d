"""Helpers of the GPU tests: move canonical numpy fields to and from the GPU."""
import numpy as np


def dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def host(t) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def empty_like_dev(a: np.ndarray):
    import torch
    return torch.full(a.shape, float("nan"), dtype=torch.complex128, device="cuda")


def handle_hop(w, U, src, dims, phases, prec, recon, in_subset, out_subset, op, kappa=0.0, nrhs=1):
    """Apply an operator through the handle API; returns the canonical result."""
    L = w.lattice(dims, phases)
    g = w.Gauge(U, L, prec, recon)  # host canonical links, staged by the library
    a = w.Spinor(L, in_subset, prec, nrhs)
    b = w.Spinor(L, out_subset, prec, nrhs)
    a.load(dev(src))
    w.wilson_dslash_h(b, g, a, kappa, op)
    out_shape = list(src.shape)
    V = int(np.prod(dims))
    n_out = V if out_subset == w.WILSON_FULL else V // 2
    out_shape[-3] = n_out
    out = empty_like_dev(np.zeros(out_shape, dtype=np.complex128))
    b.store(out)
    res = host(out)
    for h in (g, a, b):
        h.close()
    return res
