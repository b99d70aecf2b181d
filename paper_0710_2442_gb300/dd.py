"""Domain decomposition of the even-odd hopping term along t: the
sub-lattices, the split and gather of fields, and the halo exchange.

The paper decomposes its lattice over the SPEs of a Cell and over Cell
nodes (Sec. 5); the communication between nodes carries projected half
spinors, 12 reals per boundary site and face (T_ext of Table 1).  Here the
lattice Lx x Ly x Lz x Lt is cut into n sub-lattices of Lr = Lt / n
consecutive t-slices (Lr even, so that each starts at an even t and its
local parity is the global one).  Sub-lattice r holds the global t-slices
[r Lr, (r + 1) Lr); with the canonical site order (t slowest) its fields are
contiguous slices of the global ones: sites [t0 Vs, (t0 + Lr) Vs) of a full
field, half sites [t0 Vs / 2, (t0 + Lr) Vs / 2) of a parity field
(Vs = Lx Ly Lz, even).

One application of D_{p,1-p} is: ``wilson_dd_pack`` on every sub-lattice
(two face buffers each), the exchange below, ``wilson_dd_hop`` on every
sub-lattice.  The exchange moves sub-lattice r's ``send_prev`` buffer to
sub-lattice r - 1's ``recv_next`` and its ``send_next`` to sub-lattice
r + 1's ``recv_prev`` (cyclically): device copies when the sub-lattices
share a GPU (``exchange_loopback``), point-to-point sends between processes
otherwise (``exchange_dist``: NCCL between GPUs, gloo on the CPU).  This
module only moves buffers and slices arrays; every operator step runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np

# message tags: a buffer travelling to the previous sub-lattice, to the next
TAG_TO_PREV, TAG_TO_NEXT = 11, 12


class TSplit:
    """The t-split of a lattice into n sub-lattices of equal even extent."""

    def __init__(self, dims, n: int):
        dims = tuple(int(d) for d in dims)
        if n < 1 or dims[3] % n or (dims[3] // n) % 2:
            raise ValueError(f"Lt = {dims[3]} does not split into {n} sub-lattices of even extent")
        self.dims = dims
        self.n = n
        self.Lr = dims[3] // n
        self.Vs = dims[0] * dims[1] * dims[2]

    @property
    def local_dims(self):
        return (self.dims[0], self.dims[1], self.dims[2], self.Lr)

    def t0(self, r: int) -> int:
        return r * self.Lr

    def prev(self, r: int) -> int:
        return (r - 1) % self.n

    def next(self, r: int) -> int:
        return (r + 1) % self.n

    def first(self, r: int) -> bool:
        """Sub-lattice r holds the lattice's first t-slice (its backward face wraps)."""
        return r == 0

    def last(self, r: int) -> bool:
        """Sub-lattice r holds the lattice's last t-slice (its forward face wraps)."""
        return r == self.n - 1

    def full_range(self, r: int) -> slice:
        return slice(self.t0(r) * self.Vs, (self.t0(r) + self.Lr) * self.Vs)

    def half_range(self, r: int) -> slice:
        return slice(self.t0(r) * self.Vs // 2, (self.t0(r) + self.Lr) * self.Vs // 2)

    def split_gauge(self, U):
        """Global canonical links [V, 4, 3, 3] -> the sub-lattices' links."""
        return [U[self.full_range(r)] for r in range(self.n)]

    def split_half(self, psi):
        """Global parity field [V/2, ...] -> the sub-lattices' parity fields."""
        return [psi[self.half_range(r)] for r in range(self.n)]

    def gather_half(self, parts):
        """The sub-lattices' parity fields -> the global parity field."""
        if len(parts) != self.n:
            raise ValueError("one part per sub-lattice")
        if isinstance(parts[0], np.ndarray):
            return np.concatenate(parts, axis=0)
        import torch
        return torch.cat(list(parts), dim=0)


def exchange_loopback(split: TSplit, send_prev, send_next, recv_next, recv_prev):
    """All sub-lattices in one process (one GPU): every face buffer is copied
    to the sub-lattice that needs it, on the current stream."""
    for r in range(split.n):
        recv_next[split.prev(r)].copy_(send_prev[r])
        recv_prev[split.next(r)].copy_(send_next[r])


def exchange_dist(split: TSplit, rank: int, send_prev, send_next, recv_next, recv_prev, group=None):
    """One sub-lattice per process (rank r holds sub-lattice r): send_prev to
    rank r - 1, where it arrives as recv_next; send_next to rank r + 1, where
    it arrives as recv_prev.  Both directions are posted at once, in the same
    order on every rank, so that neither NCCL (which matches by order) nor
    gloo (which also matches tags) can deadlock, also when both neighbours are
    the same rank (n = 2).  Returns after the buffers have arrived."""
    import torch.distributed as dist
    if split.n == 1:
        recv_next.copy_(send_prev)
        recv_prev.copy_(send_next)
        return
    prev, nxt = split.prev(rank), split.next(rank)
    ops = [dist.P2POp(dist.isend, send_prev, prev, group, TAG_TO_PREV),
           dist.P2POp(dist.isend, send_next, nxt, group, TAG_TO_NEXT),
           dist.P2POp(dist.irecv, recv_next, nxt, group, TAG_TO_PREV),
           dist.P2POp(dist.irecv, recv_prev, prev, group, TAG_TO_NEXT)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
