"""The t-decomposition's host side on the CPU: the split of fields into
sub-lattices (contiguous slices with the global parity), and the halo
exchange between processes with gloo ranks (2 and 3 ranks) and in one
process (loopback)."""
import os
import socket
import sys

import numpy as np
import pytest

from conftest import parity_split
from paper_0710_2442_gb300 import inputs
from paper_0710_2442_gb300.dd import TSplit, exchange_dist, exchange_loopback

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_rejects_odd_or_uneven_extents():
    for n in (3, 16, 0):
        with pytest.raises(ValueError):
            TSplit((4, 4, 4, 8), n)
    with pytest.raises(ValueError):
        TSplit((4, 4, 4, 6), 2)  # Lr = 3 is odd


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 8), 2), ((4, 4, 4, 8), 4), ((6, 4, 2, 12), 3), ((2, 2, 2, 2), 1)])
def test_split_is_the_sub_lattices_own_layout(dims, n):
    """Sub-lattice r's parity fields, laid out on its own lattice {Lx, Ly,
    Lz, Lr}, are the global parity fields' half-site range of its t-slices,
    and its links the global links of its sites."""
    sp = TSplit(dims, n)
    V = inputs.volume(dims)
    psi = inputs.gaussian_spinor(V, seed=7)
    U = inputs.gauge_field(dims, "random", seed=8)
    even, odd = parity_split(psi, dims)
    loc = sp.local_dims
    Vl = inputs.volume(loc)
    for r, (ue, uo, ul) in enumerate(zip(sp.split_half(even), sp.split_half(odd), sp.split_gauge(U))):
        sl = psi[r * Vl:(r + 1) * Vl]          # the sub-lattice's sites, canonical order (t slowest)
        le, lo = parity_split(sl, loc)          # its own parity fields
        assert np.array_equal(ue, le) and np.array_equal(uo, lo)
        assert np.array_equal(ul, U[r * Vl:(r + 1) * Vl])
        assert sp.first(r) == (r == 0) and sp.last(r) == (r == n - 1)
    assert np.array_equal(sp.gather_half(sp.split_half(even)), even)


def test_loopback_exchange_routes_faces():
    import torch
    sp = TSplit((4, 4, 4, 8), 4)
    sp_prev = [torch.full((5,), 10.0 * r + 1) for r in range(4)]
    sp_next = [torch.full((5,), 10.0 * r + 2) for r in range(4)]
    rn = [torch.zeros(5) for _ in range(4)]
    rp = [torch.zeros(5) for _ in range(4)]
    exchange_loopback(sp, sp_prev, sp_next, rn, rp)
    for r in range(4):
        assert torch.all(rn[r] == 10.0 * sp.next(r) + 1)  # the next sub-lattice's first slice
        assert torch.all(rp[r] == 10.0 * sp.prev(r) + 2)  # the previous one's last slice


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_0710_2442_gb300.dd import TSplit as TS, exchange_dist as ex
    dist.init_process_group("gloo")
    sp = TS((4, 4, 4, 2 * world), world)
    n = 7
    send_prev = torch.full((n,), 10.0 * rank + 1)
    send_next = torch.full((n,), 10.0 * rank + 2)
    recv_next = torch.zeros(n)
    recv_prev = torch.zeros(n)
    for _ in range(2):  # twice: the buffers are reused across applications
        ex(sp, rank, send_prev, send_next, recv_next, recv_prev)
    ok = bool(torch.all(recv_next == 10.0 * sp.next(rank) + 1)) and bool(torch.all(recv_prev == 10.0 * sp.prev(rank) + 2))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write("ok" if ok else f"bad {recv_next.tolist()} {recv_prev.tolist()}")
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_exchange(tmp_path, world):
    """One sub-lattice per process: every rank receives its next neighbour's
    first slice and its previous neighbour's last slice (with two ranks both
    neighbours are the same process)."""
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        assert open(tmp_path / f"rank{r}.txt").read() == "ok"
