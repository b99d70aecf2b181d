"""Programmatic dependent launch leaves results unchanged: chains of 40
back-to-back hop applications (F32 and F16 single right-hand side, F32 and F16
over 12 right-hand sides) give bit-identical fields with the launch attribute
(default) and without it (WILSON_PDL=0).  A hop that touched memory before
its predecessor completed would race with it and break the equality.  The
library reads WILSON_PDL once per process, so each setting runs in a child
process."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[2])
from paper_0710_2442_gb300 import build, inputs, wilson as w
build.build()
dims = (8, 8, 8, 16)
L = w.lattice(dims)
U = inputs.gauge_field(dims, "weak", eps=0.3, seed=141)
Vh = inputs.volume(dims) // 2
out = {}
for name, prec, n in (("f32_1", w.WILSON_F32, 1), ("f16_1", w.WILSON_F16, 1),
                      ("f32_12", w.WILSON_F32, 12), ("f16_12", w.WILSON_F16, 12)):
    g = w.Gauge(U, L, prec, 12)
    a = w.Spinor(L, w.WILSON_EVEN, prec, n)
    b = w.Spinor(L, w.WILSON_ODD, prec, n)
    a.load(torch.from_numpy(inputs.gaussian_spinor(Vh, seed=142, nrhs=n)).cuda())
    for _ in range(20):
        w.wilson_dslash_h(b, g, a, 0.125, w.WILSON_OP_HOP)
        w.wilson_dslash_h(a, g, b, 0.125, w.WILSON_OP_HOP)
    res = torch.empty((n, Vh, 4, 3) if n > 1 else (Vh, 4, 3), dtype=torch.complex128, device="cuda")
    a.store(res)
    torch.cuda.synchronize()
    out[name] = res.cpu().numpy()
    for h in (g, a, b):
        h.close()
np.savez(sys.argv[1], **out)
'''


def run_child(tmp_path, pdl):
    script = tmp_path / "chain.py"
    script.write_text(CHILD)
    dest = tmp_path / f"chain_pdl{pdl}.npz"
    # one tuning cache for both children: the same launch configurations run
    env = dict(os.environ, WILSON_PDL=str(pdl), WILSON_TUNE_CACHE=str(tmp_path / "tune.txt"))
    subprocess.run([sys.executable, str(script), str(dest), ROOT], check=True, env=env, cwd=ROOT, timeout=600)
    return np.load(dest)


def test_pdl_chain_bit_identical(tmp_path):
    on = run_child(tmp_path, 1)
    off = run_child(tmp_path, 0)
    assert set(on.files) == set(off.files) == {"f32_1", "f16_1", "f32_12", "f16_12"}
    for k in on.files:
        assert np.isfinite(on[k]).all(), k
        assert np.array_equal(on[k].view(np.uint64), off[k].view(np.uint64)), k
