"""A tuning-cache file whose decisions this build cannot launch (here every
variant rewritten to 99) is ignored: the keys are tuned again, the operator
runs, and its result agrees with the one computed with the valid cache."""
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
U = inputs.gauge_field(dims, "weak", eps=0.3, seed=151)
Vh = inputs.volume(dims) // 2
g = w.Gauge(U, L, w.WILSON_F32, 12)
a = w.Spinor(L, w.WILSON_EVEN, w.WILSON_F32)
b = w.Spinor(L, w.WILSON_ODD, w.WILSON_F32)
a.load(torch.from_numpy(inputs.gaussian_spinor(Vh, seed=152)).cuda())
w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP)
out = torch.empty((Vh, 4, 3), dtype=torch.complex128, device="cuda")
b.store(out)
torch.cuda.synchronize()
np.save(sys.argv[1], out.cpu().numpy())
'''


def run_child(tmp_path, cache, dest):
    script = tmp_path / "hop.py"
    script.write_text(CHILD)
    env = dict(os.environ, WILSON_TUNE_CACHE=str(cache))
    subprocess.run([sys.executable, str(script), str(dest), ROOT], check=True, env=env, cwd=ROOT, timeout=600)
    return np.load(dest)


def test_foreign_cache_entries_are_retuned(tmp_path):
    cache = tmp_path / "tune.txt"
    first = run_child(tmp_path, cache, tmp_path / "a.npy")
    lines = cache.read_text().splitlines()
    assert lines, "the first run stores its decisions"
    # key block variant us  ->  key block 99 us
    cache.write_text("".join(f"{ln.split()[0]} {ln.split()[1]} 99 {ln.split()[3]}\n" for ln in lines))
    second = run_child(tmp_path, cache, tmp_path / "b.npy")
    # the re-tuned launch may be another variant: equal within the F32 tolerance
    assert np.linalg.norm(second - first) <= 1e-6 * np.linalg.norm(first)
    retuned = [ln.split() for ln in cache.read_text().splitlines()[len(lines):]]
    assert retuned and all(r[2] != "99" for r in retuned)
