"""The solver workloads at their full sizes, checked against the FP64 oracle:
every solution's true residual |b - M x| / |b| is recomputed by the oracle's
Wilson matrix (<= 1e-10, with 10% slack for the summation order).

- the mixed-precision CG on 24^3 x 48 (kappa 0.135) in every inner precision
  and in plain FP64, and the agreement of the mixed solutions with the FP64
  one;
- 12 spin-colour point sources on 32^3 x 64 sharing one gauge field, solved
  as lockstep CGs and as one block CG;
- the batch of 64 uneven problems in one graph launch.
"""
import numpy as np
import pytest

from conftest import rel_l2
from gpu_helpers import dev, host
from paper_0710_2442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    from paper_0710_2442_gb300 import build, wilson
    build.build()
    return wilson


def true_resid(oracle_mod, U, x, b, dims, kappa):
    return np.linalg.norm(b - oracle_mod.wilson_m(U, x, dims, kappa)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def cg_fields():
    cfg = inputs.WORKLOADS["cg_mixed_24^3x48"]
    U = inputs.gauge_field(cfg["dims"], cfg["gauge"], eps=cfg["eps"], seed=cfg["gauge_seed"])
    b = inputs.gaussian_spinor(cfg["dims"], seed=cfg["spinor_seed"])
    return cfg, U, b


def test_cg_workload_24x24x24x48(w, oracle_mod, cg_fields):
    cfg, U, b = cg_fields
    dims, kappa = cfg["dims"], cfg["kappa"]
    L = w.lattice(dims)
    Ud, bd = dev(U), dev(b)
    sols = {}
    for name in ("f64", "f16", "bf16", "f32"):
        x = dev(np.zeros_like(b))
        st = w.wilson_cg_solve(x, Ud, bd, L, kappa, w.solver_defaults(w.PREC[name]))
        assert st["rc"] == 0 and st["true_rel_resid"] <= cfg["tol"]
        sols[name] = host(x)
        assert true_resid(oracle_mod, U, sols[name], b, dims, kappa) <= 1.1 * cfg["tol"], name
    for name in ("f16", "bf16", "f32"):
        # two solutions with residual 1e-10 differ by at most cond(M) * 2e-10
        assert rel_l2(sols[name], sols["f64"]) <= 1e-7, name


@pytest.fixture(scope="module")
def mrhs_fields():
    # the links of the headline workload, as the benchmark's multi-RHS block uses them
    cfg = inputs.WORKLOADS["multirhs12_32^3x64"]
    hl = inputs.WORKLOADS["dslash_eo_f32_32^3x64"]
    U = inputs.gauge_field(hl["dims"], hl["gauge"], eps=hl["eps"], seed=hl["gauge_seed"])
    b = inputs.point_sources(cfg["dims"], site=0)
    return cfg, U, b


@pytest.mark.parametrize("block", [0, 1])
def test_multirhs_workload_32x32x32x64(w, oracle_mod, mrhs_fields, block):
    cfg, U, b = mrhs_fields
    dims, kappa = cfg["dims"], cfg["kappa"]
    p = w.solver_defaults(w.WILSON_F16)
    p.block_cg = block
    x = dev(np.zeros_like(b))
    rc, st = w.wilson_cg_solve_multi(x, dev(U), dev(b), 12, w.lattice(dims), kappa, p)
    assert rc == 0
    xs = host(x)
    for k in range(12):
        assert st[k]["true_rel_resid"] <= 1e-10
        assert true_resid(oracle_mod, U, xs[k], b[k], dims, kappa) <= 1.1e-10, k


def test_batch_workload_64_uneven(w, oracle_mod):
    probs = inputs.batch_problems()
    fields, host_fields = [], []
    for p in probs:
        U = inputs.gauge_field(p["dims"], "weak", eps=p["eps"], seed=p["gauge_seed"])
        b = inputs.gaussian_spinor(p["dims"], seed=p["spinor_seed"])
        fields.append(dict(L=w.lattice(p["dims"]), kappa=p["kappa"], gauge=dev(U), b=dev(b),
                           x=dev(np.zeros_like(b))))
        host_fields.append((p["dims"], U, b, p["kappa"]))
    rc, st, info = w.wilson_batch_solve(fields, w.solver_defaults(w.WILSON_F16))
    assert rc == 0 and info["graph_launches"] == 1 and info["device_loop"] == 1 and not info["timed_out"]
    for f, (dims, U, b, kappa), s in zip(fields, host_fields, st):
        assert s["status"] == 0 and 0 <= s["seconds"] <= info["device_seconds"] + 1e-6
        assert true_resid(oracle_mod, U, host(f["x"]), b, dims, kappa) <= 1.1e-10, dims
