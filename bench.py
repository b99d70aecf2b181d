#!/usr/bin/env python3
"""Benchmark of the Wilson hopping term on GB300 (one JSON line on stdout).

Headline workload: the FP32 even-odd hopping term on a 32^3 x 64 lattice
(weak-field links U = exp(0.3 i H) stored with 12 reals, complex64 Gaussian
spinor, kappa = 0.1350, periodic x,y,z / antiperiodic t).  One step is 100
back-to-back applications alternating D_oe and D_eo (ping-pong fields).
Rates: 1320 flops per output site (Sec. 5 of the paper) and 576 compulsory
bytes per output site (spinor in 96 B + 8 links x 48 B + spinor out 96 B).

Also reported: the end-to-end rate through the C ABI with host buffers
(spinor copied in from pinned host memory and out again every step); the
FP64 CPU oracle on the host cores, and the timed kernel's first application
against the oracle's output (parity record); a CG time-to-solution
comparison on the 24^3 x 48 lattice (mixed F32/F16/BF16-inner vs plain FP64,
true residual 1e-10); the 12-RHS hop and solves; and the batch of 64 uneven
solves against the same problems solved one by one (mixed and plain FP64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0710_2442_gb300 import inputs, model  # noqa: E402

METRIC = "Dslash GFlop/s & HBM GB/s (% roofline); CG time-to-1e-10 mixed vs FP64"
FIRST_APPLICATION = [None]  # the library's first hop application of the timed workload (host copy)
ORACLE_OUTPUT = [None]      # the oracle's output for the same input (CPU leg)
DD_OUTPUT = [None]          # the t-decomposed hop's first application (host copy), same input
# GPU solutions kept (host copies) for the oracle's residual check in the CPU leg:
# a list of (record, key, [(gauge, b, x, dims, kappa), ...][, FP64 GPU solution to compare x with]);
# gauge and b may be callables that regenerate the field from its seed
SOLUTIONS = []
# DRAM bytes (read + write) per launch of the tuned 32^3 x 64 even-odd kernel, read from one
# ncu capture of that kernel (keyed by storage precision and link reals); a fixed figure, not
# measured by this run.
NCU_TRAFFIC = {("f32", 12): 581.6e6, ("f16", 12): 298.5e6, ("f64", 18): 1621.5e6}
TRAFFIC_SOURCE = "ncu capture of the tuned kernel (dram__bytes_read.sum + dram__bytes_write.sum), fixed figure"
WORKLOAD = "dslash_eo_f32_32^3x64"
L2_NOTE = ("inputs larger than L2: each application streams 403 MB of links plus 2 x 101 MB of spinors "
           "through the 126 MB L2")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-solver", action="store_true",
                    help="skip the solver, multi-RHS and batch blocks (CG time-to-solution comparisons)")
    ap.add_argument("--blocks", default="cg,multirhs,batch,dd",
                    help="blocks to run after the headline (comma list of cg, multirhs, batch, dd)")
    ap.add_argument("--cg-prec", default="f64,f16,bf16,f32",
                    help="inner precisions of the cg block's solves (comma list; f64 = plain FP64 CG)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--apps", type=int, default=None, help="applications per step (default 100)")
    ap.add_argument("--prec", choices=["f32", "f16", "bf16", "f64"], default="f32",
                    help="storage precision of spinors and links (the workload is f32)")
    ap.add_argument("--recon", type=int, choices=[12, 18], default=12,
                    help="reals stored per link (the workload is 12)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# distributed bookkeeping (independent replicas; timing only)
# ---------------------------------------------------------------------------
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_c2_fields():
    cfg = inputs.WORKLOADS[WORKLOAD]
    dims = cfg["dims"]
    U = inputs.gauge_field(dims, cfg["gauge"], eps=cfg["eps"], seed=cfg["gauge_seed"])
    Vh = inputs.volume(dims) // 2
    src = inputs.gaussian_spinor(Vh, seed=cfg["spinor_seed"]).astype(np.complex64).astype(np.complex128)
    return cfg, dims, U, src


def workload_config(args, cfg, dims, apps, ws):
    return {"workload": WORKLOAD if (args.prec, args.recon) == ("f32", 12)
            else WORKLOAD.replace("f32", f"{args.prec}-{args.recon}"),
            "dims": list(dims), "links": f"{args.prec} {args.recon}-real", "spinor": args.prec,
            "kappa": cfg["kappa"], "applications_per_step": apps, "sites_per_application": inputs.volume(dims) // 2,
            "l2": L2_NOTE, "parallelism": "replicas" if ws > 1 else "single"}


def run_ours(args, ws, rank, local, fields):
    import torch
    from paper_0710_2442_gb300 import build, wilson as w
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, dims, U, src = fields
    Vh = inputs.volume(dims) // 2
    apps = args.apps or cfg["applications"]
    L = w.lattice(dims)
    stream = torch.cuda.current_stream(dev)
    P = w.PREC[args.prec]
    # the device's measured FMA peaks (the ALU rooflines), before any timed region
    alu = {"f64_gflops": round(w.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F64, stream), 1),
           "f32_gflops": round(w.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F32, stream), 1),
           "f32x2_gflops": round(w.wilson_probe_fma_peak(w.WILSON_PROBE_FMA_F32X2, stream), 1),
           "how": "wilson_probe_fma_peak: 8 independent FMA chains per thread, 2048 threads per SM on every "
                  "SM, best of 3 CUDA-event-timed launches; 2 flops per FMA and lane"}
    g = w.Gauge(U, L, P, args.recon, stream)
    even = w.Spinor(L, w.WILSON_EVEN, P)
    odd = w.Spinor(L, w.WILSON_ODD, P)
    src_dev = torch.from_numpy(src).to(dev)
    even.load(src_dev, stream)
    # one application kept for the parity record (compared with the oracle's output in the
    # CPU leg); outside every timed region
    first = torch.empty_like(src_dev)
    w.wilson_dslash_h(odd, g, even, 0.0, w.WILSON_OP_HOP, stream)
    odd.store(first, stream)
    torch.cuda.synchronize(dev)
    FIRST_APPLICATION[0] = first.cpu().numpy()
    del first

    def step(e=even, o=odd):
        for k in range(apps):
            if k % 2 == 0:
                w.wilson_dslash_h(o, g, e, 0.0, w.WILSON_OP_HOP, stream)
            else:
                w.wilson_dslash_h(e, g, o, 0.0, w.WILSON_OP_HOP, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize(dev)
        start.record(stream)
        for _ in range(args.steps):
            step()
        stop.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
    ms = start.elapsed_time(stop)
    ms = max_over_ranks(ms, ws)
    clocks = clk.summary()
    launches = args.steps * apps
    t_launch = ms / 1e3 / launches
    flops = model.FLOPS_PER_SITE * Vh
    comp_bytes = model.compulsory_bytes_per_site(args.prec, args.recon, eo=True) * Vh
    gflops = flops * launches * ws / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    achieved = comp_bytes / t_launch / 1e9

    # end to end through the C ABI with host buffers: each step imports its input from pinned
    # host memory, applies the hop apps times and exports the result to pinned host memory.
    # Two field sets alternate; a step's export runs on a second stream (the library orders
    # that stream after its device-to-host copy), so it overlaps the next step's hops, and a
    # set is imported again only after its previous export has read it.
    host_in = torch.from_numpy(src).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    s_out = torch.cuda.Stream(dev)
    sets = [(even, odd), (w.Spinor(L, w.WILSON_EVEN, P), w.Spinor(L, w.WILSON_ODD, P))]
    e2e_steps = max(1, min(args.steps, 50))  # the timed steps of the device measurement

    def e2e_run(n):
        exported = [None, None]
        for k in range(n):
            e, o = sets[k % 2]
            if exported[k % 2] is not None:
                stream.wait_event(exported[k % 2])
            e.load(host_in, stream)
            step(e, o)
            done = torch.cuda.Event()
            done.record(stream)
            s_out.wait_event(done)
            (o if apps % 2 else e).store(host_out[k % 2], s_out)
            exported[k % 2] = torch.cuda.Event()
            exported[k % 2].record(s_out)

    e2e_run(2)
    torch.cuda.synchronize(dev)
    barrier(ws)
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    torch.cuda.synchronize(dev)
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": round(flops * apps * e2e_steps * ws / t_e2e / 1e9, 2), "unit": "GFlop/s",
           "h2d_bytes_per_step": int(host_in.numel() * 16), "d2h_bytes_per_step": int(host_out[0].numel() * 16),
           "steps": e2e_steps,
           "api": f"wilson_spinor_import(host) + {apps} x wilson_dslash_h + wilson_spinor_export(host) per step; "
                  "two field sets, each export on a second stream overlapping the next step's hops"}
    # the hop's memory-access pattern with the arithmetic taken out, outside every timed
    # region (overwrites odd with a checksum)
    access = access_record(comp_bytes, w.wilson_probe_hop_access(odd, g, even, 50, stream), t_launch, peak)
    del src_dev
    for h in (even, odd, g, *sets[1]):
        h.close()
    torch.cuda.synchronize(dev)

    line = {
        "metric": METRIC, "value": round(gflops, 2), "unit": "GFlop/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": workload_config(args, cfg, dims, apps, ws),
        "hbm_gbs": round(achieved * ws, 1),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": NCU_TRAFFIC.get((args.prec, args.recon)),
                     "traffic_source": TRAFFIC_SOURCE, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": comp_bytes, "launch_us": round(t_launch * 1e6, 2)},
    }
    if args.prec == "f64":
        # FP64 is bound by GB300's FP64 rate (FP64 pipe 91 % busy at 12 % DRAM
        # throughput): roofline against the FP64 FMA peak measured above.
        gf_launch = flops / t_launch / 1e9
        f64_peak = alu["f64_gflops"]
        line["roofline"] = {"bound": "alu", "achieved": round(gf_launch, 1), "peak": f64_peak,
                            "unit": "GFLOP/s", "frac": round(gf_launch / f64_peak, 4),
                            "traffic": NCU_TRAFFIC.get((args.prec, args.recon)), "traffic_source": TRAFFIC_SOURCE,
                            "peak_kind": "measured (wilson_probe_fma_peak, FP64 FMA)",
                            "launch_us": round(t_launch * 1e6, 2),
                            "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                    "frac": round(achieved / peak, 4)}}
    line.update({"clocks": clocks, "e2e": e2e, "gpu_launches": launches, "alu_peaks": alu,
                 "access_pattern": access})
    if rank == 0 and not args.no_solver:
        blocks = {b.strip() for b in args.blocks.split(",")}
        if "cg" in blocks:
            line["cg"] = run_solver_block(w, torch, dev, stream, args.cg_prec.split(","), peak)
        if "multirhs" in blocks:
            line["multirhs"] = run_multirhs_block(w, torch, dev, stream, fields)
        if "dd" in blocks:
            line["dd"] = run_dd_block(w, torch, dev, stream, fields, line["roofline"]["launch_us"])
        if "batch" in blocks:
            line["batch"] = run_batch_block(w, torch, dev, stream)
    return line


def access_record(comp_bytes, t_access, t_hop, hbm_peak):
    """The paper's benchmark of Eq. 3's memory-access pattern (Sec. 5, after
    Table 1: within 20 % of the model's T_mem on the Cell) on this GPU:
    wilson_probe_hop_access makes the hop's DRAM accesses with trivial
    arithmetic.  T_mem here is the compulsory bytes at the measured copy
    bandwidth; hop_over_access is how much the arithmetic adds to the hop."""
    t_mem = comp_bytes / (hbm_peak * 1e9)
    return {"us": round(t_access * 1e6, 2), "frac": round(comp_bytes / t_access / 1e9 / hbm_peak, 4),
            "t_mem_us": round(t_mem * 1e6, 2), "access_over_t_mem": round(t_access / t_mem, 3),
            "hop_us": round(t_hop * 1e6, 2), "hop_over_access": round(t_hop / t_access, 3),
            "how": "wilson_probe_hop_access: the hop's loads and stores, XOR/add of the loaded words, best "
                   "of block sizes 64/128/256 x four register budgets, mean of back-to-back CUDA-event-timed "
                   "launches"}


def run_solver_block(w, torch, dev, stream, precs, hbm_peak):
    cfg = inputs.WORKLOADS["cg_mixed_24^3x48"]
    dims = cfg["dims"]
    U = inputs.gauge_field(dims, cfg["gauge"], eps=cfg["eps"], seed=cfg["gauge_seed"])
    b = inputs.gaussian_spinor(dims, seed=cfg["spinor_seed"])
    Ud = torch.from_numpy(U).to(dev)
    bd = torch.from_numpy(b).to(dev)
    L = w.lattice(dims)
    Vh = inputs.volume(dims) // 2
    res = {"workload": "cg_mixed_24^3x48", "kappa": cfg["kappa"], "tol": cfg["tol"]}
    sols = {}
    for name, prec in (("f64", w.WILSON_F64), ("f16", w.WILSON_F16), ("bf16", w.WILSON_BF16),
                       ("f32", w.WILSON_F32)):
        if name not in precs:
            continue
        x = torch.zeros_like(bd)
        p = w.solver_defaults(prec)
        # the first solve tunes the launch configurations; time the second
        w.wilson_cg_solve(x, Ud, bd, L, cfg["kappa"], p, stream, check=False)
        x.zero_()
        st = w.wilson_cg_solve(x, Ud, bd, L, cfg["kappa"], p, stream, check=False)
        rec = {"seconds": round(st["seconds"], 4), "inner_iters": st["inner_iters"],
               "outer_iters": st["outer_iters"], "hops": st["hop_applications"],
               "true_rel_resid": st["true_rel_resid"], "rc": st["rc"]}
        if st["inner_iters"] > 0 and st["inner_seconds"] > 0:
            # roofline of one inner CG iteration (six launches): algorithmic bytes over the
            # device time of the inner iterations, measured by the solver with CUDA events
            recon = 18 if name == "f64" else 12
            byts = model.cg_inner_bytes_per_site(name, recon) * Vh
            t_it = st["inner_seconds"] / st["inner_iters"]
            rec["roofline_inner_iteration"] = {
                "bound": "alu" if name == "f64" else "hbm", "bytes_per_site": model.cg_inner_bytes_per_site(name, recon),
                "algorithmic_bytes": byts, "us_per_iteration": round(t_it * 1e6, 2),
                "achieved_GBs": round(byts / t_it / 1e9, 1), "peak_GBs": hbm_peak,
                "frac": round(byts / t_it / 1e9 / hbm_peak, 4),
                "inner_share_of_solve": round(st["inner_seconds"] / st["seconds"], 3)}
        res[name] = rec
        sols[name] = x.cpu().numpy()
    if res.get("f64", {}).get("rc") == 0 and res.get("f16", {}).get("rc") == 0:
        res["speedup_f16_vs_f64"] = round(res["f64"]["seconds"] / res["f16"]["seconds"], 3)
    for name, xs in sols.items():
        SOLUTIONS.append((res[name], "oracle", [(U, b, xs, dims, cfg["kappa"])],
                          sols.get("f64") if name != "f64" else None))
    return res


def run_multirhs_block(w, torch, dev, stream, fields, nrhs=12):
    """12 right-hand sides sharing the 32^3 x 64 F32 12-real links: the
    multi-RHS hop against the single-RHS one, and the lockstep 12-RHS CG
    (point sources, F16 inner) against 12 sequential solves and against
    one block CG over the 12 right-hand sides."""
    cfg, dims, U, src = fields
    Vh = inputs.volume(dims) // 2
    L = w.lattice(dims)
    kappa = inputs.WORKLOADS["multirhs12_32^3x64"]["kappa"]
    hbm_peak, _ = measured_peaks()
    out = {"workload": "multirhs12_32^3x64", "links": "the headline workload's field, 12-real"}
    # the hop with 1 and 12 right-hand sides, F32 storage (keys hop_nrhs*) and the F16 storage
    # of the inner solver (keys f16_hop_nrhs*); frac: compulsory bytes against measured HBM
    for pname, prec, prefix in (("f32", w.WILSON_F32, ""), ("f16", w.WILSON_F16, "f16_")):
        g = w.Gauge(U, L, prec, 12, stream)
        for n in (1, nrhs):
            a = w.Spinor(L, w.WILSON_EVEN, prec, n)
            b = w.Spinor(L, w.WILSON_ODD, prec, n)
            a.load(torch.from_numpy(inputs.gaussian_spinor(Vh, seed=31, nrhs=n)).to(dev), stream)
            for _ in range(3):
                w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP, stream)
                w.wilson_dslash_h(a, g, b, 0.0, w.WILSON_OP_HOP, stream)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            e0.record(stream)
            for _ in range(reps // 2):
                w.wilson_dslash_h(b, g, a, 0.0, w.WILSON_OP_HOP, stream)
                w.wilson_dslash_h(a, g, b, 0.0, w.WILSON_OP_HOP, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3 / reps
            bps = model.compulsory_bytes_per_site(pname, 12, eo=True, nrhs=n)
            byts = bps * Vh
            out[f"{prefix}hop_nrhs{n}"] = {
                "us_per_application": round(t * 1e6, 2), "us_per_rhs": round(t * 1e6 / n, 2),
                "GBs_compulsory": round(byts / t / 1e9, 1), "bytes_per_site_rhs": round(bps / n, 1),
                "frac": round(byts / t / 1e9 / hbm_peak, 4),
                "TFlops": round(model.FLOPS_PER_SITE * Vh * n / t / 1e12, 3)}
            if n == 1:  # the same accesses without the arithmetic (overwrites b)
                out[f"{prefix}hop_nrhs1"]["access_pattern"] = access_record(
                    byts, w.wilson_probe_hop_access(b, g, a, reps, stream), t, hbm_peak)
            a.close()
            b.close()
        g.close()
        out[f"{prefix}rhs_speedup_per_rhs"] = round(
            out[f"{prefix}hop_nrhs1"]["us_per_rhs"] / out[f"{prefix}hop_nrhs{nrhs}"]["us_per_rhs"], 3)
    # lockstep 12-RHS CG vs 12 sequential solves (F16 inner, point sources at the origin)
    Ud = torch.from_numpy(U).to(dev)
    bsrc = torch.from_numpy(inputs.point_sources(dims, site=0)).to(dev)
    p = w.solver_defaults(w.WILSON_F16)
    x = torch.zeros_like(bsrc)
    w.wilson_cg_solve_multi(x, Ud, bsrc, nrhs, L, kappa, p, stream, check=False)  # tunes
    x.zero_()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc, st = w.wilson_cg_solve_multi(x, Ud, bsrc, nrhs, L, kappa, p, stream, check=False)
    torch.cuda.synchronize(dev)
    t_multi = time.perf_counter() - t0
    x_lock = x.cpu().numpy()  # for the oracle's check in the CPU leg
    xw = torch.zeros_like(bsrc[0])
    w.wilson_cg_solve(xw, Ud, bsrc[0], L, kappa, p, stream, check=False)  # tunes the single-RHS launches
    del xw
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    seq = []
    for k in range(nrhs):
        xk = torch.zeros_like(bsrc[k])
        seq.append(w.wilson_cg_solve(xk, Ud, bsrc[k], L, kappa, p, stream, check=False))
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    # block CG over the 12 right-hand sides (same sources, inner precision and target)
    pb = w.solver_defaults(w.WILSON_F16)
    pb.block_cg = 1
    x.zero_()
    w.wilson_cg_solve_multi(x, Ud, bsrc, nrhs, L, kappa, pb, stream, check=False)
    x.zero_()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rcb, stb = w.wilson_cg_solve_multi(x, Ud, bsrc, nrhs, L, kappa, pb, stream, check=False)
    torch.cuda.synchronize(dev)
    t_block = time.perf_counter() - t0
    out["cg"] = {"kappa": kappa, "inner": "f16", "rc": rc, "seconds_lockstep": round(t_multi, 4),
                 "seconds_sequential": round(t_seq, 4), "speedup": round(t_seq / t_multi, 3),
                 "max_true_rel_resid": max(s["true_rel_resid"] for s in st),
                 "inner_iters": [s["inner_iters"] for s in st],
                 "block_cg": {"rc": rcb, "seconds": round(t_block, 4),
                              "inner_iters": max(s["inner_iters"] for s in stb),
                              "max_true_rel_resid": max(s["true_rel_resid"] for s in stb)}}
    b_host = bsrc.cpu().numpy()
    SOLUTIONS.append((out["cg"]["block_cg"], "oracle",
                      [(U, b_host[k], x[k].cpu().numpy(), dims, kappa) for k in range(nrhs)]))
    SOLUTIONS.append((out["cg"], "oracle", [(U, b_host[k], x_lock[k], dims, kappa) for k in range(nrhs)]))
    del Ud, bsrc, x
    torch.cuda.empty_cache()
    return out


def run_dd_block(w, torch, dev, stream, fields, single_us, n=2):
    """The headline hop on the lattice split along t into n sub-lattices on
    this GPU: wilson_dd_pack on each, the loopback exchange of the face
    buffers (device copies), wilson_dd_hop on each; timed per application
    against the single-lattice hop, with the face bytes each application
    moves (12 reals per face site, the paper's T_ext data)."""
    from paper_0710_2442_gb300.dd import TSplit, exchange_loopback
    cfg, dims, U, src = fields
    sp = TSplit(dims, n)
    L = w.lattice(sp.local_dims)
    P = w.WILSON_F32
    hb = w.wilson_dd_halo_bytes(L, P)
    gauges = [w.Gauge(u, L, P, 12, stream) for u in sp.split_gauge(U)]
    ins = [w.Spinor(L, w.WILSON_EVEN, P) for _ in range(n)]
    outs = [w.Spinor(L, w.WILSON_ODD, P) for _ in range(n)]
    for s_, part in zip(ins, sp.split_half(src)):
        s_.load(torch.from_numpy(np.ascontiguousarray(part)).to(dev), stream)
    buf = lambda: [torch.empty(hb, dtype=torch.uint8, device=dev) for _ in range(n)]
    send_prev, send_next, recv_next, recv_prev = buf(), buf(), buf(), buf()

    def pack():
        for r in range(n):
            w.wilson_dd_pack(send_prev[r], send_next[r], gauges[r], ins[r], 0, stream)

    def hop():
        for r in range(n):
            w.wilson_dd_hop(outs[r], gauges[r], ins[r], recv_next[r], recv_prev[r], 0, sp.first(r), sp.last(r),
                            w.WILSON_DD_ALL, stream)

    def apply():
        pack()
        exchange_loopback(sp, send_prev, send_next, recv_next, recv_prev)
        hop()

    side = torch.cuda.Stream(dev)
    packed, moved = torch.cuda.Event(), torch.cuda.Event()

    def apply_overlapped():
        # the face copies on a second stream while the interior t-slices are applied
        pack()
        packed.record(stream)
        side.wait_event(packed)
        with torch.cuda.stream(side):
            exchange_loopback(sp, send_prev, send_next, recv_next, recv_prev)
        moved.record(side)
        for r in range(n):
            w.wilson_dd_hop(outs[r], gauges[r], ins[r], None, None, 0, sp.first(r), sp.last(r),
                            w.WILSON_DD_INTERIOR, stream)
        stream.wait_event(moved)
        for r in range(n):
            w.wilson_dd_hop(outs[r], gauges[r], ins[r], recv_next[r], recv_prev[r], 0, sp.first(r), sp.last(r),
                            w.WILSON_DD_FACES, stream)

    apply()
    parts = []
    for o in outs:
        t = torch.empty((sp.Lr * sp.Vs // 2, 4, 3), dtype=torch.complex128, device=dev)
        o.store(t, stream)
        parts.append(t.cpu().numpy())
    DD_OUTPUT[0] = sp.gather_half(parts)
    reps = 20
    res = {}
    for name, fn in (("pack_exchange_hop", apply), ("overlapped", apply_overlapped), ("hop_only", hop),
                     ("pack_only", pack)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name] = e0.elapsed_time(e1) / reps * 1e3
    Vh = inputs.volume(dims) // 2
    peak, _ = measured_peaks()
    byts = model.compulsory_bytes_per_site("f32", 12, eo=True) * Vh
    out = {"workload": "dslash_eo_f32_32^3x64 split along t", "subdomains": n, "local_dims": list(sp.local_dims),
           "exchange": "loopback device copies on one GPU",
           "face_bytes_per_application": 2 * n * 48 * sp.Vs // 2,
           "us_per_application": round(res["overlapped"], 2),
           "us_serial_pack_exchange_hop": round(res["pack_exchange_hop"], 2),
           "overlap": "face copies on a second stream during the interior t-slices' hop",
           "us_hops_only": round(res["hop_only"], 2), "us_pack_only": round(res["pack_only"], 2),
           "single_lattice_us": single_us,
           "hop_frac_of_hbm": round(byts / (res["hop_only"] * 1e-6) / 1e9 / peak, 4)}
    for h in gauges + ins + outs:
        h.close()
    return out


def run_batch_block(w, torch, dev, stream):
    """64 uneven solves in one graph launch against the same 64 solved one by one, with the
    same mixed-precision solver and with plain FP64 CG."""
    probs = inputs.batch_problems()
    fields = []
    for p in probs:
        U = inputs.gauge_field(p["dims"], "weak", eps=p["eps"], seed=p["gauge_seed"])
        b = inputs.gaussian_spinor(p["dims"], seed=p["spinor_seed"])
        fields.append(dict(L=w.lattice(p["dims"]), kappa=p["kappa"], gauge=torch.from_numpy(U).to(dev),
                           b=torch.from_numpy(b).to(dev), x=torch.zeros(b.shape, dtype=torch.complex128, device=dev)))
    prm = w.solver_defaults(w.WILSON_F16)
    w.wilson_batch_solve(fields, prm, stream, check=False)  # tunes the batched kernels
    for f in fields:
        f["x"].zero_()
    torch.cuda.synchronize(dev)
    rc, st, info = w.wilson_batch_solve(fields, prm, stream, check=False)
    lat = sorted(s["seconds"] for s in st)
    batch_x = [f["x"].cpu().numpy() for f in fields]  # for the oracle's check in the CPU leg
    sites = sum(inputs.volume(p["dims"]) for p in probs)
    # one untimed solve per lattice size tunes the single-solve launches first
    seen = set()
    for p, f in zip(probs, fields):
        if tuple(p["dims"]) in seen:
            continue
        seen.add(tuple(p["dims"]))
        xw = torch.zeros_like(f["x"])
        w.wilson_cg_solve(xw, f["gauge"], f["b"], f["L"], f["kappa"], prm, stream, check=False)
        del xw
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for f in fields:
        f["x"].zero_()
        w.wilson_cg_solve(f["x"], f["gauge"], f["b"], f["L"], f["kappa"], prm, stream, check=False)
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    # the same 64 problems with plain FP64 CG, one by one (one untimed solve per size tunes first)
    p64 = w.solver_defaults(w.WILSON_F64)
    seen = set()
    for p, f in zip(probs, fields):
        if tuple(p["dims"]) in seen:
            continue
        seen.add(tuple(p["dims"]))
        xw = torch.zeros_like(f["x"])
        w.wilson_cg_solve(xw, f["gauge"], f["b"], f["L"], f["kappa"], p64, stream, check=False)
        del xw
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc64 = 0
    for f in fields:
        f["x"].zero_()
        s64 = w.wilson_cg_solve(f["x"], f["gauge"], f["b"], f["L"], f["kappa"], p64, stream, check=False)
        rc64 = rc64 or s64["rc"]
    torch.cuda.synchronize(dev)
    t_seq64 = time.perf_counter() - t0
    q = lambda a, f: a[min(len(a) - 1, int(round(f * (len(a) - 1))))]
    by_size, iters = {}, {}
    for p, s_ in zip(probs, st):
        key = "x".join(map(str, p["dims"]))
        by_size.setdefault(key, []).append(s_["seconds"])
        iters[key] = iters.get(key, 0) + s_["inner_iters"]
    by_size = {k: {"n": len(v), "median_s": round(sorted(v)[len(v) // 2], 4), "max_s": round(max(v), 4),
                   "inner_iters": iters[k]}
               for k, v in by_size.items()}
    out = {"workload": "batch64_uneven", "problems": len(probs), "sites": sites, "inner": "f16", "rc": rc,
           "device_seconds": round(info["device_seconds"], 4), "call_seconds": round(info["seconds"], 4),
           "solves_per_s": round(len(probs) / info["device_seconds"], 1),
           "latency_p50_s": round(q(lat, 0.5), 4), "latency_p99_s": round(q(lat, 0.99), 4),
           "loop_iterations": info["iterations"], "graph_launches": info["graph_launches"],
           "device_loop": info["device_loop"], "timed_out": info["timed_out"],
           "max_true_rel_resid": max(s["true_rel_resid"] for s in st),
           "sequential_seconds": round(t_seq, 4), "speedup_vs_sequential": round(t_seq / info["device_seconds"], 3),
           "fp64_sequential_seconds": round(t_seq64, 4), "fp64_sequential_rc": rc64,
           "speedup_vs_fp64_sequential": round(t_seq64 / info["device_seconds"], 3),
           "latency_by_lattice": by_size}
    # the oracle regenerates each problem's links from its seed in the CPU leg
    SOLUTIONS.append((out, "oracle", [(
        (lambda p=p: inputs.gauge_field(p["dims"], "weak", eps=p["eps"], seed=p["gauge_seed"])),
        (lambda p=p: inputs.gaussian_spinor(p["dims"], seed=p["spinor_seed"])),
        xk, p["dims"], p["kappa"]) for p, xk in zip(probs, batch_x)]))
    del fields
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# the FP64 CPU oracle (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(dims, U, src, reps=1):
    """GFlop/s, threads and seconds of the FP64 oracle's even-odd hop (out
    parity 1) on the full lattice; its last output is kept in ORACLE_OUTPUT."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    Vh = inputs.volume(dims) // 2
    t0 = time.perf_counter()
    for _ in range(reps):
        ORACLE_OUTPUT[0] = oracle.dslash_eo(U, src, dims, 1)
    t = time.perf_counter() - t0
    return model.FLOPS_PER_SITE * Vh * reps / t / 1e9, cores, t


def parity_record(prec, got, want):
    """The first timed-kernel application against the FP64 oracle, whole lattice."""
    tol = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3}[prec]
    d = (got - want).ravel()
    rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
    return {"what": "one even-odd hop application on the full lattice against the FP64 oracle",
            "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(want)),
            "max_component_error_over_rms": float(np.max(np.maximum(np.abs(d.real), np.abs(d.imag))) / rms),
            "tolerance_rel_l2": tol, "sites": int(want.shape[0])}


def oracle_cg_per_iteration(dims, U, b, kappa, iters=10):
    """Seconds per CGNR iteration of the FP64 oracle (iters timed; the set-up
    and the final residual are included, about 3 of the 4 x iters hops)."""
    import oracle
    t0 = time.perf_counter()
    _, info = oracle.cg_solve(U, b, dims, kappa, maxiter=iters)
    return (time.perf_counter() - t0) / max(info["iterations"], 1)


def oracle_solver_baselines(line):
    """CPU baselines of the solver workloads, extrapolated from a bounded
    sample: the oracle's seconds per CG iteration times the iteration count
    of the GPU solve of the same workload."""
    import oracle
    cfg = inputs.WORKLOADS["cg_mixed_24^3x48"]
    dims = cfg["dims"]
    U = inputs.gauge_field(dims, cfg["gauge"], eps=cfg["eps"], seed=cfg["gauge_seed"])
    b = inputs.gaussian_spinor(dims, seed=cfg["spinor_seed"])
    per_it = {"24x24x24x48": oracle_cg_per_iteration(dims, U, b, cfg["kappa"])}
    out = {}
    gpu = line.get("cg", {}).get("f64", {})
    if gpu.get("inner_iters"):
        out["cg_24^3x48_fp64"] = {
            "seconds_per_iteration": round(per_it["24x24x24x48"], 4), "iterations": gpu["inner_iters"],
            "seconds_extrapolated": round(per_it["24x24x24x48"] * gpu["inner_iters"], 2),
            "gpu_fp64_seconds": gpu["seconds"],
            "gpu_f16_mixed_seconds": line["cg"].get("f16", {}).get("seconds")}
    batch = line.get("batch", {}).get("latency_by_lattice")
    if batch:
        total = 0.0
        for key, rec in batch.items():
            d = tuple(int(v) for v in key.split("x"))
            if key not in per_it:
                Us = inputs.gauge_field(d, "weak", eps=0.3, seed=inputs.SEED_BASE + 90)
                bs = inputs.gaussian_spinor(d, seed=inputs.SEED_BASE + 91)
                per_it[key] = oracle_cg_per_iteration(d, Us, bs, 0.13)
            total += per_it[key] * rec["inner_iters"]
        out["batch64_uneven"] = {"seconds_extrapolated": round(total, 2),
                                 "gpu_device_seconds": line["batch"]["device_seconds"],
                                 "sample": "10 oracle CG iterations per lattice size, times the GPU batch's "
                                           "iterations of that size"}
    return out


def oracle_solution_checks():
    """The oracle's verdict on every solver result the bench reports: each
    GPU solution's true residual |b - M x| / |b| recomputed with the FP64
    CPU oracle's Wilson matrix, and for the 24^3 x 48 solves the relative
    difference from the plain FP64 GPU solution.  Stored into the records."""
    import oracle
    for entry in SOLUTIONS:
        rec, key, probs = entry[0], entry[1], entry[2]
        xref = entry[3] if len(entry) > 3 else None
        t0 = time.perf_counter()
        res = []
        for U, b, x, dims, kappa in probs:
            U = U() if callable(U) else U
            b = b() if callable(b) else b
            r = b - oracle.wilson_m(U, x, dims, kappa)
            res.append(float(np.linalg.norm(r) / np.linalg.norm(b)))
        out = {"true_rel_resid_max": max(res), "problems": len(res),
               "how": "|b - M x| / |b| with the FP64 CPU oracle's M on the GPU solution"}
        if len(res) > 1:
            out["true_rel_resid_median"] = float(np.median(res))
        if xref is not None:
            x = probs[0][2]
            out["rel_diff_vs_fp64_gpu_solution"] = float(np.linalg.norm(x - xref) / np.linalg.norm(xref))
        out["seconds"] = round(time.perf_counter() - t0, 2)
        rec[key] = out
    SOLUTIONS.clear()


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    cfg, dims, U, src = make_c2_fields()
    oracle_sample(dims, U, src)  # build + first touch
    vals = []
    for _ in range(args.warmup):
        oracle_sample(dims, U, src)
    t_all = 0.0
    for _ in range(args.steps):
        v, cores, t = oracle_sample(dims, U, src)
        vals.append(v)
        t_all += t
    Vh = inputs.volume(dims) // 2
    value = model.FLOPS_PER_SITE * Vh * args.steps / t_all / 1e9
    sample = (f"one FP64 application of the even-odd hopping term on the full 32^3x64 lattice per step "
              f"(the workload's step is 100 F32 applications)")
    return {"metric": METRIC, "value": round(value, 4), "unit": "GFlop/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_all / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args, cfg, dims, args.apps or cfg["applications"], ws),
            "cpu_baseline": {"value": round(value, 4), "unit": "GFlop/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    fields = make_c2_fields()
    line = run_ours(args, ws, rank, local, fields)
    if rank == 0 and ws == 1 and not args.no_cpu:
        cfg, dims, U, src = fields
        import oracle
        v, cores, t = oracle_sample(dims, U, src)
        oracle.set_num_threads(1)
        v1, _, t1 = oracle_sample(dims, U, src)
        oracle.set_num_threads(cores)
        line["cpu_baseline"] = {"value": round(v, 4), "unit": "GFlop/s", "cores": cores, "kind": "oracle",
                                "sample": f"one FP64 even-odd application on the full 32^3x64 lattice "
                                          f"({t:.1f} s of CPU time)",
                                "value_1core": round(v1, 4)}
        if FIRST_APPLICATION[0] is not None and ORACLE_OUTPUT[0] is not None:
            line["parity"] = parity_record(args.prec, FIRST_APPLICATION[0], ORACLE_OUTPUT[0])
        if DD_OUTPUT[0] is not None and ORACLE_OUTPUT[0] is not None and "dd" in line:
            line["dd"]["parity"] = parity_record("f32", DD_OUTPUT[0], ORACLE_OUTPUT[0])
        if not args.no_solver:
            oracle_solution_checks()
            line["cpu_baseline"]["solvers"] = oracle_solver_baselines(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
