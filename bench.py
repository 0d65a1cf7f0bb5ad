"""Benchmark: AMG setup + FCG solve to 1e-8 relative residual on one GB300 per rank.

A step is one pass of the whole hot path over the workload: amg_setup (weights, Suitor
matching, aggregation, prolongator, Galerkin products, level after level) followed by
amg_pcg_solve (FCG with the l1-Jacobi V-cycle) from x = 0, then amg_free.

Default workload: 3D linear elasticity, trilinear Q1 hexahedra on 64^3 nodes, face x = 0
clamped (n = 774,144, nnz = 60,756,300 with the assembled pattern's stored zeros), E = 1,
nu = 0.3, v = the three rigid translations with seeded U[0.5, 1.5] weights, 2 matching
sweeps per level (aggregates of 4), coarse n <= 1000, body force b ~ U[-1, 1] (seed 0);
FP64 setup, FP32 V-cycle inside the FP64 FCG, rtol 1e-8.  The all-FP64 run of the same
workload is timed beside it (`variants`).

Prints ONE JSON line (rank 0).  `value` is milliseconds per step (setup + solve) with the
inputs already resident in HBM; `e2e` times the same C-ABI calls made on pinned host
arrays (amg_setup reads the CSR and v from host memory, amg_pcg_solve reads b and the
initial guess and writes x back, every transfer inside the timed region).  `--impl reference` times the CPU FP64 oracle (the reference arm).
Under torchrun every rank runs an independent replica (the solver does not shard).
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_1810_04221_gb300 import problems as P  # noqa: E402

METRIC = "AMG setup ms + PCG solve ms to 1e-8 rel. residual"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.txt")  # JSON text
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e data-sheet rate, reported beside the measured copy peak


def workload(name: str):
    """(description, (rp, ci, val), v, b, x* or None, sweeps, coarse_max, fp32, extra params)."""
    xs = None
    if name == "poisson3d_128":
        mat = P.poisson3d(128)
        n = len(mat[0]) - 1
        v = np.ones(n)
        sweeps, cmax, fp32 = 3, 1000, False
        desc = "3D Poisson 7-point 128^3, v=1, 3 sweeps/level, coarse<=1000, FP64 setup+FCG/V-cycle"
    elif name == "poisson2d_64":
        mat = P.poisson2d(64)
        n = len(mat[0]) - 1
        v = np.ones(n)
        sweeps, cmax, fp32 = 2, 40, False
        desc = "2D Poisson 5-point 64^2, v=1, 2 sweeps/level, coarse<=40, FP64"
    elif name in ("lognormal_160", "lognormal_80"):
        m = int(name.split("_")[1])
        mat = P.lognormal_diffusion(m, sigma=2.0, seed=0)
        n = len(mat[0]) - 1
        v = np.ones(n)
        sweeps, cmax, fp32 = 3, 1000, True
        desc = (f"3D FV diffusion {m}^3, log-kappa N(0,4), 3 sweeps/level, coarse<=1000, stall ratio 1.2, "
                "FP32 V-cycle in FP64 FCG")
    elif name in ("elasticity_64", "elasticity_48", "elasticity_32"):
        m = int(name.split("_")[1])
        mat = P.elasticity_q1(m)
        n = len(mat[0]) - 1
        v = P.smooth_vector_components(n, seed=0)
        sweeps, cmax, fp32 = 2, 1000, True
        desc = (f"3D Q1 elasticity {m}^3 nodes, x=0 clamped, E=1, nu=0.3, 2 sweeps/level, coarse<=1000, "
                "b ~ U[-1,1], FP32 V-cycle in FP64 FCG")
        b = np.random.default_rng(0).uniform(-1.0, 1.0, size=n)
    else:
        raise SystemExit(f"unknown workload {name}")
    extra = {"stall_ratio": 1.2} if name.startswith("lognormal") else {}
    if not name.startswith("elasticity"):
        xs, b = P.manufactured_rhs(*mat, seed=0)
    return desc, mat, v, b, xs, sweeps, cmax, fp32, extra


# The CPU oracle's timed sample of each workload: the same problem family and parameters on
# a coarser grid (about 10 s of single-threaded work), its time scaled to the full size by
# the ratio of stored entries.  The full-size iteration count is higher than the sample's,
# so the scaled figure underestimates the oracle's full-size time.
CPU_SAMPLE = {"poisson3d_128": "poisson3d_128", "poisson2d_64": "poisson2d_64",
              "lognormal_160": "lognormal_80", "elasticity_64": "elasticity_32", "elasticity_48": "elasticity_32"}
# elasticity_48 (n = 324,864, 25.2M entries, the 3x3-block copy 213 MB > L2) is the
# profiling-size case of the elasticity family
WORKLOADS = ["elasticity_64", "poisson3d_128", "lognormal_160", "poisson2d_64", "elasticity_48"]


def bench_config(name: str, n: int, nnz: int, desc: str, sweeps: int, cmax: int, rtol: float, fp32: bool,
                 world: int) -> dict:
    """The `config` object of both arms' JSON lines."""
    return {"workload": name, "desc": desc, "n": n, "nnz": nnz, "sweeps_per_level": sweeps,
            "coarse_max": cmax, "rtol": rtol, "vcycle_fp32": bool(fp32),
            "l2": "inputs larger than L2 (CSR %.0f MB > 129 MB), no flush" % ((12 * nnz + 4 * n) / 1e6),
            "parallelism": f"replicas{world}"}


# --------------------------------------------------------------------- helpers ----

def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return FALLBACK_HBM_GBS, "fallback"


def _traffic_for(kernel_class: str, workload: str | None):
    """DRAM bytes per launch of a kernel class on a workload, from a committed ncu summary
    (the file maps workload -> class -> capture), or None if absent or stale."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        e = d[workload][kernel_class]
        src = os.path.join(ROOT, e["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if sha != e["source_sha256"]:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:  # noqa: BLE001
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        if self.gpu < 0:
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, f[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:  # noqa: BLE001
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, dist, device=None) -> float:
    """The largest `value` over all ranks (the job time of replicas); identity without dist."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- CUDA arm ----

def run_cuda(args, rank, world, dist):
    import torch
    from paper_1810_04221_gb300 import binding as B
    from paper_1810_04221_gb300 import build as cuda_build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    if dist is not None:
        dist.barrier()
    B.load()
    desc, mat, v, b, xs, sweeps, cmax, fp32, extra = workload(args.workload)
    if args.fp32 is not None:
        fp32 = bool(args.fp32)
    rp, ci, val = mat
    n, nnz = len(rp) - 1, len(ci)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    d_rp, d_ci, d_val, d_v, d_b = dev(rp), dev(ci), dev(val), dev(v), dev(b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    extra = dict(extra, block3=args.block3)

    def params(trace=0, filt=""):
        return B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, vcycle_fp32=int(fp32), trace=trace,
                                    trace_filter=filt, check_input=0, **extra)

    def step(prm, evs=None):
        if evs:
            evs[0].record(stream)
        h = B.amg_setup(d_rp, d_ci, d_val, d_v, prm)
        if evs:
            evs[1].record(stream)
        x.zero_()
        st, info = B.amg_pcg_solve(h, d_b, x, rtol=args.rtol, itmax=args.itmax)
        if evs:
            evs[2].record(stream)
        return h, st, info

    # warm-up; the last one traces every kernel class (per-class roofline, dominant class)
    dominant, trace_all, level_sizes = None, [], []
    nwarm = max(args.warmup, 1)
    for w in range(nwarm):
        h, st, info = step(params(trace=1 if w == nwarm - 1 else 0))
        if w == nwarm - 1:
            trace_all = B.amg_trace(h)
            if trace_all:
                dominant = max(trace_all, key=lambda e: e["total_ms"])["name"]
            level_sizes = [list(B.amg_level_info(h, k)[:2]) for k in range(B.amg_num_levels(h))]
        h.free()
    torch.cuda.synchronize()

    # timed region: K steps, device events on the launching stream; the dominant class is
    # traced (an event pair around each of its launches) in the first timed step only: the
    # event nodes cost ~0.6 ms per FP64 solve (they also end the programmatic-dependent-launch
    # overlap around the traced kernel), which would otherwise weigh on every step's time
    clocks = Clocks(local) if not args.profile else Clocks(-1)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    traces, infos, statuses = [], [], []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = B.amg_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        h, st, info = step(params(trace=1 if k == 0 else 0, filt=dominant or ""), evs[k])
        if k == 0:
            traces.append(B.amg_trace(h))
        infos.append(info)
        statuses.append(st)
        h.free()
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = B.amg_launch_count() - l0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    setup_ms = [e[0].elapsed_time(e[1]) for e in evs]
    solve_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = max_over_ranks(total_ms, dist, device="cuda")
    ms_per_step = total_ms / args.steps
    x_main = x.cpu().numpy()
    relerr = lambda a, ref: None if ref is None else float(np.linalg.norm(a - ref) / np.linalg.norm(ref))  # noqa: E731
    err = relerr(x_main, xs)

    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": round(ms_per_step, 3), "dominant": dominant}))
        return

    # e2e through the C ABI with host buffers (pinned): amg_setup reads the CSR and v from
    # host memory, amg_pcg_solve reads b and the zero initial guess and writes x back, all
    # inside the timed region (the library moves page-locked arrays with its own copy kernel)
    h_rp, h_ci, h_val, h_v, h_b = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (rp, ci, val, v, b))
    h_x = torch.empty(n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_rp, h_ci, h_val, h_v, h_b, h_x))
    d2h = h_x.numel() * h_x.element_size()

    def e2e_step():
        hh = B.amg_setup(h_rp, h_ci, h_val, h_v, params())
        h_x.zero_()
        B.amg_pcg_solve(hh, h_b, h_x, rtol=args.rtol, itmax=args.itmax)
        torch.cuda.current_stream().synchronize()
        hh.free()

    for _ in range(2):
        e2e_step()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        es[k].record(stream)
        e2e_step()
    es[args.steps].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_steps = [round(es[k].elapsed_time(es[k + 1]), 3) for k in range(args.steps)]
    # the host -> device copies of one step alone (what e2e adds to the device-resident
    # step), done the way the library does them (cwm_copy); best of three
    g_copy = [torch.empty_like(t, device="cuda") for t in (h_rp, h_ci, h_val, h_v, h_b, h_x)]
    h2d_times = []
    for _ in range(3):
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for dst, src in zip(g_copy, (h_rp, h_ci, h_val, h_v, h_b, h_x)):
            B.cwm_copy(dst, src)
        c1.record(stream)
        torch.cuda.synchronize()
        h2d_times.append(c0.elapsed_time(c1))
    h2d_ms = min(h2d_times)
    del g_copy

    # roofline of the dominant kernel class over the timed region
    peak, peak_kind = _peaks()
    roof = None
    if dominant:
        ms = sum(e["total_ms"] for t in traces for e in t if e["name"] == dominant)
        byt = sum(e["bytes"] for t in traces for e in t if e["name"] == dominant)
        nl = sum(e["launches"] for t in traces for e in t if e["name"] == dominant)
        if ms > 0 and nl > 0:
            ach = byt / (ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": dominant, "achieved": round(ach, 1), "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": round(ach / peak, 4),
                    "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": round(ach / NOMINAL_HBM_GBS, 4),
                    "traffic": _traffic_for(dominant, args.workload), "launches": nl,
                    "bytes_per_launch": byt / nl, "avg_launch_us": ms / nl * 1e3}
            roof["classes"] = class_rooflines(trace_all, peak, args.workload)
            # the FP64-issue-bound classes against the FP64 rates measured on this GPU now
            try:
                r_fma, r_div = B.cwm_fp64_rates()
                roof["fp64"] = {"probe": "cwm_fp64_rates: 8 independent FP64 chains per thread, 8 blocks of 256 "
                                         "threads per SM, CUDA events", "fma_per_s": r_fma, "div_per_s": r_div,
                                "classes": fp64_fractions(roof["classes"], n, nnz, int(np.count_nonzero(val)),
                                                          r_fma, r_div)}
            except Exception as exc:  # noqa: BLE001
                roof["fp64"] = {"error": str(exc)}

    # precision variants on the same workload (not part of the timed value): the other
    # V-cycle precision, and binary32 Galerkin products for every coarse operator with the
    # float32 V-cycle
    variants = []
    check_cost = None
    if args.variant and dist is None:
        # the cost of the input check (structure, positive diagonal, bit symmetry; the library
        # default) that the timed steps leave off: setup with and without it, best of three
        tset = {0: [], 1: []}
        for _ in range(3):
            for chk in (0, 1):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                e[0].record(stream)
                hc = B.amg_setup(d_rp, d_ci, d_val, d_v, B.amg_default_params(
                    sweeps_per_level=sweeps, coarse_max=cmax, vcycle_fp32=int(fp32), check_input=chk, **extra))
                e[1].record(stream)
                torch.cuda.synchronize()
                hc.free()
                tset[chk].append(e[0].elapsed_time(e[1]))
        check_cost = {"setup_ms_check_off": round(min(tset[0]), 3), "setup_ms_check_on": round(min(tset[1]), 3),
                      "check_input_ms": round(min(tset[1]) - min(tset[0]), 3)}
        for vf32, gf32 in ((int(not fp32), 0), (1, 1)):
            prmv = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, vcycle_fp32=vf32,
                                        galerkin_fp32_from=gf32, check_input=0, **extra)
            res = []
            for _ in range(3):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                h, st, info = step(prmv, e)
                h.free()
                torch.cuda.synchronize()
                xv = x.cpu().numpy()
                res.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), info, relerr(xv, xs), xv))
            best = min(res, key=lambda r: r[0] + r[1])
            variants.append({"vcycle": "fp32" if vf32 else "fp64", "galerkin": "fp32" if gf32 else "fp64",
                             "ms_per_step": round(best[0] + best[1], 3), "setup_ms": round(best[0], 3),
                             "solve_ms": round(best[1], 3), "iters": best[2]["iters"],
                             "rel_res_true": best[2]["rel_res_true"], "err_vs_xstar": best[3], "_x": best[4]})

    # the full-size oracle solve of the same system (for each result's distance to it) runs in
    # a spawned worker on one host core beside the CPU baseline, after every GPU measurement,
    # so that the timed loops (the FCG makes a host round trip per iteration) share the host
    # with no other busy process
    oracle_job = None
    if rank == 0 and world == 1 and args.oracle_check:
        import concurrent.futures as cf
        import multiprocessing as mp
        oracle_pool = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
        oracle_job = oracle_pool.submit(oracle_full_solve, args.workload, args.rtol, args.itmax)

    # CPU baseline: the oracle as it stands on a bounded sample of the workload, rank 0 at N=1
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, nnz, args.rtol, args.itmax)
    # each result's distance to the FP64 oracle's solution of the same full-size system
    x_oracle, oracle_iters = None, None
    if oracle_job is not None:
        x_oracle, oracle_iters = oracle_job.result()
        oracle_pool.shutdown()
    err_oracle = relerr(x_main, x_oracle)
    for vr in variants:
        xv = vr.pop("_x")
        vr["err_vs_oracle"] = relerr(xv, x_oracle)

    last = infos[-1]
    out = {
        "metric": METRIC, "value": round(ms_per_step, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if not fp32 else "f64+f32-vcycle",
        "data": "synthetic",
        "config": bench_config(args.workload, n, nnz, desc, sweeps, cmax, args.rtol, fp32, world),
        "setup_ms": round(statistics.median(setup_ms), 3), "solve_ms": round(statistics.median(solve_ms), 3),
        "iters": last["iters"], "ms_per_iter": round(statistics.median(solve_ms) / max(last["iters"], 1), 4),
        "levels": last["nl"], "vcmplx": round(last["vcmplx"], 4), "cratio": round(last["cratio"], 4),
        "level_sizes": level_sizes,
        "rel_res_true": last["rel_res_true"], "err_vs_xstar": err, "err_vs_oracle": err_oracle,
        "oracle_iters": oracle_iters, "input_check": check_cost,
        "status": [B.status_name(s) for s in statuses][-1],
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "h2d_ms": round(h2d_ms, 3), "h2d_gbs": round(h2d / (h2d_ms * 1e-3) / 1e9, 1),
                "median_ms": round(statistics.median(e2e_steps), 3), "steps_ms": e2e_steps},
        "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "kernel_classes": sorted([{k: (round(v, 4) if isinstance(v, float) else v) for k, v in e.items()}
                                  for e in trace_all], key=lambda e: -e["total_ms"])[:12],
    }
    if variants:
        out["variants"] = variants
    if rank == 0:
        print(json.dumps(out))


def class_rooflines(trace, peak, workload=None):
    """Per kernel class of one traced step: launches, algorithmic bytes per launch, average
    launch time and the fraction of the HBM peak those bytes reach."""
    out = []
    for e in sorted(trace, key=lambda e: -e["total_ms"]):
        if e["launches"] <= 0 or e["total_ms"] <= 0:
            continue
        us = e["total_ms"] / e["launches"] * 1e3
        bpl = e["bytes"] / e["launches"]
        row = {"kernel": e["name"], "launches": e["launches"], "total_ms": round(e["total_ms"], 4),
               "bytes_per_launch": round(bpl), "avg_launch_us": round(us, 2),
               "achieved_gbs": round(bpl / us * 1e-3, 1), "frac": round(bpl / us * 1e-3 / peak, 4)}
        tr = _traffic_for(e["name"], workload)
        if tr is not None:
            row["traffic"] = tr
        out.append(row)
    return out


def fp64_fractions(classes, n, nnz, nnz_nonzero, r_fma, r_div):
    """FP64 issue fraction of the FP64-bound classes: the time their FP64 operations take at
    the measured rates over their measured launch time.  spmv_dots: one FMA per stored entry
    and three per row (the dot products); weights@0 (the first sweep on the input operator):
    two multiplies and two adds per evaluation (2a is an exponent increment and the division
    runs on the integer pipes), once per stored off-diagonal nonzero pair on short-row
    operators, once per such slot where rows average more than 32 slots (every slot is
    evaluated in its own row).  r_div is kept for callers; no class uses it now."""
    out = []
    edges = max(nnz_nonzero - n, 0) / 2.0
    for c in classes:
        if c["kernel"] in ("spmv_dots", "spmv_dots_b3"):
            t = (nnz + 3.0 * n) / r_fma
            what = "(nnz + 3n) FMA"
        elif c["kernel"] == "weights@0":
            if nnz > 32 * n:
                t = 2.0 * edges * 4.0 / r_fma
                what = "per stored off-diagonal nonzero slot 4 FP64 ops (division on the integer pipes)"
            else:
                t = edges * 4.0 / r_fma
                what = "per edge 4 FP64 ops (division on the integer pipes)"
        else:
            continue
        out.append({"kernel": c["kernel"], "ops": what, "fp64_us": round(t * 1e6, 2),
                    "avg_launch_us": c["avg_launch_us"], "fp64_frac": round(t * 1e6 / c["avg_launch_us"], 4)})
    return out


def _oracle_step(name, rtol, itmax):
    """One oracle step (setup + FCG) on workload `name`: (x, iterations, setup ms, solve ms)."""
    import oracle
    desc, mat, v, b, xs, sweeps, cmax, fp32, extra = workload(name)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax, stall_ratio=extra.get("stall_ratio", 0.0))
    t1 = time.perf_counter()
    xr, st, it, _, _ = H.pcg(b, rtol=rtol, itmax=itmax)
    t2 = time.perf_counter()
    H.close()
    return xr, it, (t1 - t0) * 1e3, (t2 - t1) * 1e3, len(mat[1])


def oracle_full_solve(name, rtol, itmax):
    """The oracle's FP64 solution of the full-size workload and its iteration count."""
    xr, it, _, _, _ = _oracle_step(name, rtol, itmax)
    return xr, it


def cpu_baseline(name, nnz_full, rtol, itmax):
    """The oracle, single-threaded, on CPU_SAMPLE[name]; value scaled by nnz_full / nnz_sample."""
    sample = CPU_SAMPLE[name]
    _, it, setup, solve, nnz_s = _oracle_step(sample, rtol, itmax)
    scale = nnz_full / nnz_s
    return {"value": round((setup + solve) * scale, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample_ms": round(setup + solve, 1), "sample_setup_ms": round(setup, 1),
            "sample_solve_ms": round(solve, 1), "sample_iters": it, "scale_nnz": round(scale, 4),
            "sample": (f"one step (setup + FCG to the same rtol) of {sample} ({nnz_s} stored entries), the same "
                       f"problem family and parameters on a coarser grid, single-threaded C oracle; value = "
                       f"sample ms x {round(scale, 4)} (ratio of stored entries)" if sample != name else
                       "the full workload, one step (setup + FCG), single-threaded C oracle"),
            "host_cores": os.cpu_count()}


# --------------------------------------------------------------------- reference arm ----

def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, one bounded sample per step (the
    cpu_baseline sample of the workload, scaled the same way)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    desc, mat, v, b, xs, sweeps, cmax, fp32, extra = workload(args.workload)
    n, nnz = len(mat[0]) - 1, len(mat[1])
    del mat, v, b, xs
    # warm-up on a small instance of the same problem family (pages code in)
    small = P.poisson3d(16)
    for _ in range(args.warmup):
        Hs = oracle.Hierarchy(*small, np.ones(16 ** 3), sweeps=sweeps, coarse_max=cmax)
        Hs.pcg(P.manufactured_rhs(*small, seed=0)[1], rtol=args.rtol)
        Hs.close()
    sample = CPU_SAMPLE[args.workload]
    smat = workload(sample)
    times, it, nnz_s = [], 0, len(smat[1][1])
    for _ in range(args.steps):
        t0 = time.perf_counter()
        H = oracle.Hierarchy(*smat[1], smat[2], sweeps=smat[5], coarse_max=smat[6],
                             stall_ratio=smat[8].get("stall_ratio", 0.0))
        _, st, it, _, _ = H.pcg(smat[3], rtol=args.rtol, itmax=args.itmax)
        times.append((time.perf_counter() - t0) * 1e3)
        H.close()
    scale = nnz / nnz_s
    ms = sum(times) / len(times) * scale
    samp = (f"per step one oracle step (setup + FCG) of {sample} ({nnz_s} stored entries), value = sample ms x "
            f"{round(scale, 4)} (ratio of stored entries); single-threaded C oracle; warm-up on 16^3")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.workload, n, nnz, desc, sweeps, cmax, args.rtol, fp32, world),
        "iters": it, "sample_ms": round(sum(times) / len(times), 1),
        "cpu_baseline": {"value": round(ms, 1), "unit": "ms", "cores": 1, "kind": "oracle", "sample": samp},
        "e2e": {"value": round(ms, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="elasticity_64", choices=WORKLOADS)
    ap.add_argument("--fp32", type=int, default=None, help="override the workload's V-cycle precision")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--itmax", type=int, default=5000)
    ap.add_argument("--variant", type=int, default=1,
                    help="also time the precision variants (other V-cycle precision; binary32 Galerkin)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block3", type=int, default=0, choices=[0, -1],
                    help="3x3-block layout of the finest operator: 0 auto (when its pattern qualifies), -1 never")
    ap.add_argument("--oracle-check", type=int, default=1,
                    help="solve the full-size system with the oracle too (spawned worker) and report each "
                         "result's distance to its solution")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (no e2e, variant, CPU baseline): for ncu launch lists")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "cuda" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_cuda(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
