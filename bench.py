#!/usr/bin/env python
"""Benchmark of the CPTR-FGMRES hot path on one GB300 per rank.

A step is one pass of the whole path on one Jacobian: cptr_setup (decoupling, p-T extraction,
two AMG hierarchies built on the device, block ILU(0)) followed by cptr_solve (FGMRES(30) with
the two-stage CPTR preconditioner to a 1e-6 relative residual), on the seeded synthetic
100x100x20 workload (200k cells, 600k unknowns).  Inputs are resident in HBM when the timed
region starts and L2 is flushed before every step.  Ranks (torchrun) run independent replicas:
the method has no data-parallel split of one system, so there is no collective on the data path.

--impl reference times the FP64 CPU oracle on the same workload (host cores).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPTR-FGMRES solve time & dofs/s to 1e-6 rel. residual; SpMV/V-cycle HBM GB/s"
UNIT = "dofs/s"
RTOL = 1e-6
WORKLOAD = "cptr200k"
L2_BYTES = 129 * 2 ** 20
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
LEARNED_STEPS, LEARNED_LR = 2000, 2e-3
# DRAM bytes (read + write) per launch from the ncu captures summarised under profiles/ (the
# current kernels; None where no capture of the current code exists)
PROFILED_TRAFFIC = {"spmv": 113_717_248, "stage1_resid": None, "ilu_fwd": 102_685_952, "ilu_bwd": 122_592_512,
                    # the finest V-cycle level of the pressure hierarchy (cold-L2 captures, one launch each)
                    "vcycle_p_down": 20_470_528, "vcycle_p_restrict": 6_354_944, "vcycle_p_prolong": 7_413_760,
                    "vcycle_p_post": 22_069_504, "vcycle_p_down_mixed": 13_381_120,
                    "vcycle_p_restrict_mixed": 4_057_344, "vcycle_p_prolong_mixed": 4_857_600,
                    "vcycle_p_post_mixed": 14_180_608}
# the ILU figures belong to one sweep configuration (schedule 2: grouped levels; levels per group;
# lanes per row): they are attached only when the timed solver runs that configuration
PROFILED_ILU_SCHEDULE = (2, 2, 16)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-three-phase", action="store_true")
    p.add_argument("--no-small", action="store_true", help="skip the 16x16x4 two-level configuration")
    p.add_argument("--no-ensemble", action="store_true")
    p.add_argument("--three-phase-grid", type=int, nargs=3, default=None,
                   help="run the three-phase section on an NX NY NZ box instead of 200x200x50 (profiling)")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="fixed launch shapes in the headline solver (default: autotuned at the first set-up, cached)")
    p.add_argument("--graph", choices=["cycle", "step"], default="cycle",
                   help="headline solver: each restart cycle as one graph launch (device-side loop), or one "
                        "graph launch per Arnoldi step (what per-kernel profilers see kernel by kernel)")
    p.add_argument("--ilu-group", type=int, default=0,
                   help="levels per group of the grouped-level (paired) sweeps; 0: the library's choice")
    p.add_argument("--ilu-lanes", type=int, default=0,
                   help="lanes per row of the grouped-level sweeps (4, 8, 16); 0: the library's choice")
    p.add_argument("--ilu-sweep", choices=["auto", "levels", "chunked", "paired", "tiled"], default="auto",
                   help="schedule of the headline solver's ILU(0) sweeps")
    p.add_argument("--ensemble-total", type=float, default=4e6,
                   help="total cells of the ensemble (profiling runs use a smaller one)")
    p.add_argument("--no-oracle-errors", action="store_true",
                   help="skip the oracle solutions of the three-phase and ensemble workloads (errors against "
                        "the FP64 oracle are then reported for the cptr200k forms only)")
    p.add_argument("--no-newton", action="store_true", help="skip the Newton time-stepping section")
    p.add_argument("--no-mesh-study", action="store_true",
                   help="skip the 2-D mesh-refinement study (Tables meshW, meshH, anisomeshW analogues)")
    p.add_argument("--mesh-study-max-n", type=int, default=640)
    p.add_argument("--ncu-range", choices=["headline", "vcycle", "vcycle_mixed", "spmv_b4"], default=None,
                   help="after the warm-up, run one untimed piece of work between cudaProfilerStart and "
                        "cudaProfilerStop (for ncu --profile-from-start off): a headline step; one V-cycle of "
                        "the headline's pressure hierarchy; the same in the mixed form; one outer SpMV and one "
                        "preconditioner application of the three-phase FP64 S_e solver")
    p.add_argument("--three-phase-forms", default=None,
                   help="comma-separated subset of the three-phase forms to run (default: all)")
    p.add_argument("--profile-steps", type=int, default=3,
                   help="steps of the separate pass that times kernel families with CUDA events")
    return p.parse_args()


# the add-on forms, each timed on the same workload to the same tolerance (outside the headline)
VARIANTS = {
    "cpr_fp64": dict(stage1="cpr"),
    "cptr_fp64_multicolor_ilu": dict(ilu_order="multicolor"),
    "cptr_mixed": dict(precision="mixed"),
    "cptr_mixed_multicolor_ilu": dict(precision="mixed", ilu_order="multicolor"),
    "cptr_fp64_autotuned": dict(autotune=1),
    "cptr_mixed_autotuned": dict(precision="mixed", autotune=1),
    # the paper's parallel second stage (Sec. 4): ILU(0) on each of 16 parts of the domain (4 x 4
    # columns of 25 x 25 x 20 cells), as 16 processes would apply it
    "cptr_fp64_block_jacobi16": dict(autotune=1, part=(4, 4)),
    "cptr_mixed_block_jacobi16": dict(precision="mixed", autotune=1, part=(4, 4)),
}


def grid_parts(nx, ny, nz, px, py):
    """Part id per cell of a natural-order nx x ny x nz grid cut into px x py columns."""
    i = np.arange(nx * ny * nz)
    x, y = i % nx, (i // nx) % ny
    return ((x * px) // nx + px * ((y * py) // ny)).astype(np.int32)
# the variant whose kernels get roofline lines of their own ("..._mixed")
MIXED_PROFILED = "cptr_mixed_autotuned"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return PEAKS_FALLBACK["hbm_gbs"], "fallback"


# ------------------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd.insert(1, f"--id={self.gpu_id}")
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_identifier(torch, dev):
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        u = str(uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    return None


# ------------------------------------------------------------------------------------------------
def oracle_step(s):
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle.from_system(s)
    x, info = o.solve(s["rhs"], RTOL)
    return time.perf_counter() - t0, info, x


def oracle_job(kind, arg=None):
    """FP64 oracle solution of one of the benchmark's workloads, run in a spawned worker process
    (one host core) while the GPU part runs: (seconds for set-up + solve, info, x)."""
    import synth
    if kind == "three_phase":
        s = synth.recipe("three_phase2m").system() if arg is None else synth.make_box(
            *arg, 1.0, 1.0, 0.5, seed=21, sigma=2.5, nphase=3, wells="four", T_inj=500.0, q_inj=4e-6).system()
    elif kind == "newton":   # the first implicit Euler step of the Newton section, by the oracle's driver
        import oracle
        r = newton_reservoir()
        t0 = time.perf_counter()
        x, info = oracle.newton_step(r, r.x0.copy(), r.x0, NEWTON_RTOL)
        secs = time.perf_counter() - t0
        return secs, {k: v for k, v in info.items() if k != "per_iteration"}, x.reshape(-1)
    elif kind == "ensemble":
        total, k = arg
        shapes = synth.ensemble_sizes(total=total, lo=min(20e3, total / 64))
        s = synth.ensemble_member(k, shapes[k]).system()
    else:
        raise KeyError(kind)
    secs, info, x = oracle_step(s)
    return secs, {"iters": int(info["iters"]), "converged": bool(info["converged"])}, x


def start_oracle_jobs(args):
    """Oracle solutions for the error of every form against the FP64 oracle, started before any
    GPU call in a spawn-context pool: the three-phase workload, and four instances of the
    ensemble (the smallest, the largest and two between)."""
    import multiprocessing as mp
    jobs = {}
    if args.no_oracle_errors:
        return None, jobs
    pool = mp.get_context("spawn").Pool(processes=3)
    if not args.no_three_phase:
        jobs["three_phase"] = pool.apply_async(oracle_job, ("three_phase", args.three_phase_grid))
    if not args.no_newton:
        jobs["newton"] = pool.apply_async(oracle_job, ("newton",))
    if not args.no_ensemble:
        import synth
        shapes = synth.ensemble_sizes(total=args.ensemble_total, lo=min(20e3, args.ensemble_total / 64))
        cells = [sh[0] * sh[1] * sh[2] for sh in shapes]
        order = np.argsort(cells)
        pick = sorted({int(order[0]), int(order[len(order) // 3]), int(order[2 * len(order) // 3]), int(order[-1])})
        jobs["ensemble"] = {k: pool.apply_async(oracle_job, ("ensemble", (args.ensemble_total, k))) for k in pick}
    pool.close()
    return pool, jobs


def errors_per_kind(xg, xo, b):
    """Relative error of a GPU solution against the FP64 oracle's, per unknown kind and overall."""
    xg, xo = np.asarray(xg, np.float64), np.asarray(xo, np.float64)
    per = [float(np.linalg.norm(xg[u::b] - xo[u::b]) / max(np.linalg.norm(xo[u::b]), 1e-300)) for u in range(b)]
    return {"per_unknown_kind": [float("%.3e" % e) for e in per],
            "overall": float("%.3e" % (np.linalg.norm(xg - xo) / max(np.linalg.norm(xo), 1e-300)))}


# GB300's FP64 rate: 152 SMs x 2.07 GHz x 2 FP64 FMA/clk/SM x 2 flop (nominal 1.25 TFLOP/s; not measured)
FP64_PEAK_TFLOPS = 1.258


def algorithmic_bytes(s, mixed=False):
    """Bytes each kernel must move once per launch (int32 indices; FP64 values and vectors, or in
    the mixed form FP32 values of the preconditioner and FP32 vectors inside it):
    spmv: blocks (b*b values + column) + chunk offsets + z read + w written (FP64 in both forms);
    stage1_resid: the p and T columns of every block (2b values + column) + chunk offsets + v read
    (FP64) + b1 written + dp, dT read; ilu_fwd: L blocks + columns + positions + r read + y
    written; ilu_bwd: U blocks + columns + inverted pivot blocks + positions (2) + y read + the
    intermediate written + z written (FP64) + dp, dT read."""
    n, b = s["n"], s["b"]
    rp, ci = s["row_ptr"], s["col_idx"]
    nnzb = int(rp[-1])
    rows = np.repeat(np.arange(n), np.diff(rp))
    lower = int((ci < rows).sum())
    upper = nnzb - n - lower
    chunks = (n + 31) // 32
    nb = n * b
    f = 4 if mixed else 8   # preconditioner values and inner vectors
    return {"spmv": nnzb * (8 * b * b + 4) + (chunks + 1) * 8 + 2 * nb * 8,
            "stage1_resid": nnzb * (f * 2 * b + 4) + (chunks + 1) * 8 + nb * 8 + nb * f + 2 * n * f,
            "ilu_fwd": lower * (f * b * b + 4) + n * 4 + 2 * nb * f,
            "ilu_bwd": upper * (f * b * b + 4) + n * f * b * b + n * 8 + 2 * nb * f + nb * 8 + 2 * n * f}


VC_STEPS = {"down": "k_vc_down (pre-smoothing from zero + residual, t = D^-1 b, r = b - A t)",
            "restrict": "k_csr_spmv (restriction b_c = P^T r)",
            "prolong": "k_csr_spmv (prolongation t += P x_c)",
            "post": "k_vc_post (post-smoothing x = t + D^-1 (b - A t))"}


def vcycle_bytes(info, f):
    """Algorithmic bytes of the finest level's four V-cycle kernels from the level sizes (n rows,
    nnz of A, nnz of P, nc coarse rows), f = bytes per value and per vector entry (8 in FP64; 4 in
    the mixed form, whose finest level is FP32): down reads A (values + columns + row pointers),
    D^-1 and b, writes t and r; restrict reads P^T and r, writes b_c; prolong reads P and x_c,
    reads and writes t; post reads A, D^-1, b and t, writes x."""
    n, nnz, nnzp = info[0]["n"], info[0]["nnz"], info[0]["nnzP"]
    nc = info[1]["n"]
    return {"down": nnz * (4 + f) + 4 * (n + 1) + 4 * f * n,
            "restrict": nnzp * (4 + f) + 4 * (nc + 1) + f * n + f * nc,
            "prolong": nnzp * (4 + f) + 4 * (n + 1) + f * nc + 2 * f * n,
            "post": nnz * (4 + f) + 4 * (n + 1) + 4 * f * n}


def roofline_line(kernel, alg, ms_tot, cnt, steps, peak, peak_kind, traffic=None):
    avg_ms = ms_tot / max(cnt, 1)
    achieved = alg / (avg_ms / 1e3) / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": int(alg), "avg_launch_us": round(avg_ms * 1e3, 2),
            "launches_per_step": cnt / steps, "ms_per_step": round(ms_tot / steps, 3)}


def family_kernels(cp, S, b, mixed):
    """Kernel names of the profiled families of solver S (from its ILU schedule)."""
    tun = cp.cptr_tuning(S.ctx)
    sched, group = [t for t in tun if t[2] == 5][0][3:5]
    lanes = [t for t in tun if t[2] == 7][0][3]
    t = "float" if mixed else "double"
    sweep = {0: "level sets", 1: "chunked wavefront", 2: "paired levels" if group == 2 else f"groups of {group} levels",
             3: "tiled"}[sched]
    four = sched == 2 or (sched == 0 and not mixed)
    how = sweep + (f", a row over {lanes if sched == 2 else 4} lanes" if four else "")
    if sched == 2 and lanes in (8, 16):
        fwd, bwd = f"k_ilu_fwd_h<{b},{t},...>", f"k_ilu_bwd_h<{b},{t},...>"
    elif sched == 1:
        fwd, bwd = f"k_ilu_cw<{b},{t},...,FWD>", f"k_ilu_cw<{b},{t},...,BWD>"
    elif sched == 3:
        fwd, bwd = f"k_ilu_tile<{b},{t},...,FWD>", f"k_ilu_tile<{b},{t},...,BWD>"
    elif four:
        fwd, bwd = f"k_ilu_fwd_g<{b},{t},...>", f"k_ilu_bwd_g<{b},{t},...>"
    else:
        fwd, bwd = f"k_ilu_fwd_sf<{b},{t},...>", f"k_ilu_bwd_sf<{b},{t},...>"
    return {"spmv": f"k_sell_spmv<{b},0> (outer w = A' z_j, FP64)",
            "stage1_resid": (f"k_sell_resid_pt32<{b}> (stage-1 residual, FP32 values)" if mixed else
                             f"k_sell_spmv<{b},2> (stage-1 residual)"),
            "ilu_fwd": f"{fwd} (forward ILU(0) sweep, {how})",
            "ilu_bwd": f"{bwd} (backward ILU(0) sweep, {how})"}, sched


def vcycle_lines(cp, S, vc_sum, steps, peak, peak_kind, mixed, suffix, traffic=None):
    """Roofline lines of the finest level's V-cycle kernels of both hierarchies."""
    lines = {}
    f = 4 if mixed else 8
    vt = "float" if mixed else "double"
    for h, which in (("p", 0), ("T", 1)):
        if vc_sum.get(f"{h}_down", (0.0, 0))[1] == 0:
            continue
        info = cp.cptr_hierarchy_info(S.ctx, which)
        if len(info) < 2:
            continue
        alg = vcycle_bytes(info, f)
        for k, desc in VC_STEPS.items():
            ms_tot, cnt = vc_sum[f"{h}_{k}"]
            name = f"vcycle_{h}_{k}{suffix}"
            lines[name] = roofline_line(f"{desc.split(' ', 1)[0]}<..., {vt}> {desc.split(' ', 1)[1]}, finest level of "
                                        f"the {'pressure' if h == 'p' else 'temperature'} hierarchy "
                                        f"({info[0]['n']} rows, {info[0]['nnz']} entries)",
                                        alg[k], ms_tot, cnt, steps, peak, peak_kind,
                                        (traffic or {}).get(name))
    return lines


def profiled_pass(cp, S, step, flush, steps, mask):
    """Steps with CUDA events around the families and kernels that `mask` selects; summed times."""
    cp.cptr_set_profiling(S.ctx, mask)
    fam, vc = {}, {}
    for _ in range(steps):
        flush.zero_()
        step()
        for src, dst in ((cp.cptr_profile(S.ctx), fam), (cp.cptr_profile_vcycle(S.ctx), vc)):
            for k, (ms, cnt) in src.items():
                acc = dst.setdefault(k, [0.0, 0])
                acc[0] += ms
                acc[1] += cnt
    cp.cptr_set_profiling(S.ctx, 0)
    return fam, vc


def profiled_range(args, section, work):
    """work() once, untimed, inside a profiler range when --ncu-range names this section."""
    if args.ncu_range != section:
        return
    import torch
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    work()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


def vcycle_once(cp, S, n, dev):
    """One V-cycle of the pressure hierarchy on a seeded right-hand side (cptr_apply_vcycle)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(5)
    b = torch.randn(n, generator=g, dtype=torch.float64).to(dev)
    x = torch.empty_like(b)
    return lambda: cp.cptr_apply_vcycle(S.ctx, 0, b, x)


def ours(args, rank, world, local_rank, oracle_jobs):
    import numpy as np
    import torch

    import synth
    import paper_1907_04229_gb300 as cp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    r = synth.recipe(WORKLOAD)
    s = r.system()
    n, b, nnzb = s["n"], s["b"], int(s["row_ptr"][-1])
    dofs = n * b
    nx, ny, nz = s["grid"]
    ilu_levels = nx + ny + nz - 2
    host = {"rp": s["row_ptr"], "ci": s["col_idx"], "vals": s["vals"].reshape(-1), "kind": s["unknown_kind"],
            "W": s["weights"].reshape(-1), "st": s["st"], "rhs": s["rhs"].reshape(-1)}
    d = {k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in host.items()}
    x = torch.empty(dofs, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    head_opts = dict(autotune=int(args.autotune), ilu_sweep=args.ilu_sweep, use_graph=1 if args.graph == "cycle" else 2,
                     ilu_group=args.ilu_group, ilu_lanes=args.ilu_lanes)
    S = cp.Solver(stream=stream, **head_opts)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        S.setup(n, b, d["rp"], d["ci"], d["vals"], d["kind"], d["W"], d["st"])
        return S.solve(d["rhs"], RTOL, x=x)[1]

    for _ in range(args.warmup):
        info = step()
    assert info["status"] == "CPTR_OK", info
    profiled_range(args, "headline", step)
    profiled_range(args, "vcycle", vcycle_once(cp, S, n, dev))
    # the headline: plain steps, no per-kernel events in the timed region
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks = Clocks(gpu_identifier(torch, dev))
    clocks.start()
    launches0 = cp.cptr_launch_count()
    events = []
    infos = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(step())
        e1.record(stream)
        events.append((e0, e1))
    torch.cuda.synchronize(dev)
    launches = cp.cptr_launch_count() - launches0
    barrier(world)
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(bb) for a, bb in events)
    value, ms_per_step = aggregate(total_ms, world, dofs, args.steps, dev)
    setup_ms = statistics.mean(i["setup_ms"] for i in infos)
    solve_ms = statistics.mean(i["solve_ms"] for i in infos)
    iters = infos[-1]["iters"]
    x_head = x.cpu().numpy().copy()
    # a separate pass of the same steps with CUDA events around every kernel family (on the
    # library's stream): the per-family split and the per-launch rooflines come from it
    cp.cptr_set_profiling(S.ctx, 0b1111111)
    prof_sum = {}
    prof_events = []
    for _ in range(args.profile_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        prof_events.append((e0, e1))
        for k, (ms, cnt) in cp.cptr_profile(S.ctx).items():
            acc = prof_sum.setdefault(k, [0.0, 0])
            acc[0] += ms
            acc[1] += cnt
    torch.cuda.synchronize(dev)
    cp.cptr_set_profiling(S.ctx, 0)
    prof_ms_per_step = sum(a.elapsed_time(bb) for a, bb in prof_events) / max(len(prof_events), 1)

    # rooflines from per-launch CUDA events inside the timed region; the dominant single kernel
    # (largest total time) is reported as "roofline"
    peak, peak_kind = peaks()
    alg = algorithmic_bytes(s)
    kernels, schedule = family_kernels(cp, S, b, False)
    chunked, paired = schedule == 1, schedule == 2
    tun = cp.cptr_tuning(S.ctx)
    group = [t for t in tun if t[2] == 5][0][4]
    ilu_config = (schedule, group, [t for t in tun if t[2] == 7][0][3])
    lines = {}
    for fam, kname in kernels.items():
        ms_tot, cnt = prof_sum[fam]
        lines[fam] = roofline_line(kname, alg[fam], ms_tot, cnt, args.profile_steps, peak, peak_kind,
                                   PROFILED_TRAFFIC.get(fam) if not fam.startswith("ilu") or
                                   ilu_config == PROFILED_ILU_SCHEDULE else None)
    # the finest level's V-cycle kernels, timed one by one in a pass of their own
    _, vc_sum = profiled_pass(cp, S, step, flush, args.profile_steps, cp.PROFILE_MASK_VCYCLE)
    lines.update(vcycle_lines(cp, S, vc_sum, args.profile_steps, peak, peak_kind, False, "", PROFILED_TRAFFIC))
    # FP64 ALU view of the SpMV: 9 FMA per 3x3 block (2 flop each) against 1.258 TFLOP/s
    # (152 SMs x 2.07 GHz x 2 FP64 FMA/clk x 2)
    spmv_flops = 2 * b * b * nnzb
    lines["spmv"]["alu"] = {"achieved_tflops": round(spmv_flops / (lines["spmv"]["avg_launch_us"] * 1e-6) / 1e12, 3),
                            "peak_tflops": FP64_PEAK_TFLOPS, "peak_source": "nominal (not measured)",
                            "frac": round(
                                spmv_flops / (lines["spmv"]["avg_launch_us"] * 1e-6) / 1e12 / FP64_PEAK_TFLOPS, 4)}
    # the Arnoldi family (three CGS2 passes + the new basis vector) against the FP64 rate: Arnoldi
    # step j of a restart cycle (nc = j + 1 columns) does 8 nc + 3 flop per vector entry (two dot
    # passes, two updates, the norm, the scaling) and moves 3 nc + 7 vector entries
    cols = [it % S.opts.restart + 1 for it in range(iters)]
    cgs_flops = sum(8 * c + 3 for c in cols) * dofs
    cgs_bytes = sum(3 * c + 7 for c in cols) * dofs * 8
    a_ms = prof_sum["arnoldi"][0] / args.profile_steps
    a_tf = cgs_flops / (a_ms * 1e-3) / 1e12
    a_gbs = cgs_bytes / (a_ms * 1e-3) / 1e9
    lines["arnoldi"] = {"kernel": "k_cgs<0>, k_cgs<1>, k_cgs<2>, k_scale (CGS2 passes, v_{j+1} = w / ||w||)",
                        "bound": "alu", "achieved": round(a_tf, 3), "peak": FP64_PEAK_TFLOPS,
                        "peak_source": "nominal FP64 rate (not measured)", "unit": "TFLOP/s",
                        "frac": round(a_tf / FP64_PEAK_TFLOPS, 4), "traffic": None,
                        "algorithmic_flops_per_step": cgs_flops, "ms_per_step": round(a_ms, 3),
                        "hbm": {"achieved": round(a_gbs, 1), "peak": peak, "frac": round(a_gbs / peak, 4),
                                "algorithmic_bytes_per_step": cgs_bytes}}
    dominant = max(("ilu_fwd", "ilu_bwd", "spmv", "stage1_resid"), key=lambda f: prof_sum[f][0])
    roofline = dict(lines[dominant])
    if dominant.startswith("ilu"):
        roofline["note"] = ((f"latency bound: a dependency chain of {ilu_levels} level sets per sweep, "
                             f"run as {(ilu_levels + group - 1) // group} steps of groups of {group} levels" if paired else
                             f"latency bound: a dependency chain of {ilu_levels} level sets per sweep")
                            + (f"; DRAM traffic {roofline['traffic'] / roofline['algorithmic_bytes_per_launch']:.2f}x "
                               "the algorithmic ILU(0) bytes (the grouped tables hold the substituted blocks)"
                               if roofline["traffic"] and paired else ""))
    families = {k: {"ms_per_step": round(v[0] / args.profile_steps, 3),
                    "regions_per_step": v[1] / args.profile_steps} for k, v in prof_sum.items()}
    families["note"] = (f"separate pass of {args.profile_steps} steps with CUDA events around every kernel family "
                        f"({prof_ms_per_step:.3f} ms per step with the events, {ms_per_step:.3f} ms without)")

    # end to end through the public API with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hp = {k: torch.as_tensor(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
        xh = torch.empty(dofs, dtype=torch.float64).pin_memory()
        Sh = cp.Solver(stream=stream, **head_opts)

        def step_host():
            Sh.setup(n, b, hp["rp"].numpy(), hp["ci"].numpy(), hp["vals"].numpy(), hp["kind"].numpy(),
                     hp["W"].numpy(), hp["st"].numpy())
            return Sh.solve(hp["rhs"].numpy(), RTOL, x=xh.numpy())[1]

        for _ in range(max(1, min(args.warmup, 2))):
            step_host()
        barrier(world)
        torch.cuda.synchronize(dev)
        t_tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ih = step_host()
            t_tot += time.perf_counter() - t0
        t_tot = allreduce_max(t_tot * 1e3, world, dev)
        h2d = sum(v.numel() * v.element_size() for v in hp.values())
        e2e = {"value": world * dofs * args.steps / (t_tot / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": dofs * 8, "ms_per_step": t_tot / args.steps, "iters": ih["iters"]}

    sols = {}
    variants = None
    if not args.no_variants:
        variants = {}
        for name, opts in VARIANTS.items():
            opts = dict(opts)
            parts = opts.pop("part", None)
            Sv = cp.Solver(stream=stream, **opts)
            if parts:
                cp.cptr_set_partition(Sv.ctx, torch.as_tensor(grid_parts(nx, ny, nz, *parts), device=dev))

            def step_v():
                Sv.setup(n, b, d["rp"], d["ci"], d["vals"], d["kind"], d["W"], d["st"])
                return Sv.solve(d["rhs"], RTOL, x=x)[1]

            step_v()
            if name == "cptr_mixed":
                profiled_range(args, "vcycle_mixed", vcycle_once(cp, Sv, n, dev))
            evs, infs = [], []
            for _ in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                infs.append(step_v())
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize(dev)
            ms = sum(a.elapsed_time(bb) for a, bb in evs) / len(evs)
            sols["variant_" + name] = x.cpu().numpy().copy()
            variants[name] = {"ms_per_step": round(ms, 3), "dofs_per_s": round(dofs / (ms / 1e3), 1),
                              "setup_ms": round(statistics.mean(i["setup_ms"] for i in infs), 3),
                              "solve_ms": round(statistics.mean(i["solve_ms"] for i in infs), 3),
                              "iters": infs[-1]["iters"], "true_rel_res": infs[-1]["true_rel_res"],
                              "status": infs[-1]["status"]}
            if name == MIXED_PROFILED:
                # the mixed form's kernels: families and the finest V-cycle level, one profiled pass
                fam, vc = profiled_pass(cp, Sv, step_v, flush, args.profile_steps, 0xFF)
                kern, _ = family_kernels(cp, Sv, b, True)
                alg_m = algorithmic_bytes(s, mixed=True)
                for f in ("stage1_resid", "ilu_fwd", "ilu_bwd"):
                    lines[f + "_mixed"] = roofline_line(kern[f], alg_m[f], *fam[f], args.profile_steps, peak,
                                                        peak_kind, PROFILED_TRAFFIC.get(f + "_mixed"))
                lines.update(vcycle_lines(cp, Sv, vc, args.profile_steps, peak, peak_kind, True, "_mixed",
                                          PROFILED_TRAFFIC))
            Sv.close()

    small = None
    if not args.no_small:
        small = small_section(args, dev, stream, flush)

    tp = None
    if not args.no_three_phase:
        del flush
        torch.cuda.empty_cache()
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        tp, tp_sols, tp_lines = three_phase(args, dev, stream, flush)
        lines.update(tp_lines)
    ens = None
    if not args.no_ensemble:
        ens, ens_sols = ensemble(args, dev, stream, flush)

    newton = None
    if not args.no_newton:
        newton, newton_x = newton_section(args, dev, stream)

    mesh = None
    if not args.no_mesh_study:
        mesh = mesh_study(args, dev, stream)

    cpu = None
    oracle_errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, oinfo, x_or = oracle_step(s)
        cpu = {"value": dofs / secs, "unit": UNIT, "cores": 1, "cores_available": os.cpu_count(), "kind": "oracle",
               "sample": f"one full setup+solve of the {WORKLOAD} workload ({dofs} dofs) by the serial FP64 C oracle, "
                         f"{secs:.2f} s, {oinfo['iters']} iterations"}
        # every form's solution against the FP64 oracle's solution of the same system
        oracle_errors = {"note": "relative error of each form's solution (rtol 1e-6) against the FP64 oracle's "
                                 "solution of the same system (rtol 1e-6), per unknown kind (p, T, saturations)",
                         "cptr200k": {"oracle_iters": int(oinfo["iters"]),
                                      "headline_fp64": errors_per_kind(x_head, x_or, b)}}
        for k, xv in sols.items():
            oracle_errors["cptr200k"][k] = errors_per_kind(xv, x_or, b)
        if tp is not None and "three_phase" in oracle_jobs:
            osecs, oi, xo3 = oracle_jobs["three_phase"].get()
            e3 = {"oracle_iters": oi["iters"], "oracle_converged": oi["converged"]}
            for k, xv in tp_sols.items():
                e3[k] = errors_per_kind(xv, xo3, 4)
            oracle_errors["three_phase"] = e3
            tp["cpu_baseline"] = {"value": tp_dofs(tp) / osecs, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": f"one full setup+solve by the serial FP64 C oracle, {osecs:.2f} s, "
                                            f"{oi['iters']} iterations (S_e), run in a worker process meanwhile"}
        if newton is not None and "newton" in oracle_jobs:
            osecs, oi, xo = oracle_jobs["newton"].get()
            oracle_errors["newton_first_step"] = dict(errors_per_kind(newton_x, xo, b), oracle_newton_its=oi["newton_its"],
                                                      oracle_linear_its=oi["linear_its"])
            newton["cpu_baseline"] = {"value": round(osecs * 1e3, 1), "unit": "ms per time step", "cores": 1,
                                      "kind": "oracle", "sample": f"the first time step by the oracle's Newton driver "
                                      f"({oi['newton_its']} Newton, {oi['linear_its']} linear iterations), run in a "
                                      "worker process meanwhile"}
        if ens is not None and "ensemble" in oracle_jobs:
            ee, osecs, ocells = {}, 0.0, 0
            for k, job in oracle_jobs["ensemble"].items():
                sk, oi, xo = job.get()
                osecs += sk
                ocells += xo.size // 3
                ee[f"instance_{k}"] = dict(errors_per_kind(ens_sols[k], xo, 3), oracle_iters=oi["iters"])
            oracle_errors["ensemble"] = ee
            tot_cells = ens["total_cells"]
            ens["cpu_baseline"] = {"value": 3 * ocells / osecs, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"{len(ee)} of the {ens['instances']} instances ({ocells} cells) set up "
                                             f"and solved one after another by the serial FP64 C oracle in "
                                             f"{osecs:.2f} s; the whole ensemble extrapolates to "
                                             f"{osecs * tot_cells / ocells:.1f} s"}
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "cptr200k: 100x100x20 cells, 3 unknowns/cell (600k dofs), layered lognormal "
                                      "permeability sigma 2, kv/kh 0.1, k_T 2 W/m/K, 500 K injector; CPTR "
                                      "(full block factorisation, S_e Schur approximation) + ILU(0), FGMRES(30), "
                                      "rtol 1e-6, FP64",
                          "step": "cptr_setup + cptr_solve", "parallelism": f"replicas x{world}",
                          "solver": {"autotune": bool(args.autotune), "ilu_sweep": args.ilu_sweep,
                                     "ilu_schedule_used": ("chunked wavefront" if chunked else
                                                           "paired levels" if paired else "level sets"),
                                     "ilu_sweep_tuning": [t for t in cp.cptr_tuning(S.ctx) if t[2] in (4, 5)],
                                     "amg_shapes_hier_level_kernel_G_T": [t for t in cp.cptr_tuning(S.ctx)
                                                                          if t[2] in (0, 1, 2)],
                                     "tuning_note": "launch shapes timed at the first (warm-up) set-up and cached "
                                                    "by operator size; timed steps reuse them"},
                          "l2": "flushed before every step (256 MB write); working set > 1 GB"},
               "iters": iters, "setup_ms": round(setup_ms, 3), "solve_ms": round(solve_ms, 3),
               "solve_dofs_per_s": round(dofs / (solve_ms / 1e3), 1),
               "true_rel_res": infos[-1]["true_rel_res"], "levels": [infos[-1]["levels_p"], infos[-1]["levels_T"]],
               "families": families, "roofline": roofline, "rooflines": lines, "variants": variants,
               "small_1024": small, "three_phase": tp, "ensemble": ens, "newton": newton, "mesh_refinement": mesh,
               "errors_vs_fp64_oracle": oracle_errors,
               "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "launches_before_timed": launches0, "clocks": clk}
        print(json.dumps(out), flush=True)


def train_learned(dev, stream, base):
    """Train the Schur-scaling network on the GPU: features of the 16 three-phase training grids
    (32x32x8) computed by the library against the base approximation ("se": the discrete S_e,
    "att": A_TT), targets asinh((S_T)_ii / B_ii) stored with the package (written by the oracle).
    Returns (params, train ms, first and last loss, samples)."""
    import torch

    import synth
    import paper_1907_04229_gb300 as cp

    data = np.load(os.path.join(ROOT, "paper_1907_04229_gb300", "data", "schur_targets.npz"))
    targets, shape = data["targets_" + base], tuple(int(v) for v in data["shape"])
    feats = []
    S = cp.Solver(stream=stream, stage1="none", stage2="none")
    for k in range(targets.shape[0]):
        g = synth.learned_training_grid(k, *shape).system()
        S.setup(g["n"], g["b"], g["row_ptr"], g["col_idx"], g["vals"].reshape(-1), g["unknown_kind"],
                g["weights"].reshape(-1), g["st"] if base == "se" else None)
        f = torch.empty((g["n"], cp.MLP_FEATURES), dtype=torch.float64, device=dev)
        cp.cptr_schur_features(S.ctx, f)
        feats.append(f)
    X = torch.cat(feats)
    T = torch.as_tensor(targets.reshape(-1).astype(np.float64), device=dev)
    P = torch.as_tensor(synth.mlp_init(10), device=dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist = cp.cptr_mlp_train(S.ctx, X, T, P, LEARNED_STEPS, lr=LEARNED_LR)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    S.close()
    return P, e0.elapsed_time(e1), float(hist[0]), float(hist[-1]), int(T.numel())


def three_phase(args, dev, stream, flush):
    """The three-phase 200x200x50 workload (2M cells, 4 unknowns/cell, 8M dofs): FP64 CPTR with
    the paper's S_e, with the learned scaling diag(s) S_e, with A_TT and with diag(s) A_TT (the
    networks trained on the GPU first), and the learned S_e form with the mixed-precision
    preconditioner."""
    import torch

    import synth
    import paper_1907_04229_gb300 as cp

    forms = None if args.three_phase_forms is None else set(args.three_phase_forms.split(","))
    nets, training = {}, {}
    for base in ("se", "att"):
        if forms is not None and not any(f"learned_{base}" in f for f in forms):
            continue
        P, train_ms, loss0, loss1, nsamp = train_learned(dev, stream, base)
        nets[base] = P
        training[base] = {"samples": nsamp, "steps": LEARNED_STEPS, "lr": LEARNED_LR, "train_ms": round(train_ms, 2),
                          "loss_first": loss0, "loss_last": loss1}
    if args.three_phase_grid:
        nx, ny, nz = args.three_phase_grid
        s = synth.make_box(nx, ny, nz, 1.0, 1.0, 0.5, seed=21, sigma=2.5, nphase=3, wells="four", T_inj=500.0,
                           q_inj=4e-6).system()
    else:
        s = synth.recipe("three_phase2m").system()
    n, b = s["n"], s["b"]
    dofs = n * b
    alg = algorithmic_bytes(s)
    d = {k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in
         {"rp": s["row_ptr"], "ci": s["col_idx"], "vals": s["vals"].reshape(-1), "kind": s["unknown_kind"],
          "W": s["weights"].reshape(-1), "st": s["st"], "rhs": s["rhs"].reshape(-1)}.items()}
    del s
    peak, peak_kind = peaks()
    lines = {}
    x = torch.empty(dofs, dtype=torch.float64, device=dev)
    sols = {}
    out = {"dofs": dofs,
           "workload": (f"three-phase {n} cells, 4 unknowns/cell ({dofs} dofs)" if args.three_phase_grid else
                        "three_phase2m: 200x200x50 cells, 4 unknowns/cell (8M dofs)") +
                       ", lognormal permeability sigma 2.5, 4 injectors + 4 producers; CPTR + ILU(0), FGMRES(30), "
                       "rtol 1e-6",
           "training": dict(training, data="16 three-phase 32x32x8 grids (coupling drawn per grid), exact Schur "
                                           "diagonal ratios from the oracle")}
    # (name, options, network base, timed runs); the converging forms are autotuned at their untimed
    # first set-up; the A_TT forms stall on this workload, so they run once with a 200-step limit
    # and fixed launch shapes
    runs = (("fp64_se", dict(autotune=1), "se", None, 2),
            ("fp64_learned_se", dict(schur="learned", autotune=1), "se", "se", 2),
            ("mixed_learned_se", dict(schur="learned", precision="mixed", autotune=1), "se", "se", 2),
            ("fp64_att", dict(schur="att", max_it=200), None, None, 1),
            ("fp64_learned_att", dict(schur="learned", max_it=200), None, "att", 1))
    for name, opts, st_base, net, nrun in runs:
        if forms is not None and name not in forms:
            continue
        Sv = cp.Solver(stream=stream, **opts)
        if net:
            cp.cptr_set_mlp(Sv.ctx, nets[net])

        def step_v():
            Sv.setup(n, b, d["rp"], d["ci"], d["vals"], d["kind"], d["W"], d["st"] if st_base == "se" else None)
            return Sv.solve(d["rhs"], RTOL, x=x)[1]

        if nrun > 1:
            step_v()
        if name == "fp64_se":
            zt, wt = torch.zeros_like(x).normal_(), torch.empty_like(x)

            def spmv_and_precond():
                cp.cptr_apply_matrix(Sv.ctx, zt, wt)
                cp.cptr_apply_precond(Sv.ctx, zt, wt)
            profiled_range(args, "spmv_b4", spmv_and_precond)
        evs, infs = [], []
        for _ in range(nrun):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infs.append(step_v())
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(bb) for a, bb in evs) / len(evs)
        prof = cp.cptr_profile(Sv.ctx)
        solve_ms = statistics.mean(i["solve_ms"] for i in infs)
        out[name] = {"ms_per_step": round(ms, 3), "dofs_per_s": round(dofs / (ms / 1e3), 1),
                     "setup_ms": round(statistics.mean(i["setup_ms"] for i in infs), 3),
                     "solve_ms": round(solve_ms, 3), "solve_dofs_per_s": round(dofs / (solve_ms / 1e3), 1),
                     "iters": infs[-1]["iters"], "true_rel_res": infs[-1]["true_rel_res"],
                     "status": infs[-1]["status"], "schur_used": infs[-1]["schur_used"],
                     "learned_setup_ms": round(prof["setup_other"][0], 3), "timed_runs": nrun}
        sols[name] = x.cpu().numpy().copy()
        if name == "fp64_se":
            # b = 4 kernels on a working set far above L2: families and the finest V-cycle level
            fam, vc = profiled_pass(cp, Sv, step_v, flush, 1, 0xFF)
            kern, _ = family_kernels(cp, Sv, b, False)
            for f in ("spmv", "stage1_resid", "ilu_fwd", "ilu_bwd"):
                lines[f + "_b4"] = roofline_line(kern[f], alg[f], *fam[f], 1, peak, peak_kind,
                                                 PROFILED_TRAFFIC.get(f + "_b4"))
            lines.update(vcycle_lines(cp, Sv, vc, 1, peak, peak_kind, False, "_b4", PROFILED_TRAFFIC))
        Sv.close()
    out["rooflines_note"] = ("the b = 4 lines of the top-level rooflines come from the fp64_se solve of this "
                             "workload (one profiled step)")
    return out, sols, lines


NEWTON_RTOL, NEWTON_STEPS = 1e-8, 3


def newton_reservoir():
    """The Newton section's model: the cptr200k reservoir (100x100x20, layered permeability, 2 W/m/K,
    500 K injector) with 30-day implicit Euler steps."""
    import synth
    r = synth.recipe("cptr200k")
    r.dt = 30 * 86400.0
    return r


def newton_section(args, dev, stream):
    """Three implicit Euler steps on the device (cptr_newton: assembly, CPTR-FGMRES with the headline
    solver's options, line search), linear tolerance 1e-8 as in Sec. 4; per step the Newton and linear
    iterations and the GPU time (CUDA events)."""
    import torch

    import paper_1907_04229_gb300 as cp

    r = newton_reservoir()
    S = cp.Solver(stream=stream, autotune=1)
    cp.cptr_model_set(S.ctx, {k: (torch.as_tensor(np.ascontiguousarray(v), device=dev) if isinstance(v, np.ndarray)
                                  else v) for k, v in r.model_fields().items()})
    x = torch.as_tensor(np.ascontiguousarray(r.x0.reshape(-1)), device=dev)
    warm = x.clone()
    cp.cptr_newton(S.ctx, warm, x.clone(), NEWTON_RTOL, 20)   # tunes the launch shapes (cached)
    steps = []
    first_x = None
    for k in range(NEWTON_STEPS):
        xn = x.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = cp.cptr_newton(S.ctx, x, xn, NEWTON_RTOL, 20)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if k == 0:
            first_x = x.cpu().numpy().copy()
        steps.append({"step_ms": round(e0.elapsed_time(e1), 2), "newton_its": info["newton_its"],
                      "linear_its": info["linear_its"], "line_search_cuts": info["line_search_cuts"],
                      "status": info["status"], "res0": info["res0"], "res": info["res"],
                      "setup_ms": round(info["setup_ms"], 2), "solve_ms": round(info["solve_ms"], 2)})
    S.close()
    total_ms = sum(t["step_ms"] for t in steps)
    return {"workload": "cptr200k model (100x100x20, 600k dofs) with 30-day implicit Euler steps; Newton with "
                        "backtracking line search, tolerance 1e-8 (function and step norms), CPTR-FGMRES to 1e-8",
            "steps": steps, "ms_per_time_step": round(total_ms / NEWTON_STEPS, 2),
            "newton_its_per_step": sum(t["newton_its"] for t in steps) / NEWTON_STEPS,
            "linear_its_per_newton": sum(t["linear_its"] for t in steps) / max(1, sum(t["newton_its"] for t in steps))}, first_x


MESH_METHODS = (("CPR-AMG", dict(stage1="cpr")), ("CPR-AMG(TI)", dict(stage1="cpr", decouple="ti")),
                ("CPR-AMG-ILU(1)", dict(stage1="cpr", ilu_fill=1)), ("CPTR-Block(AMG)", dict(stage1="full")),
                ("CPTR-uAMG", dict(stage1="uamg")), ("CPTR-uAMG(TI)", dict(stage1="uamg", decouple="ti")))


def mesh_study(args, dev, stream):
    """The 2-D mesh-refinement study of Sec. 4.1.1 (Tables meshW, meshH, anisomeshW) on its synthetic
    analogues (synth.mesh_refinement_case): for N = 20 .. 640 and the paper's six methods, one
    Jacobian per case (the first Newton iterate of the first 10-day step), GMRES tolerance 1e-8 as in
    Sec. 4, FP64; iterations and GPU set-up and solve times (CUDA events, one untimed run first)."""
    import torch

    import synth
    import paper_1907_04229_gb300 as cp

    out = {"tolerance": 1e-8, "note": "one Jacobian per case (first Newton iterate of the first 10-day step), "
                                      "not the paper's average over Newton iterations of two steps"}
    Ns = [n for n in (20, 40, 80, 160, 320, 640) if n <= args.mesh_study_max_n]
    for kind in ("wells", "heaters", "aniso"):
        res = {m: {} for m, _ in MESH_METHODS}
        for N in Ns:
            s = synth.mesh_refinement_case(kind, N).system()
            d = {k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in
                 {"rp": s["row_ptr"], "ci": s["col_idx"], "vals": s["vals"].reshape(-1), "kind": s["unknown_kind"],
                  "W": s["weights"].reshape(-1), "st": s["st"], "rhs": s["rhs"].reshape(-1)}.items()}
            x = torch.empty(s["n"] * s["b"], dtype=torch.float64, device=dev)
            for name, opts in MESH_METHODS:
                S = cp.Solver(stream=stream, max_it=500, **opts)

                def run():
                    S.setup(s["n"], s["b"], d["rp"], d["ci"], d["vals"], d["kind"], d["W"], d["st"])
                    return S.solve(d["rhs"], 1e-8, x=x)[1]

                run()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = run()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                res[name][N] = {"iters": info["iters"], "status": info["status"], "setup_ms": round(info["setup_ms"], 2),
                                "solve_ms": round(info["solve_ms"], 2), "step_ms": round(e0.elapsed_time(e1), 2)}
                S.close()
        out[kind] = res
    return out


def small_section(args, dev, stream, flush):
    """The small plain-CPTR configuration: 16x16x4 cells (3072 dofs), FP64, two-level AMG (its
    coarsest level a dense inverse of a few hundred rows) + ILU(0), FGMRES(30) to 1e-8; set-up and
    solve timed like the headline step, the oracle's set-up + solve of the same system beside it,
    and the error against the oracle per unknown kind."""
    import torch

    import oracle
    import synth
    import paper_1907_04229_gb300 as cp
    s = synth.recipe("parity").system()
    n, b = s["n"], s["b"]
    d = {k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in
         {"rp": s["row_ptr"], "ci": s["col_idx"], "vals": s["vals"].reshape(-1), "kind": s["unknown_kind"],
          "W": s["weights"].reshape(-1), "st": s["st"], "rhs": s["rhs"].reshape(-1)}.items()}
    x = torch.empty(n * b, dtype=torch.float64, device=dev)
    S = cp.Solver(stream=stream, max_levels=2)

    def step():
        S.setup(n, b, d["rp"], d["ci"], d["vals"], d["kind"], d["W"], d["st"])
        return S.solve(d["rhs"], 1e-8, x=x)[1]

    for _ in range(max(args.warmup, 3)):
        step()
    evs, infs = [], []
    for _ in range(10):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infs.append(step())
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(bb) for a, bb in evs) / len(evs)
    lev = [L["n"] for L in S.hierarchy(0)]
    xg = x.cpu().numpy().copy()
    S.close()
    t0 = time.perf_counter()
    o = oracle.Oracle.from_system(s, max_levels=2)
    xo, io = o.solve(s["rhs"], 1e-8)
    osecs = time.perf_counter() - t0
    return {"workload": "16x16x4 cells (3072 dofs), two-phase thermal, FP64 CPTR, two-level AMG (dense coarsest "
                        "inverse) + ILU(0), FGMRES(30), rtol 1e-8",
            "ms_per_step": round(ms, 3), "dofs_per_s": round(n * b / (ms / 1e3), 1),
            "setup_ms": round(statistics.mean(i["setup_ms"] for i in infs), 3),
            "solve_ms": round(statistics.mean(i["solve_ms"] for i in infs), 3), "iters": infs[-1]["iters"],
            "levels_p": lev, "status": infs[-1]["status"],
            "error_vs_fp64_oracle": errors_per_kind(xg, xo, b), "oracle_iters": int(io["iters"]),
            "cpu_baseline": {"value": round(n * b / osecs, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"one set-up + solve by the serial FP64 C oracle, {osecs * 1e3:.1f} ms"}}


def tp_dofs(tp):
    return tp["dofs"]


def ensemble(args, dev, stream, flush):
    """The ensemble workload: 64 two-phase instances with sizes from 20k to 430k cells (4M cells,
    12M dofs in total), mixed-precision CPTR, rtol 1e-6 per instance, set up and solved as one
    batch (one captured graph per Arnoldi step for all instances) with autotuned launch shapes;
    and, for comparison, the same instances set up and solved one after another with the
    single-system calls."""
    import torch

    import synth
    import paper_1907_04229_gb300 as cp

    shapes = synth.ensemble_sizes(total=args.ensemble_total, lo=min(20e3, args.ensemble_total / 64))
    systems = [synth.ensemble_member(k, sh).system() for k, sh in enumerate(shapes)]
    b = systems[0]["b"]
    kind = torch.as_tensor(systems[0]["unknown_kind"], device=dev)
    inst, rhs = [], []
    for s in systems:
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
        inst.append(dict(n_cells=s["n"], row_ptr=t(s["row_ptr"]), col_idx=t(s["col_idx"]), vals=t(s["vals"].reshape(-1)),
                         row_weights=t(s["weights"].reshape(-1)), st_vals=t(s["st"])))
        rhs.append(t(s["rhs"].reshape(-1)))
    cells = [s["n"] for s in systems]
    dofs = sum(cells) * b
    del systems
    xs = [torch.empty_like(r) for r in rhs]
    opts = dict(precision="mixed", autotune=1)
    S = cp.Solver(stream=stream, **opts)

    def step():
        S.setup_batch(b, inst, kind)
        return S.solve_batch(rhs, RTOL, x=xs)

    step()
    evs, res = [], []
    for _ in range(2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res.append(step())
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(bb) for a, bb in evs) / len(evs)
    _, status, infos = res[-1]
    its = [i["iters"] for i in infos]
    sols = {k: xk.cpu().numpy().copy() for k, xk in enumerate(xs)}
    out = {"instances": len(cells), "total_cells": sum(cells),
           "workload": f"{len(cells)} two-phase instances (3 unknowns/cell), {min(cells)}..{max(cells)} cells, "
                       f"{sum(cells)} cells / {dofs} dofs in total, mixed-precision CPTR + ILU(0), FGMRES(30), "
                       "rtol 1e-6 per instance",
           "batched": {"ms_per_step": round(ms, 3), "dofs_per_s": round(dofs / (ms / 1e3), 1),
                       "setup_ms": round(infos[0]["setup_ms"], 3), "solve_ms": round(infos[0]["solve_ms"], 3),
                       "status": status, "iters_min": min(its), "iters_median": int(np.median(its)),
                       "iters_max": max(its), "max_true_rel_res": max(i["true_rel_res"] for i in infos),
                       "levels": [infos[0]["levels_p"], infos[0]["levels_T"]],
                       "autotuned_shapes": [list(r) for r in cp.cptr_tuning(S.ctx)]}}
    S.close()
    # the same instances one after another through the single-system calls
    Sq = cp.Solver(stream=stream, **opts)

    def seq():
        inf = []
        for I, r, x in zip(inst, rhs, xs):
            Sq.setup(I["n_cells"], b, I["row_ptr"], I["col_idx"], I["vals"], kind, I["row_weights"], I["st_vals"])
            inf.append(Sq.solve(r, RTOL, x=x)[1])
        return inf

    seq()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    inf = seq()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = e0.elapsed_time(e1)
    its_s = [i["iters"] for i in inf]
    out["sequential"] = {"ms_per_step": round(ms_seq, 3), "dofs_per_s": round(dofs / (ms_seq / 1e3), 1),
                         "setup_ms": round(sum(i["setup_ms"] for i in inf), 3),
                         "solve_ms": round(sum(i["solve_ms"] for i in inf), 3),
                         "iters_min": min(its_s), "iters_median": int(np.median(its_s)), "iters_max": max(its_s),
                         "all_converged": all(i["status"] == "CPTR_OK" for i in inf)}
    out["speedup_batched_vs_sequential"] = round(ms_seq / ms, 3)
    Sq.close()
    return out, sols


def reference(args, rank, world):
    if rank != 0:
        return
    import synth
    s = synth.recipe(WORKLOAD).system()
    dofs = s["n"] * s["b"]
    for _ in range(args.warmup):
        oracle_step(s)
    total = 0.0
    for _ in range(args.steps):
        secs, info, _x = oracle_step(s)
        total += secs
    value = dofs * args.steps / total
    sample = f"one full setup+solve of the {WORKLOAD} workload per step, serial FP64 C oracle, {info['iters']} iterations"
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "cptr200k: 100x100x20 cells, 3 unknowns/cell (600k dofs), CPTR + ILU(0), "
                                  "FGMRES(30), rtol 1e-6, FP64", "step": "setup + solve"},
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------------------
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(total_ms_local, world, dofs_per_rank, steps, dev):
    """Whole-job throughput of independent replicas: every rank solved `steps` systems of
    `dofs_per_rank` unknowns; the job took the slowest rank's time.  Returns (dofs/s, ms/step)."""
    total_ms = allreduce_max(total_ms_local, world, dev)
    return world * dofs_per_rank * steps / (total_ms / 1e3), total_ms / steps


def allreduce_max(v, world, dev):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    if args.impl == "reference":
        reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    # the oracle's reference solutions run in spawned worker processes, started before any GPU call
    pool, jobs = start_oracle_jobs(args) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else (None, {})
    import __graft_entry__
    __graft_entry__.build()
    ours(args, rank, world, local_rank, jobs)
    if pool is not None:
        pool.terminate()
        pool.join()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
