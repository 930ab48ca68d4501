"""Benchmark: w-corrected visibilities/s (degrid + grid) of the GB300
w-stacking w-projection operator on the MWA-like snapshot workload
(2048^2 image, 4096^2 grid, FOV 25 deg, 1.95M visibilities, 8 k-means
w-stacks, conjugate fold, FP32 with FP64 chirp phase, quadrature tol 1e-6).

One step = one y = Phi x (phi_degrid) plus one x = Re(Phi^H y) (phi_grid)
over every visibility, i.e. every stage of the hot path: per stack S~_k/Z,
cuFFT, fused w-kernel quadrature + degridding, fused quadrature + gridding,
inverse cuFFT, crop/chirp/sum.  The plan (fold, Algorithm 1, sort) is built
once per observation and timed separately; the e2e figure includes it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank runs an
independent replica of the workload (the operator of one observation does
not shard across GPUs here) and `value` sums their visibilities over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "w-corrected visibilities/s (degrid+grid) at <=1e-5 rel err vs FP64; p50/p99 latency"
UNIT = "vis/s"
FLOPS_PER_TAP_NODE = 36.0     # J0 by a rational/asymptotic approximation (28) + 2 weighted complex MACs (8)
FP32_LANES_PER_SM = 128       # FP32 FMA lanes per SM per clock (Blackwell)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64, nominal
RADIAL_POINTS = 16            # Chebyshev points per piece, FP32 radial mode
RADIAL_FLOPS_PER_TAP = 96     # 15 Clenshaw steps x (2 FMA + 2 subtractions) + the last step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mwa",
                    choices=["mwa", "serve", "plan", "precision", "diff", "dde"],
                    help="mwa: the headline operator benchmark; serve: the serving stream; "
                         "plan: Algorithm 1 and the fold at the paper's scale")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="offered load of the Poisson stream as a fraction of the measured capacity")
    ap.add_argument("--serve-kernel-mode", default="quadrature", choices=["quadrature", "radial"],
                    help="kernel mode of every request in the serving stream")
    ap.add_argument("--serve-full-scale", type=int, default=1,
                    help="append the 126.6M-visibility request to the serving stream")
    ap.add_argument("--support-rule", default="stack", choices=["stack", "vis"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cycles-per-panel", type=float, default=0.0,
                    help="a-priori quadrature panel width in integrand cycles (0: library default)")
    ap.add_argument("--kernel-mode", default="quadrature", choices=["quadrature", "table", "radial"],
                    help="quadrature: every tap integrated (the hot path); table: pre-sampled "
                         "1-D w-planes with bilinear interpolation (Sec. 5.1.1)")
    ap.add_argument("--table-tol", type=float, default=1e-4)
    ap.add_argument("--tile", type=int, default=32, help="uv tile side of the visibility sort")
    ap.add_argument("--grid-staging", type=int, default=None, choices=[0, 1, 2],
                    help="table path: 0 one warp per visibility, 1 uv tiles staged in shared "
                         "memory, 2 w-rows of the table staged in shared memory (default 2 "
                         "with --kernel-mode table, else 0)")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"],
                    help="f32: FP32 path with FP64 chirp phase, quadrature tol 1e-6 (the "
                         "headline); f64: everything in FP64, quadrature tol 1e-12")
    ap.add_argument("--grid-deterministic", type=int, default=0, choices=[0, 1],
                    help="1: gridding sums in 64-bit fixed point (the same bits on every "
                         "run); 0: FP atomics (the default)")
    ap.add_argument("--no-det-check", action="store_true",
                    help="skip the deterministic-gridding comparison of the default run")
    ap.add_argument("--no-serve-check", action="store_true",
                    help="skip the short FP32/FP64 serving stream of the default run")
    ap.add_argument("--max-vis", type=int, default=0,
                    help="use only the first N visibilities (small profiling case)")
    args = ap.parse_args()
    if args.grid_staging is None:
        args.grid_staging = 2 if args.kernel_mode == "table" else 0
    elif args.grid_staging and args.kernel_mode != "table":
        ap.error("--grid-staging applies to --kernel-mode table only")
    return args


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    """The largest value over all ranks (the slowest rank's time)."""
    if ws == 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(ms_step_local, n_units_local, ws):
    """Whole-job throughput of N independent replicas: the units all ranks
    processed over the slowest rank's step time.  Returns (value, ms)."""
    ms = max_over_ranks(ms_step_local, ws)
    if ws > 1:
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(n_units_local)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        n_total = float(t.item())
    else:
        n_total = float(n_units_local)
    return n_total / (ms / 1e3), ms


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="phi_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        os.remove(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def device_sms(dev=None):
    """Streaming multiprocessors of the device, as the driver reports them."""
    return torch.cuda.get_device_properties(dev if dev is not None else
                                            torch.cuda.current_device()).multi_processor_count


def fp32_peak_tflops(sms, sm_mhz):
    """FP32 FMA peak: SMs x 128 FP32 lanes x 2 flops x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("phi_ops.cu", "bessel_j0.cuh", "phi_internal.cuh", "table_index.cuh",
              "fixed_point.cuh"):
        with open(os.path.join(ROOT, "paper_1903_06555_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(stage):
    """DRAM bytes per launch of the fused kernel from the committed ncu launch
    list, or None when the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "vis_kernel_mwa-2048-8stack_launches.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        key = line.strip().split(":")[0]
        if ":" in line and (key == "kernel_source_sha256" or key.startswith("traffic_bytes_per_launch_")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    v = vals.get(f"traffic_bytes_per_launch_{stage}")
    return float(v) if v else None


def profiled_pipes():
    """FMA-pipe and issue-slot activity of the fused degrid kernel from the
    committed small-case ncu capture, or None when the kernel sources changed
    since it was taken."""
    p = os.path.join(ROOT, "profiles", "vis_kernel_degrid_mwa-2048-first40000_full.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    keys = ("fma_pipe_pct", "fma_heavy_pipe_pct", "issue_active_pct", "warp_inst_per_tap_node")
    out = {k: float(vals[k]) for k in keys if k in vals}
    out["source"] = "profiles/vis_kernel_degrid_mwa-2048-first40000_full.md (40,000-visibility case)"
    return out


def profiled_fp64():
    """DP flops per tap-node and FP64-pipe activity of vis_kernel<double> from
    the committed small-case ncu capture, or None when the kernel sources
    changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "vis_kernel_f64_degrid_mwa-2048-first2000.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    keys = ("fp64_flops_per_tap_node", "fp64_pipe_pct", "issue_active_pct")
    out = {k: float(vals[k]) for k in keys if k in vals}
    out["source"] = "profiles/vis_kernel_f64_degrid_mwa-2048-first2000.md"
    return out


def load_oracle_counts():
    p = os.path.join(ROOT, "tests", "golden", "mwa_oracle_evals.json")
    with open(p) as f:
        return json.load(f)


def covered_grid_cells(uvw_np, info, conj_fold):
    """Distinct grid cells that the J_w x J_w boxes of the kept visibilities
    cover, summed over the stacks: the grid part of a launch's minimum HBM
    traffic (each such cell is read, or written, at least once).  Host-side
    from the plan's own centres and supports: fold to w >= 0, nearest centre
    (first on ties), drop outside [-Npad/2, Npad/2), box from
    floor(u/du) - J_w/2 + 1, circular."""
    import scipy.ndimage as nd
    u, v, w = (np.array(uvw_np[:, i], np.float64) for i in range(3))
    if conj_fold:
        f = w < 0
        u[f], v[f], w[f] = -u[f], -v[f], -w[f]
    npad, du = int(info["npad"]), float(info["du"])
    wbar = np.asarray(info["wbar"], np.float64)
    jw = np.asarray(info["jw"], np.int64)
    stack = np.argmin(np.abs(w[:, None] - wbar[None, :]), axis=1)
    up, vp = u / du, v / du
    keep = (up >= -npad / 2) & (up < npad / 2) & (vp >= -npad / 2) & (vp < npad / 2)
    total = 0
    for k in range(len(wbar)):
        sel = keep & (stack == k)
        if not sel.any():
            continue
        J = int(jw[k])
        q0u = (np.floor(up[sel]).astype(np.int64) - J // 2 + 1) % npad
        q0v = (np.floor(vp[sel]).astype(np.int64) - J // 2 + 1) % npad
        m = np.zeros((npad, npad), np.uint8)
        m[q0v, q0u] = 1
        for ax in (0, 1):
            m = nd.maximum_filter1d(m, size=J, axis=ax, mode="wrap", origin=(J - 1) // 2)
        total += int(np.count_nonzero(m))
    return total


def flush_l2(buf):
    buf.add_(1.0)   # 256 MiB read-modify-write: larger than the 129 MB L2


def workload_inputs(wl):
    uvw = W.uvw_for(wl)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    return uvw, x


# ---------------------------------------------------------------------------- reference arm

def cpu_oracle_rate(wl, uvw, x, budget_s=20.0, tol=1e-6, rate_tol12=False):
    """The FP64 oracle, as it stands, on the host cores: degrid of a bounded
    random sample of the workload's kept visibilities in chunks (per-stack
    grids built before the clock starts), gridding of the same sample in one
    call, plus one stack's image-domain steps (S~, pad, FFT forward; inverse
    FFT, crop, S~^H) and one padded-grid allocation timed once and charged
    K times.  Returns (vis/s projected to the full workload,
    sampled visibilities, measured seconds, threads, rate at tol 1e-12), the
    last (with rate_tol12=True) the same projection for the oracle at the
    parity tolerance 1e-12, timed on 64 kept visibilities of the
    widest-support stack."""
    import oracle as O
    geo = O.geometry_from(wl, tol_rel=tol, tol_abs=tol)
    plan = O.make_plan(uvw, geo, wl.n_stacks, wl.conj_fold)
    kept = np.nonzero(~plan.dropped)[0]
    order = np.random.default_rng(3).permutation(kept)
    t0 = time.perf_counter()
    g0 = O.stack_grids(plan, x, [0])
    O.image_from_grids(plan, g0)
    t_image = time.perf_counter() - t0
    grids = O.stack_grids(plan, x)
    y = W.random_vis(len(uvw), 9)
    threads = len(os.sched_getaffinity(0))
    # degrid in chunks for half the budget; the oracle degrids a chunk stack
    # by stack, spreading each stack's share over its OpenMP threads 4
    # visibilities at a time, so a chunk holds 4 per thread per stack
    min_chunk = 4 * threads * wl.n_stacks
    n_done, t_deg, chunk = 0, 0.0, min_chunk
    vis_budget = max(2.0, budget_s - t_image)
    while t_deg < vis_budget / 2 and n_done < len(order):
        sel = np.sort(order[n_done:n_done + chunk])
        t0 = time.perf_counter()
        O.degrid_from_grids(plan, grids, sel)
        t_deg += time.perf_counter() - t0
        n_done += sel.size
        chunk = int(max(min_chunk, min(n_done / t_deg * (vis_budget / 2 - t_deg), 4096)))
    # grid the same visibilities in one call; its per-stack grids are
    # allocated and zeroed once, as in a whole-workload run, so that cost is
    # timed apart and charged once per stack rather than per visibility
    sel = np.sort(order[:n_done])
    t0 = time.perf_counter()
    O.grid_to_stacks(plan, y[sel], sel)
    t_grid = time.perf_counter() - t0
    stacks = sorted(set(int(k) for k in plan.stack[sel]))
    t0 = time.perf_counter()
    for _ in stacks:
        np.zeros((geo.Npad, geo.Npad), np.complex128)
    t_alloc = (time.perf_counter() - t0) / max(1, len(stacks))
    t_used = t_deg + max(t_grid - len(stacks) * t_alloc, 0.0)
    t_full = t_used * (kept.size / n_done) + wl.n_stacks * (t_image + t_alloc)
    acc = None
    if rate_tol12:
        k = int(np.argmax([plan.jw[kept][plan.stack[kept] == s].max(initial=0)
                           for s in range(wl.n_stacks)]))
        sel = np.sort(order[plan.stack[order] == k][:64])
        t0 = time.perf_counter()
        O.degrid_from_grids(plan, grids, sel, 1e-12, 1e-12)
        O.grid_to_stacks(plan, y[sel], sel, 1e-12, 1e-12)
        t12 = max(time.perf_counter() - t0 - t_alloc, 1e-9)   # one stack's grid allocation
        acc = kept.size / (t12 * kept.size / sel.size + wl.n_stacks * (t_image + t_alloc))
    return kept.size / t_full, n_done, t_deg + t_grid + t_image, threads, acc


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = W.mwa_snapshot()
    uvw, x = workload_inputs(wl)
    per_step = []
    n_tot = 0
    rates = []
    for s in range(args.warmup + args.steps):
        rate, n, t, threads, _ = cpu_oracle_rate(wl, uvw, x, budget_s=8.0)
        if s >= args.warmup:
            per_step.append((n, t))
            rates.append(rate)
            n_tot = n
    tot_t = sum(t for _, t in per_step)
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "image_n": wl.image_n, "n_stacks": wl.n_stacks,
                       "quad_tol": 1e-6, "sample_per_step": n_tot},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n_tot} random kept visibilities per step, degrid+grid, "
                                       "FP64 oracle at quadrature tol 1e-6, plus one stack's "
                                       "image-domain steps charged per stack; projected to the "
                                       "full workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- our arm

def run_ours(args, ws, rank, local):
    import paper_1903_06555_gb300 as phi
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = W.mwa_snapshot(seed=0)
    uvw_np, x_np = workload_inputs(wl)
    if args.max_vis:
        uvw_np = np.ascontiguousarray(uvw_np[:args.max_vis])
    M = len(uvw_np)
    desc = dict(image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg), oversample=wl.oversample,
                support=wl.support, n_stacks=wl.n_stacks, conj_fold=int(wl.conj_fold),
                precision=args.precision, support_rule=args.support_rule,
                cycles_per_panel=args.cycles_per_panel, kernel_mode=args.kernel_mode,
                table_tol=args.table_tol, tile=args.tile, grid_staging=args.grid_staging,
                grid_deterministic=args.grid_deterministic)
    f64 = args.precision == "f64"
    quad_tol = 1e-12 if f64 else 1e-6
    desc.update(quad_rel_tol=quad_tol, quad_abs_tol=quad_tol)
    rdt, cdt = (torch.float64, torch.complex128) if f64 else (torch.float32, torch.complex64)
    stream = torch.cuda.current_stream()
    uvw = torch.from_numpy(uvw_np).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = phi.Plan(uvw, **desc)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    info = plan.info()
    n_kept = info["n_kept"]
    x = torch.from_numpy(x_np).to(dev, rdt)
    y_obs = plan.degrid(x)
    rms = torch.sqrt(torch.mean(torch.abs(y_obs) ** 2)).item()
    noise = torch.from_numpy(W.complex_noise(M, 0.01 * rms, 0)).to(dev, cdt)
    y_obs = y_obs + noise
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        y = plan.degrid(x)
        d = plan.grid(y_obs)
        return y, d

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.stats_full(reset=True)
    plan.timings(reset=True)
    plan.set_timing(True)
    times = []
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_id = vis.split(",")[torch.cuda.current_device()] if vis else str(torch.cuda.current_device())
    with ClockSampler(gpu_id) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush_l2(flush)
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(ws)
    plan.set_timing(False)
    times = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    stages = plan.timings(reset=True)
    bad, taps, tap_nodes = plan.stats_full(reset=True)
    ms_step = sum(times) / len(times)
    value, ms_step_max = aggregate_value(ms_step, n_kept, ws)
    lat = sorted(times)
    p50 = statistics.median(lat)
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    table_info = radial_info = None
    if args.kernel_mode != "quadrature":
        qdesc = dict(desc, kernel_mode="quadrature", grid_staging=0)
        qplan = phi.Plan(uvw, **qdesc)
        yq = qplan.degrid(x)
        yt = plan.degrid(x)
        qplan.close()
        rel_q = float(torch.linalg.vector_norm(yt - yq) / torch.linalg.vector_norm(yq))
        if args.kernel_mode == "table":
            table_info = {"table_tol": args.table_tol, "n_rho": info["table_n_rho"],
                          "n_w": info["table_n_w"], "h_rho": info["table_h_rho"],
                          "h_w": info["table_h_w"],
                          "bytes": 16 * info["table_n_rho"] * (info["table_n_w"] - 1),
                          "rel_l2_vs_quadrature_path": rel_q}
        else:
            radial_info = {"piece_width_px": 2.0 / info["window_radius"],
                           "points_per_piece": RADIAL_POINTS,
                           "quadrature_points_per_vis": tap_nodes / (2 * args.steps * n_kept),
                           "rel_l2_vs_quadrature_path": rel_q}

    # deterministic gridding beside the default: the same phi_grid call on a
    # plan with 64-bit fixed-point grid sums, timed the same way, its bits
    # compared across two calls and its image against the FP-atomic one
    det_info = None
    if not (args.grid_deterministic or args.no_det_check) and args.kernel_mode == "quadrature":
        dplan = phi.Plan(uvw, **dict(desc, grid_deterministic=1))

        def grid_ms(pl, reps=3):
            out = []
            for _ in range(reps):
                flush_l2(flush)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.grid(y_obs)
                e1.record(stream)
                torch.cuda.synchronize()
                out.append(e0.elapsed_time(e1))
            return sum(out) / len(out)

        d1 = dplan.grid(y_obs)
        d2 = dplan.grid(y_obs)
        dref = plan.grid(y_obs)
        det_info = {"grid_call_ms": grid_ms(dplan), "fp_atomic_grid_call_ms": grid_ms(plan),
                    "bitwise_repeatable": bool(torch.equal(d1, d2)),
                    "rel_l2_vs_fp_atomic": float(torch.linalg.vector_norm((d1 - dref).double()) /
                                                 torch.linalg.vector_norm(dref.double()))}
        dplan.close()
        del d1, d2, dref

    # roofline: the dominant kernel (fused quadrature + degrid or + grid)
    counts = load_oracle_counts()
    evals_per_vis = counts["evals_per_vis_mean"]
    dom = max(("degrid", "grid"), key=lambda s: stages[s][0])
    ms_dom, n_dom = stages[dom]
    launches_per_step = n_dom / args.steps
    # algorithmic flops of one step's dominant-stage launches = all kept vis
    flops_step = n_kept * evals_per_vis * FLOPS_PER_TAP_NODE
    achieved = flops_step / launches_per_step / ((ms_dom / n_dom) / 1e3) / 1e12
    peaks = measured_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    sms = device_sms(dev)
    peak_fp32 = fp32_peak_tflops(sms, sm_mhz)
    clocks = clk.summary()
    if args.kernel_mode == "table":
        # HBM bytes one launch (all stacks of the resident group) must move at
        # least: records + permutation + visibility per visibility, the
        # covered grid cells once, the plane pairs once
        cnt = np.array(info["counts"], float)
        cells = covered_grid_cells(uvw_np, info, desc.get("conj_fold", 0))
        table_b = 16.0 * info["table_n_rho"] * (info["table_n_w"] - 1)
        groups = max(1, int(round(launches_per_step)))
        bytes_step = float(cnt.sum()) * (32 + 4 + 8) + 8.0 * cells + groups * table_b
        ach_gbs = bytes_step / launches_per_step / ((ms_dom / n_dom) / 1e3) / 1e9
        hbm = peaks.get("hbm_gbs", 6800.0)
        tname = {0: "vis_table_kernel", 1: "tile_table_kernel", 2: "row_table_kernel"}[args.grid_staging]
        roof = {"bound": "hbm", "kernel": f"{tname} ({dom})", "achieved": ach_gbs,
                "peak": hbm, "unit": "GB/s", "frac": ach_gbs / hbm,
                "traffic": profiled_traffic("table_" + dom) if args.grid_staging == 2 else None,
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "covered_grid_cells": cells,
                "work_note": "records 32 B + permutation 4 B + visibility 8 B per visibility, "
                             "8 B per grid cell covered by a kernel box, the plane pairs once "
                             "per launch; the kernel is bound by its shared-memory reads (L1/TEX "
                             "86-94% busy in ncu for the w-row kernel), far below the HBM roofline"}
    elif args.kernel_mode == "radial":
        # executed work: the quadrature at the Chebyshev points (tap-nodes) and
        # the series evaluated at every tap; degrid and grid do the same work
        per_launch = (tap_nodes * FLOPS_PER_TAP_NODE + taps * RADIAL_FLOPS_PER_TAP) / (2.0 * n_dom)
        ach = per_launch / ((ms_dom / n_dom) / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": f"vis_radial_kernel ({dom})", "achieved": ach,
                "peak": peak_fp32, "unit": "TFLOP/s", "frac": ach / peak_fp32,
                "traffic": profiled_traffic("radial_" + dom),
                "peak_note": f"FP32 FMA: {sms} SMs (device count) x {FP32_LANES_PER_SM} lanes x 2 flops x "
                             f"{sm_mhz:.0f} MHz (recipe unit counts, max clock)",
                "work_note": f"{FLOPS_PER_TAP_NODE:.0f} flops per quadrature tap-node at the "
                             f"Chebyshev points + {RADIAL_FLOPS_PER_TAP} flops per tap for its "
                             "series (executed work, not the oracle's per-tap count)"}
    elif f64:
        # FP64 path: DP flops per tap-node from the committed ncu capture of
        # vis_kernel<double> (its DFMA/DMUL/DADD counts over the tap-nodes of
        # the captured launch) x this run's tap-nodes, against the FP64 peak
        gpu_nodes = tap_nodes / (2 * args.steps * n_kept)
        prof = profiled_fp64()
        peak64 = FP64_NOMINAL_TFLOPS * sms / 152.0 * sm_mhz / 2070.0
        ach = None
        if prof and "fp64_flops_per_tap_node" in prof:
            ach = n_kept * gpu_nodes * prof["fp64_flops_per_tap_node"] / launches_per_step / \
                ((ms_dom / n_dom) / 1e3) / 1e12
        roof = {"bound": "fp64", "kernel": f"vis_kernel<double> ({dom})", "achieved": ach,
                "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64 if ach else None,
                "traffic": None, "ncu": prof,
                "peak_note": f"nominal FP64 {FP64_NOMINAL_TFLOPS} TFLOP/s at 152 SMs, 2070 MHz, "
                             f"scaled to {sms} SMs and {sm_mhz:.0f} MHz (no measured FP64 peak)",
                "work_note": f"{gpu_nodes:.0f} tap-nodes per visibility (GK 15/31 at tol 1e-12) "
                             "x the DP flops per tap-node counted by ncu"}
    else:
        # executed work: the tap-nodes this run's launches evaluated (counted
        # on the device, refinements included) x the flops of one tap-node
        gpu_nodes = tap_nodes / (2 * args.steps * n_kept)
        ex = n_kept * gpu_nodes * FLOPS_PER_TAP_NODE / launches_per_step / \
            ((ms_dom / n_dom) / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": f"vis_kernel ({dom})", "achieved": ex,
                "peak": peak_fp32, "unit": "TFLOP/s", "frac": ex / peak_fp32,
                "traffic": profiled_traffic(dom),
                "peak_note": f"FP32 FMA: {sms} SMs (device count) x {FP32_LANES_PER_SM} lanes x 2 flops x "
                             f"{sm_mhz:.0f} MHz (recipe unit counts, max clock)",
                "work_note": f"{FLOPS_PER_TAP_NODE:.0f} flops per tap-node x the tap-nodes the "
                             f"launch evaluated ({gpu_nodes:.0f} per visibility, Gauss-Kronrod "
                             "15/31 on shared equal panels, refinements included)",
                # the same flops over the oracle's own count (globally adaptive
                # GK 7/15 per tap at tol 1e-6): credits the quadrature schedule
                # as well as the kernel, so it can exceed the peak
                "oracle_work": {"tap_nodes_per_vis": evals_per_vis, "achieved": achieved,
                                "frac": achieved / peak_fp32}}
        roof["ncu"] = profiled_pipes()
    if roof["traffic"]:
        # HBM moved per launch (committed ncu figure) over this run's launch time
        gbs = roof["traffic"] / ((ms_dom / n_dom) / 1e3) / 1e9
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        roof["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak}

    # end to end through the public API from pinned host buffers
    e2e = run_e2e(phi, desc, uvw_np, x_np, args.e2e_steps, dev) if args.e2e_steps > 0 else None

    # a short serving stream through the serving engine, FP32 and FP64 on the
    # same requests (the full stream is --workload serve)
    serving = None
    if not args.no_serve_check and not args.max_vis and rank == 0:
        from paper_1903_06555_gb300 import serve as S
        serving = {"stream": "6 observations of 5e4-1.5e5 visibilities, 512^2-1024^2 images, "
                             "|w|max 50-3000, arriving together; 4 slots; degrid + grid each"}
        for prec in ("f32", "f64"):
            reqs = serve_requests(6, seed=11, mmin=5e4, mmax=1.5e5, sizes=(512, 1024),
                                  precision=prec)
            for r in reqs:
                r.raise_stacks = True
            with S.Server(150 * 10 ** 9, slots=4) as srv:
                serving[prec] = S.summarize(srv.run_stream(reqs, realtime=False), t_first=0.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": wl.name + (f"-first{M}" if args.max_vis else ""), "image_n": wl.image_n, "npad": info["npad"],
                   "fov_deg": wl.fov_deg, "n_vis": M, "n_kept": n_kept,
                   "n_dropped": info["n_dropped"], "n_stacks": wl.n_stacks, "conj_fold": wl.conj_fold,
                   "support": wl.support, "support_rule": args.support_rule,
                   "jw_per_stack": info["jw"], "quad_tol": quad_tol, "l2": "flushed (256 MiB write) between steps",
                   "grid_deterministic": args.grid_deterministic,
                   "parallelism": f"replicas x{ws}"},
        "latency_ms": {"p50": p50, "p99": p99, "min": lat[0], "max": lat[-1]},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "plan_ms": plan_ms,
        "kmeans_sweeps": info["kmeans_sweeps"],
        "quadrature": {"taps_per_step": taps / args.steps, "unconverged_taps": bad,
                       "gpu_tap_nodes_per_vis": tap_nodes / (2 * args.steps * n_kept),
                       "oracle_tap_nodes_per_vis_tol1e-6": evals_per_vis},
        "roofline": roof,
        "kernel_mode": args.kernel_mode,
        "table": table_info,
        "radial": radial_info,
        "deterministic_grid": det_info,
        "e2e": e2e,
        "serving": serving,
        # this library's kernels in the timed steps (prep, fused degrid, fused
        # grid, finish: one each per stack group; with deterministic gridding
        # also the term bound, the exponent and the fixed-point conversion of
        # each grid launch); cuFFT's and the memsets are not counted
        "gpu_launches": int(sum(stages[k][1] for k in ("prep", "degrid", "grid", "finish")) +
                            (3 * stages["grid"][1] if args.grid_deterministic else 0)),
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        rate, n, t, threads, rate12 = cpu_oracle_rate(wl, uvw_np, x_np, budget_s=20.0,
                                                      rate_tol12=not args.max_vis)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{n} random kept visibilities of the workload, degrid+grid, "
                                          f"FP64 oracle at quadrature tol 1e-6, plus one stack's "
                                          f"image-domain steps charged per stack ({t:.1f} s "
                                          "measured); projected to the full workload"}
        if rate12 is not None:
            line["cpu_baseline"]["value_tol1e-12"] = rate12
        if not args.max_vis:
            line["accuracy_vs_fp64_oracle"] = accuracy_vs_oracle(plan, x, uvw_np, wl, dev, cdt)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def accuracy_vs_oracle(plan, x, uvw_np, wl, dev, cdt=torch.complex64):
    """This run's FP32 results (the full plan, the timed launch configuration)
    against the FP64 oracle at quadrature tolerance 1e-12, from
    tests/golden/mwa_dense_cells.npz (written from oracle/ alone by
    tests/golden/make_dense_cells.py): degrid values of 2,000 kept
    visibilities, 250 per stack; and, per stack, the image gridded from a
    visibility vector that is zero except on the visibilities covering that
    stack's busiest grid cell, which they fill to its full-run density
    (960 to 2,552 contributions), then all stacks together."""
    import oracle as O
    g = np.load(os.path.join(ROOT, "tests", "golden", "mwa_dense_cells.npz"))
    geo = O.geometry_from(wl, tol_rel=1e-12, tol_abs=1e-12)
    full = O.make_plan(uvw_np, geo, wl.n_stacks, wl.conj_fold)
    M = len(uvw_np)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    y32 = plan.degrid(x).cpu().numpy().astype(np.complex128)
    s = g["sample_sel"]
    deg = [rel(y32[s][full.stack[s] == k], g["sample_y_ref"][full.stack[s] == k])
           for k in range(wl.n_stacks)]
    sel = g["dense_sel"]
    y_in = W.random_vis(M, int(g["vis_seed"]))
    grid_k, img_sum, ref_sum = [], 0.0, 0.0
    for k in range(wl.n_stacks):
        pick = sel[full.stack[sel] == k]
        ym = np.zeros(M, np.complex128)
        ym[pick] = y_in[pick]
        img = plan.grid(torch.from_numpy(ym).to(dev, cdt)).cpu().numpy().astype(np.float64)
        J = int(g["stack_jw"][k])
        v0, u0 = (int(t) for t in g[f"dense_patch_origin_{k}"])
        grid = np.zeros((geo.Npad, geo.Npad), np.complex128)
        grid[np.ix_(np.arange(v0, v0 + 2 * J - 1) % geo.Npad,
                    np.arange(u0, u0 + 2 * J - 1) % geo.Npad)] = g[f"dense_patch_{k}"]
        ref = O.image_from_grids(full, {k: grid})
        grid_k.append(rel(img, ref))
        img_sum = img_sum + img
        ref_sum = ref_sum + ref
    return {"degrid_rel_l2": rel(y32[s], g["sample_y_ref"]), "degrid_rel_l2_max_stack": max(deg),
            "degrid_rel_l2_per_stack": deg,
            "grid_rel_l2": rel(img_sum, ref_sum), "grid_rel_l2_max_stack": max(grid_k),
            "grid_rel_l2_per_stack": grid_k,
            "bound": 1e-10 if cdt == torch.complex128 else 1e-5,
            "sample": f"degrid: {s.size} kept visibilities, {s.size // wl.n_stacks} per stack; "
                      f"grid: {sel.size} visibilities covering each stack's busiest cell "
                      f"({int(g['dense_count'].min())}-{int(g['dense_count'].max())} "
                      "contributions, the full-run count); oracle at quadrature tol 1e-12 "
                      "(tests/golden/mwa_dense_cells.npz)"}


def run_e2e(phi, desc, uvw_np, x_np, steps, dev):
    """Public-API round trip per step: pinned host uvw + image -> device,
    plan build (fold, Algorithm 1, sort), degrid, grid, results -> host."""
    f64 = desc.get("precision") == "f64"
    rdt, cdt = (torch.float64, torch.complex128) if f64 else (torch.float32, torch.complex64)
    uvw_h = torch.from_numpy(uvw_np).pin_memory()
    x_h = torch.from_numpy(x_np).to(rdt).pin_memory()
    M = len(uvw_np)
    y_h = torch.empty(M, dtype=cdt).pin_memory()
    d_h = torch.empty(x_np.shape, dtype=rdt).pin_memory()
    times = []
    n_kept = None
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        uvw = uvw_h.to(dev, non_blocking=True)
        x = x_h.to(dev, non_blocking=True)
        plan = phi.Plan(uvw, **desc)
        y = plan.degrid(x)
        d = plan.grid(y)
        y_h.copy_(y, non_blocking=True)
        d_h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        n_kept = plan.info()["n_kept"]
        plan.close()
    t = min(times)
    return {"value": n_kept / t, "unit": UNIT, "seconds": t,
            "h2d_bytes_per_step": int(uvw_h.numel() * 8 + x_h.numel() * x_h.element_size()),
            "d2h_bytes_per_step": int(y_h.numel() * y_h.element_size() +
                                      d_h.numel() * d_h.element_size()),
            "note": "includes plan build (fold, k-means, sort, tables, cuFFT plan)"}


# ---------------------------------------------------------------------------- serving

def serve_requests(n, seed=0, mmin=5e4, mmax=2e7, sizes=(512, 1024, 2048, 4096, 8192),
                   precision="f32", cap=64, kernel_mode="quadrature"):
    """Synthetic serving stream: observations of log-uniform visibility
    counts, image sizes log-uniform over powers of two, |w|max ~ U[50, 3000]
    (fold on), K ~ U{1..64} raised by the client where the support would
    exceed the cap."""
    from paper_1903_06555_gb300 import serve as S
    rng = np.random.default_rng(seed)
    fov = math.radians(25.0)
    c_sup = 0.5 * 2 * fov / math.sqrt(1 - (0.5 * 2 * fov) ** 2) * 2 * fov  # l_win/(n_win du), os 2
    reqs = []
    for i in range(n):
        m = int(math.exp(rng.uniform(math.log(mmin), math.log(mmax))))
        N = int(rng.choice(sizes))
        wmax = float(rng.uniform(50, 3000))
        k = int(rng.integers(1, 65))
        k = min(126, max(k, int(math.ceil(1.6 * wmax * c_sup / (cap - 4)))))
        n_times = -(-m // 8128)
        uvw = W.uvw_earth_rotation(128, 3000.0, 150e6, -26.7, -37.2, -float(n_times) / 240,
                                   float(n_times) / 240, n_times, wmax=wmax, seed=seed * 1000 + i)[:m]
        desc = dict(image_n=N, fov_rad=fov, n_stacks=k, conj_fold=1, precision=precision,
                    max_support=cap, quad_rel_tol=1e-12 if precision == "f64" else 1e-6,
                    quad_abs_tol=1e-12 if precision == "f64" else 1e-6, kernel_mode=kernel_mode)
        img = W.point_sources(N, 20, seed * 1000 + i)
        reqs.append(S.Request(i, np.ascontiguousarray(uvw), desc, image=img,
                              ops=("degrid", "grid")))
    return reqs


def poisson_arrivals(reqs, rate, seed=0):
    t = 0.0
    rng = np.random.default_rng(seed + 77)
    for r in reqs:
        t += rng.exponential(1.0 / rate)
        r.arrival = t
    return reqs


def run_serve(args):
    """The serving workload: a closed-loop pass over requests drawn from the
    stream's distribution measures capacity (kept visibilities/s); the
    Poisson stream then arrives at `--serve-load` (default 80%) of it.  Requests whose support would
    exceed the cap are retried by the engine with twice the stacks."""
    from paper_1903_06555_gb300 import serve as S
    budget = 150 * 10 ** 9
    km = args.serve_kernel_mode
    probe = serve_requests(24, seed=99, kernel_mode=km)
    for r in probe:
        r.raise_stacks = True
    with S.Server(budget, slots=4) as srv:
        pres = srv.run_stream(probe, realtime=False)
    cap = S.summarize(pres, t_first=0.0)
    reqs = serve_requests(args.serve_requests, seed=1, kernel_mode=km)
    for r in reqs:
        r.raise_stacks = True
    # offered load = arrival rate x mean kept visibilities per request of
    # THIS stream (sizes are heavy-tailed: a small probe's own mean is far
    # off) / the probe's throughput
    kept_frac = cap["vis"] / max(cap["vis_submitted"], 1)
    mean_kept = kept_frac * float(np.mean([r.uvw.shape[0] for r in reqs]))
    rate = args.serve_load * cap["vis_per_s"] / mean_kept
    poisson_arrivals(reqs, rate)
    if args.serve_full_scale:
        from paper_1903_06555_gb300.serve import Request
        n_times = -(-126_600_000 // 8128)
        uvw = W.uvw_earth_rotation(128, 3000.0, 150e6, -26.7, -37.2, -n_times / 240,
                                   n_times / 240, n_times, wmax=600.0, seed=5)[:126_600_000]
        full = Request(10_000, np.ascontiguousarray(uvw),
                       dict(image_n=8192, fov_rad=math.radians(25.0), n_stacks=64, conj_fold=1,
                            kernel_mode=km),
                       image=W.point_sources(8192, 200, 5), ops=("degrid", "grid"),
                       arrival=reqs[len(reqs) // 2].arrival, raise_stacks=True)
        reqs.append(full)
    with S.Server(budget, slots=4) as srv:
        res = srv.run_stream(reqs)
        peak = srv.peak_bytes
    summ = S.summarize(res)
    full_res = [r for r in res if r.rid == 10_000]
    raised = sum(1 for r, q in zip(res, reqs) if r.status == "ok" and r.n_stacks > q.desc["n_stacks"])
    # FP32 vs FP64 on the same reduced stream, back to back
    cmp = {}
    for prec in ("f32", "f64"):
        small = poisson_arrivals(serve_requests(16, seed=7, mmin=5e4, mmax=4e5, sizes=(512, 1024),
                                                precision=prec), rate=1000.0)
        for r in small:
            r.raise_stacks = True
        with S.Server(budget, slots=4) as srv:
            r2 = srv.run_stream(small)
        cmp[prec] = S.summarize(r2)
    line = {"metric": "served w-corrected visibilities/s (degrid+grid per request), p50/p99 latency",
            "value": summ.get("vis_per_s"), "unit": UNIT, "n_gpus": 1, "dtype": "f32",
            "workload": "serving: Poisson stream of %d observations (5e4-2e7 vis, 512^2-8192^2, "
                        "|w|max 50-3000, K 1-64 raised to fit J_w <= 64) + 126.6M-vis 8192^2 request"
                        % args.serve_requests,
            "kernel_mode": km, "capacity_closed_loop": cap, "offered_load": args.serve_load,
            "mean_kept_per_request": mean_kept, "arrival_rate_per_s": rate, "hbm_budget_bytes": budget,
            "peak_admitted_bytes": peak, "summary": summ, "stacks_raised": raised,
            "full_scale": None if not full_res else {
                "status": full_res[0].status, "error": full_res[0].error,
                "latency_s": full_res[0].latency, "n_vis": full_res[0].n_vis,
                "n_kept": full_res[0].n_kept, "device_bytes": full_res[0].device_bytes},
            "fp32_vs_fp64_reduced_stream": cmp}
    print(json.dumps(line), flush=True)


def run_plan_study(args):
    """Plan building (fold, Algorithm 1, sort, tables) and kernel
    construction (one degrid: every tap's kernel integrated once) with the
    conjugate fold on and off, on the MWA-like snapshot (8 stacks) and at the
    paper's scale (126.6M visibilities, |w| <= 600 after the fold, 1200
    before, 50 stacks, 2048^2 image; Sec. 4)."""
    import paper_1903_06555_gb300 as phi
    dev = torch.device("cuda", torch.cuda.current_device())
    out = []
    n_times = -(-126_600_000 // 8128)
    cases = [("mwa-2048-8stack", W.uvw_for(W.mwa_snapshot()), 2048, 8),
             ("paper-scale-126.6M-50stack",
              W.uvw_earth_rotation(128, 3000.0, 150e6, -26.7, -37.2, -n_times / 240,
                                   n_times / 240, n_times, wmax=600.0, seed=5)[:126_600_000],
              2048, 50)]
    for name, uvw_np, n_img, k in cases:
        uvw = torch.from_numpy(np.ascontiguousarray(uvw_np)).to(dev)
        x = torch.from_numpy(W.point_sources(n_img, 200, 0)).to(dev, torch.float32)
        for fold in (1, 0):
            rec = {"case": name, "conj_fold": fold, "n_vis": int(uvw.shape[0]), "n_stacks": k}
            try:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                plan = phi.Plan(uvw, image_n=n_img, fov_rad=math.radians(25.0), n_stacks=k,
                                conj_fold=fold, max_support=256)
                torch.cuda.synchronize()
                rec["plan_ms"] = 1e3 * (time.perf_counter() - t0)
                info = plan.info()
                cnt = np.array(info["counts"], float)
                jw = np.array(info["jw"], float)
                rec.update(kmeans_sweeps=info["kmeans_sweeps"], n_kept=info["n_kept"],
                           max_jw=info["max_jw"],
                           mean_jw2=float((cnt * jw ** 2).sum() / max(cnt.sum(), 1)),
                           w_span=float(max(info["wbar"]) - min(info["wbar"])))
                plan.degrid(x)
                plan.stats_full(reset=True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                plan.degrid(x)
                torch.cuda.synchronize()
                rec["kernel_construction_s"] = time.perf_counter() - t0
                bad, taps, nodes = plan.stats_full(reset=True)
                rec.update(taps=taps, tap_nodes=nodes, unconverged=bad,
                           kernels_per_s=info["n_kept"] / rec["kernel_construction_s"])
                plan.close()
                if fold:
                    for staged in (0, 1, 2):
                        tp = phi.Plan(uvw, image_n=n_img, fov_rad=math.radians(25.0), n_stacks=k,
                                      conj_fold=fold, max_support=256, kernel_mode="table",
                                      grid_staging=staged)
                        y = tp.degrid(x)
                        tp.grid(y)
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        y = tp.degrid(x)
                        tp.grid(y)
                        torch.cuda.synchronize()
                        rec[f"table_degrid_grid_s_staging{staged}"] = time.perf_counter() - t0
                        tp.close()
            except phi.PhiError as e:
                rec["error"] = str(e)
            out.append(rec)
            print(json.dumps(rec), flush=True)
    line = {"metric": "plan build and kernel construction, conjugate fold on/off",
            "paper_context": "Sec. 4: 126.6M visibilities, 50 stacks: k-means < 5 s in 6 "
                             "iterations; kernel construction 15 min on 50 nodes (800 cores)",
            "cases": out}
    print(json.dumps(line), flush=True)


def timed_ms(fn, steps, warmup):
    """Mean milliseconds of fn() over `steps` calls after `warmup`, CUDA
    events on the current stream."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def run_precision(args):
    """The precision study (4096^2 image, 8192^2 grid, 17.5M visibilities,
    |w| <= 1500, 32 stacks, fold on): the FP32 path (FP64 chirp phase) timed
    at full size; FP32 and FP64 (quadrature tol 1e-12) on a 20,000-visibility
    sub-observation with the full plan's centres and supports, i.e. the same
    operator, timed and compared."""
    import paper_1903_06555_gb300 as phi
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = W.precision_study()
    uvw = W.uvw_for(wl)
    kw = dict(image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg), n_stacks=wl.n_stacks,
              conj_fold=int(wl.conj_fold))
    x_np = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    plan = phi.Plan(torch.from_numpy(uvw).to(dev), **kw)
    info = plan.info()
    x32 = torch.from_numpy(x_np).to(dev, torch.float32)
    y = torch.from_numpy(W.random_vis(len(uvw), 4)).to(dev, torch.complex64)
    ms32 = timed_ms(lambda: (plan.degrid(x32), plan.grid(y)), args.steps, args.warmup)
    plan.close()
    sel = np.sort(np.random.default_rng(2).choice(len(uvw), 20000, replace=False))
    sub = torch.from_numpy(np.ascontiguousarray(uvw[sel])).to(dev)
    fixed = dict(centres=info["wbar"], stack_jw=info["jw"], **kw)
    p32 = phi.Plan(sub, **fixed)
    p64 = phi.Plan(sub, precision="f64", quad_rel_tol=1e-12, quad_abs_tol=1e-12, **fixed)
    n_sub = p64.info()["n_kept"]
    x64 = x32.double()
    ys = y[torch.from_numpy(sel).to(dev)]
    ms_sub32 = timed_ms(lambda: (p32.degrid(x32), p32.grid(ys)), 3, 1)
    ms_sub64 = timed_ms(lambda: (p64.degrid(x64), p64.grid(ys.to(torch.complex128))), 1, 1)

    def rel(a, b):
        return float(torch.linalg.vector_norm(a.to(b.dtype) - b) / torch.linalg.vector_norm(b))
    y64 = p64.degrid(x64)
    g64 = p64.grid(ys.to(torch.complex128))
    # the FP64 path against the FP64 pipe: DP flops per tap-node from the
    # committed ncu capture of vis_kernel<double> x the tap-nodes counted here
    p64.stats_full(reset=True)
    p64.degrid(x64)
    p64.grid(ys.to(torch.complex128))
    nodes64 = p64.stats_full(reset=True)[2]
    prof64 = profiled_fp64()
    peaks = measured_peaks()
    peak64 = FP64_NOMINAL_TFLOPS * device_sms() / 152.0 * peaks.get("sm_max_mhz", 2070.0) / 2070.0
    fp64_roof = {"tap_nodes_per_vis": nodes64 / (2 * n_sub), "peak": peak64, "unit": "TFLOP/s",
                 "peak_note": "nominal FP64 (no measured FP64 peak)", "ncu": prof64}
    if prof64 and "fp64_flops_per_tap_node" in prof64:
        ach = nodes64 * prof64["fp64_flops_per_tap_node"] / (ms_sub64 / 1e3) / 1e12
        fp64_roof.update(achieved=ach, frac=ach / peak64,
                         note="degrid + grid of the sub-observation, FFTs and prep included in "
                              "the time, so the kernel's own fraction is higher")
    # the radial interpolation mode: FP32 at full size, FP32 and FP64 on the
    # sub-observation, both against the FP64 per-tap quadrature
    rplan = phi.Plan(torch.from_numpy(uvw).to(dev), kernel_mode="radial", **kw)
    ms_r32 = timed_ms(lambda: (rplan.degrid(x32), rplan.grid(y)), args.steps, args.warmup)
    rplan.close()
    r32 = phi.Plan(sub, kernel_mode="radial", **fixed)
    r64 = phi.Plan(sub, kernel_mode="radial", precision="f64", quad_rel_tol=1e-12,
                   quad_abs_tol=1e-12, **fixed)
    ms_rsub64 = timed_ms(lambda: (r64.degrid(x64), r64.grid(ys.to(torch.complex128))), 2, 1)
    radial = {"fp32_full_vis_per_s": info["n_kept"] / (ms_r32 / 1e3), "fp32_full_ms_per_step": ms_r32,
              "fp64_sub_vis_per_s": n_sub / (ms_rsub64 / 1e3),
              "fp32_vs_fp64_quadrature_rel_l2": {"degrid": rel(r32.degrid(x32), y64),
                                                  "grid": rel(r32.grid(ys), g64)},
              "fp64_vs_fp64_quadrature_rel_l2": {"degrid": rel(r64.degrid(x64), y64),
                                                  "grid": rel(r64.grid(ys.to(torch.complex128)), g64)}}
    line = {"metric": "precision study: FP32 (FP64 chirp phase) vs FP64, degrid+grid",
            "workload": f"{wl.name}: {wl.image_n}^2 image, {info['npad']}^2 grid, "
                        f"{len(uvw)} visibilities, {wl.n_stacks} stacks, |w| <= {wl.uvw['wmax']:g}",
            "fp32_full": {"vis_per_s": info["n_kept"] / (ms32 / 1e3), "ms_per_step": ms32,
                          "n_kept": info["n_kept"], "max_jw": info["max_jw"]},
            "sub_observation": {
                "n_kept": n_sub,
                "fp32_vis_per_s": n_sub / (ms_sub32 / 1e3), "fp64_vis_per_s": n_sub / (ms_sub64 / 1e3),
                "fp32_vs_fp64_rel_l2": {"degrid": rel(p32.degrid(x32), y64),
                                        "grid": rel(p32.grid(ys), g64)},
                "fp64_roofline": fp64_roof,
                "note": "same centres and supports as the full plan; FP64 path at quadrature "
                        "tol 1e-12 (parity-tested against the FP64 oracle to 1e-10)"},
            "radial_mode": radial,
            "paper_context": "Paper I: 17.5M visibilities"}
    print(json.dumps(line), flush=True)


def run_diff(args):
    """The differentiable workload (4096^2 image, 8192^2 grid, 10M visibilities,
    16 stacks): L = 1/2 ||Phi x - y||^2 through autograd.PhiDegrid (backward =
    phi_grid), timed per forward+backward; the directional derivative on 64
    random pixels against a central difference; 20 power iterations for
    ||Phi||^2 and 20 gradient-descent steps."""
    import paper_1903_06555_gb300 as phi
    from paper_1903_06555_gb300 import autograd as PA, solvers
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = W.differentiable()
    uvw = W.uvw_for(wl)
    plan = phi.Plan(torch.from_numpy(uvw).to(dev), image_n=wl.image_n,
                    fov_rad=math.radians(wl.fov_deg), n_stacks=wl.n_stacks,
                    conj_fold=int(wl.conj_fold), max_support=192)
    info = plan.info()
    x_true = torch.from_numpy(W.point_sources(wl.image_n, wl.n_sources, wl.seed)).to(dev).float()
    y = plan.degrid(x_true)
    x = (0.5 * x_true).requires_grad_(True)

    def fwd_bwd():
        x.grad = None
        loss = 0.5 * torch.sum(torch.abs(PA.degrid(x, plan) - y) ** 2)
        loss.backward()
    ms = timed_ms(fwd_bwd, args.steps, args.warmup)
    rng = np.random.default_rng(3)
    n = wl.image_n
    v = torch.zeros(n * n, device=dev)
    v[torch.from_numpy(rng.choice(n * n, 64, replace=False)).to(dev)] = \
        torch.from_numpy(rng.standard_normal(64)).to(dev).float()
    v = v.view(n, n)
    fwd_bwd()
    g_dir = float(torch.sum(x.grad.double() * v.double()))

    def L(t):
        return 0.5 * float(torch.sum(torch.abs((plan.degrid(t) - y).to(torch.complex128)) ** 2))
    eps = 1e-2 * float(x_true.abs().max())
    fd = (L(x.detach() + eps * v) - L(x.detach() - eps * v)) / (2 * eps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, _ = solvers.power_method(plan, 20)
    torch.cuda.synchronize()
    t_pm = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, losses = solvers.least_squares(plan, y, steps=20, step=1.0 / lam)
    torch.cuda.synchronize()
    t_gd = time.perf_counter() - t0
    line = {"metric": "differentiable operator: forward+backward of 1/2||Phi x - y||^2",
            "workload": f"{wl.name}: {wl.image_n}^2 image, {info['npad']}^2 grid, "
                        f"{len(uvw)} visibilities, {wl.n_stacks} stacks",
            "fwd_bwd_ms": ms, "vis_per_s": info["n_kept"] / (ms / 1e3),
            "finite_difference": {"directional_grad": g_dir, "central_difference": fd,
                                  "rel_diff": abs(fd - g_dir) / abs(g_dir),
                                  "direction": "64 random pixels, eps = 1e-2 max|x|, FP32 path"},
            "power_method": {"iters": 20, "norm_sq": lam, "seconds": t_pm},
            "gradient_descent": {"steps": 20, "seconds": t_gd, "loss_first": losses[0],
                                 "loss_last": losses[-1],
                                 "monotone": all(b <= a * (1 + 1e-6)
                                                 for a, b in zip(losses, losses[1:]))}}
    print(json.dumps(line), flush=True)


def dde_macs(counts, jws, jd):
    """Complex multiply-adds of the separable DDE convolution per call: per
    visibility of support J_w, J_D J_w^2 in the row pass (each w-kernel tap
    feeds J_D columns) and J_D J_w (J_w + J_D - 1) in the column pass (each
    row of R feeds J_D combined rows, over J_w + J_D - 1 columns)."""
    return sum(c * jd * j * (j + j + jd - 1) for c, j in zip(counts, jws))


def run_dde(args):
    """Direction-dependent effects (Sec. 5.2): the MWA-like snapshot without
    the fold (16 stacks), a synthetic separable DDE kernel of 5 x 5 taps per
    visibility convolved with the w-kernel; degrid + grid timed against the
    plain operator on the same plan."""
    import paper_1903_06555_gb300 as phi
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = W.mwa_snapshot()
    uvw_np, x_np = workload_inputs(wl)
    jd = 5
    a_np, b_np = W.dde_kernels(len(uvw_np), jd, 77)
    plan = phi.Plan(torch.from_numpy(uvw_np).to(dev), image_n=wl.image_n,
                    fov_rad=math.radians(wl.fov_deg), n_stacks=16, conj_fold=0)
    info = plan.info()
    x = torch.from_numpy(x_np).to(dev, torch.float32)
    y = torch.from_numpy(W.random_vis(len(uvw_np), 4)).to(dev, torch.complex64)
    a = torch.from_numpy(a_np).to(dev, torch.complex64)
    b = torch.from_numpy(b_np).to(dev, torch.complex64)
    ms_plain = timed_ms(lambda: (plan.degrid(x), plan.grid(y)), args.steps, args.warmup)
    plan.stats_full(reset=True)
    ms_dde = timed_ms(lambda: (plan.degrid_dde(x, a, b), plan.grid_dde(y, a, b)), args.steps,
                      args.warmup)
    bad, taps, nodes = plan.stats_full(reset=True)
    calls = 2 * (args.steps + args.warmup)
    n_kept = info["n_kept"]
    yq = plan.degrid_dde(x, a, b)
    plan.close()
    # the same with the w-kernel box filled from the radial mode's series
    rplan = phi.Plan(torch.from_numpy(uvw_np).to(dev), image_n=wl.image_n,
                     fov_rad=math.radians(wl.fov_deg), n_stacks=16, conj_fold=0,
                     kernel_mode="radial")
    ms_rdde = timed_ms(lambda: (rplan.degrid_dde(x, a, b), rplan.grid_dde(y, a, b)), args.steps,
                       args.warmup)
    ms_rplain = timed_ms(lambda: (rplan.degrid(x), rplan.grid(y)), args.steps, args.warmup)
    yr = rplan.degrid_dde(x, a, b)
    radial = {"vis_per_s": n_kept / (ms_rdde / 1e3), "ms_per_step": ms_rdde,
              "plain_operator_ms_per_step": ms_rplain,
              "rel_l2_vs_quadrature_box": float(torch.linalg.vector_norm(yr - yq) /
                                                torch.linalg.vector_norm(yq))}
    rplan.close()
    # executed work: the quadrature tap-nodes of the w-kernel boxes and the
    # separable convolution's complex multiply-adds (8 flops each): per
    # visibility of support J_w, J_D J_w^2 for the row pass (J_w rows of the
    # J_w + J_D - 1 columns, J_D taps inside the box per w-kernel tap) and
    # J_D J_w (J_w + J_D - 1) for the column pass
    macs = dde_macs(info["counts"], info["jw"], jd)
    flops = nodes * FLOPS_PER_TAP_NODE / calls + macs * 8.0
    ach = flops / (ms_dde / 2 / 1e3) / 1e12
    peaks = measured_peaks()
    peak_fp32 = fp32_peak_tflops(device_sms(), peaks.get("sm_max_mhz", 2070.0))
    line = {"metric": "w-corrected visibilities/s with a DDE per visibility (degrid+grid)",
            "value": n_kept / (ms_dde / 1e3), "unit": UNIT,
            "workload": f"{wl.name} without the fold: 16 stacks (J_w up to {info['max_jw']}), "
                        f"{n_kept} kept visibilities, separable {jd}x{jd} DDE kernels",
            "ms_per_step": ms_dde, "plain_operator_ms_per_step": ms_plain,
            "plain_operator_vis_per_s": n_kept / (ms_plain / 1e3),
            "combined_taps_per_vis": taps / calls / n_kept,
            "quadrature_tap_nodes_per_vis": nodes / calls / n_kept, "unconverged": bad,
            "radial_mode": radial,
            "roofline": {"bound": "alu", "kernel": "vis_dde_kernel", "achieved": ach,
                         "peak": peak_fp32, "unit": "TFLOP/s", "frac": ach / peak_fp32,
                         "work_note": "executed work: 36 flops per quadrature tap-node + "
                                      "J_D J_w (2 J_w + J_D - 1) complex multiply-adds per "
                                      "visibility (separable row and column passes)"}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "serve":
        if rank == 0:
            run_serve(args)
    elif args.workload == "plan":
        if rank == 0:
            run_plan_study(args)
    elif args.workload == "precision":
        if rank == 0:
            run_precision(args)
    elif args.workload == "diff":
        if rank == 0:
            run_diff(args)
    elif args.workload == "dde":
        if rank == 0:
            run_dde(args)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
