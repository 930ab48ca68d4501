"""Serving engine: continuous batching of imaging requests on one GPU.

A request is one observation (baselines, image geometry, stack count) plus
the operator applications wanted on it: y = Phi x (degrid), d = Re(Phi^H y)
(grid) or both.  The engine

* admits requests as soon as a slot and enough of the HBM budget are free --
  not in arrival batches: a request that arrives while others run starts as
  soon as it fits, and later small requests may start ahead of an earlier
  large one that does not fit yet (backfill);
* runs every admitted request on its own CUDA stream from its own worker
  thread (the library calls release the GIL), so plan builds, FFTs and the
  fused quadrature kernels of different requests overlap on the device;
* keeps plans (sorted visibility records, stack tables, padded grid, cuFFT
  plan) resident under the request's `obs_key`, so later requests on the
  same observation skip planning; resident plans are evicted least recently
  used when admission needs their memory;
* records per-request latency (arrival -> result on the host) and the
  stream's throughput, and isolates failures: a request whose plan or call
  fails returns an error result and releases its memory without touching
  the others.

Memory admission is by a conservative per-request estimate of the device
bytes the plan build and the calls need (inputs, outputs, plan-build
temporaries, records, grid, cuFFT workspace), released when the request
completes; a resident plan keeps its measured size.
"""
from __future__ import annotations

import math
import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import PHI_ERR_SUPPORT, PhiError, Plan

__all__ = ["Request", "Result", "Server", "estimate_bytes"]


@dataclass
class Request:
    rid: int
    uvw: np.ndarray                 # (M, 3) float64, wavelengths
    desc: dict                      # plan descriptor fields (image_n, fov_rad, n_stacks, ...)
    image: np.ndarray | None = None  # (N, N) real, for degrid
    vis: np.ndarray | None = None    # (M,) complex, for a grid-only request
    ops: tuple = ("degrid",)        # any of "degrid", "grid" (grid of the degrid output if both)
    arrival: float = 0.0            # seconds after the stream starts
    obs_key: str | None = None      # keep/reuse the plan under this key
    raise_stacks: bool = False      # on PHI_ERR_SUPPORT retry with twice the stacks (<= 126)


@dataclass
class Result:
    rid: int
    status: str                     # "ok" or "error"
    error: str = ""
    y: np.ndarray | None = None
    dirty: np.ndarray | None = None
    n_vis: int = 0
    arrival: float = 0.0
    admitted: float = 0.0
    started: float = 0.0
    done: float = 0.0
    plan_reused: bool = False
    device_bytes: int = 0
    n_kept: int = 0                 # visibilities inside the grid (w-corrected)
    n_stacks: int = 0               # stacks used (after any raising)

    @property
    def latency(self):
        return self.done - self.arrival


def estimate_bytes(req: Request, planned: bool = False) -> int:
    """Upper bound of the device bytes a request needs while it runs: with
    planned=True only its inputs and outputs (the plan is already resident),
    otherwise also the plan-build temporaries (folded w, flags, stack ids,
    sort keys and values with their CUB buffers), the records, per-pixel
    tables, the padded grids of one stack group (as many stacks as fit
    max_grid_mib, default 4 GiB) and cuFFT workspace (at most one grid per
    batched transform plus one), and with grid_deterministic the
    fixed-point sums of the group's grids (16 bytes a cell).  A request that
    may raise its stacks is charged for the most stacks a retry can reach
    (126)."""
    m = int(req.uvw.shape[0])
    n = int(req.desc["image_n"])
    os_ = float(req.desc.get("oversample", 2.0))
    # the library's lround: halves away from zero (Python's round() takes halves to even)
    npad = int(math.floor(os_ * n + 0.5))
    f64 = req.desc.get("precision", "f32") == "f64"
    c = 16 if f64 else 8
    r = 8 if f64 else 4
    io = m * 2 * c + n * n * 2 * r + (16 << 20)
    if planned:
        return io
    per_vis = 24 + 8 + 1 + 4 + 16 + 16 + (52 if f64 else 36)
    per_pix = 12 + r
    grid = c * npad * npad
    fixed = 16 * npad * npad if int(req.desc.get("grid_deterministic", 0)) else 0
    k = 126 if req.raise_stacks else int(req.desc.get("n_stacks", 1))
    cap = (int(req.desc.get("max_grid_mib", 0)) or 4096) << 20
    group = max(1, min(k, cap // (grid + fixed)))
    return (io + m * per_vis + n * n * per_pix + (2 * group + 1) * grid + group * fixed +
            (8 << 20))


class Server:
    def __init__(self, hbm_budget_bytes: int, slots: int = 4, device: int = 0,
                 keep_plans: bool = True):
        self.budget = int(hbm_budget_bytes)
        self.slots = int(slots)
        self.device = torch.device("cuda", device)
        self.keep_plans = keep_plans
        self._lock = threading.Condition()
        self._pending: collections.deque = collections.deque()
        self._in_use = 0                 # bytes admitted for running requests
        self._resident = collections.OrderedDict()   # obs_key -> (Plan, bytes)
        self._resident_bytes = 0
        self._running = 0
        self._busy_keys = set()
        self._closed = False
        self.peak_bytes = 0
        self.t0 = time.perf_counter()
        with torch.cuda.device(self.device):
            self._streams = [torch.cuda.Stream(device=self.device) for _ in range(self.slots)]
        self._free_streams = list(range(self.slots))
        self._pool = cf.ThreadPoolExecutor(max_workers=self.slots)
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # ------------------------------------------------------------------ API
    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> cf.Future:
        fut: cf.Future = cf.Future()
        with self._lock:
            if self._closed:
                raise RuntimeError("server closed")
            self._pending.append((req, fut, self.now()))
            self._lock.notify_all()
        return fut

    def run_stream(self, requests, realtime: bool = True):
        """Submit requests at their arrival times (relative to now) and wait
        for all results; returns them in request order."""
        start = time.perf_counter()
        futs = []
        for req in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                delay = req.arrival - (time.perf_counter() - start)
                if delay > 0:
                    time.sleep(delay)
            futs.append((req.rid, self.submit(req)))
        res = {rid: f.result() for rid, f in futs}
        return [res[r.rid] for r in requests]

    def close(self):
        with self._lock:
            self._closed = True
            self._lock.notify_all()
        self._sched.join()
        self._pool.shutdown(wait=True)
        for plan, _ in self._resident.values():
            plan.close()
        self._resident.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ scheduling
    def _need(self, req):
        if req.obs_key is not None and req.obs_key in self._resident:
            return estimate_bytes(req, planned=True)
        return estimate_bytes(req)

    def _evict_for(self, need):
        """Drop least-recently-used resident plans not in use until `need`
        fits; returns True if it fits."""
        for key in list(self._resident.keys()):
            if self._in_use + self._resident_bytes + need <= self.budget:
                break
            if key in self._busy_keys:
                continue
            plan, b = self._resident.pop(key)
            self._resident_bytes -= b
            plan.close()
        return self._in_use + self._resident_bytes + need <= self.budget

    def _schedule(self):
        with self._lock:
            while True:
                while not self._pending and not self._closed:
                    self._lock.wait()
                if self._closed and not self._pending:
                    return
                started = False
                if self._free_streams:
                    for idx, (req, fut, arr) in enumerate(self._pending):
                        if req.obs_key is not None and req.obs_key in self._busy_keys:
                            continue
                        need = self._need(req)
                        if need > self.budget:
                            del self._pending[idx]
                            fut.set_result(Result(req.rid, "error", "request exceeds the HBM budget",
                                                  n_vis=len(req.uvw), arrival=arr, done=self.now()))
                            started = True
                            break
                        if self._evict_for(need):
                            del self._pending[idx]
                            self._in_use += need
                            self.peak_bytes = max(self.peak_bytes, self._in_use + self._resident_bytes)
                            sid = self._free_streams.pop()
                            if req.obs_key is not None:
                                self._busy_keys.add(req.obs_key)
                            self._running += 1
                            self._pool.submit(self._work, req, fut, arr, need, sid, self.now())
                            started = True
                            break
                if not started:
                    # nothing fits now: every change that can make room (a
                    # request finishing, a new one arriving, close) notifies
                    self._lock.wait()

    # ---------------------------------------------------------------- worker
    def _work(self, req, fut, arrival, need, sid, admitted):
        res = Result(req.rid, "ok", n_vis=int(len(req.uvw)), arrival=arrival, admitted=admitted)
        stream = self._streams[sid]
        plan = None
        keep = False
        try:
            res.started = self.now()
            with torch.cuda.device(self.device), torch.cuda.stream(stream):
                if req.obs_key is not None and req.obs_key in self._resident:
                    plan = self._resident[req.obs_key][0]
                    res.plan_reused = True
                else:
                    uvw = torch.from_numpy(np.ascontiguousarray(req.uvw, np.float64)).pin_memory()
                    uvw_d = uvw.to(self.device, non_blocking=True)
                    desc = dict(req.desc)
                    while True:
                        try:
                            plan = Plan(uvw_d, stream=stream, **desc)
                            break
                        except PhiError as e:
                            k = int(desc.get("n_stacks", 1))
                            if e.status != PHI_ERR_SUPPORT or not req.raise_stacks or k >= 126:
                                raise
                            desc["n_stacks"] = min(126, 2 * k)
                info = plan.info()
                res.device_bytes = info["device_bytes"]
                res.n_kept = info["n_kept"]
                res.n_stacks = info["n_stacks"]
                y = None
                if "degrid" in req.ops:
                    x = torch.from_numpy(np.ascontiguousarray(req.image)).pin_memory()
                    y = plan.degrid(x.to(self.device, plan.real_dtype, non_blocking=True),
                                    stream=stream)
                if "grid" in req.ops:
                    if y is None:
                        v = torch.from_numpy(np.ascontiguousarray(req.vis)).pin_memory()
                        y = v.to(self.device, plan.complex_dtype, non_blocking=True)
                    d = plan.grid(y, stream=stream)
                    res.dirty = d.to("cpu", non_blocking=True)
                if "degrid" in req.ops:
                    res.y = y.to("cpu", non_blocking=True)
                stream.synchronize()
                if res.y is not None:
                    res.y = res.y.numpy()
                if res.dirty is not None:
                    res.dirty = res.dirty.numpy()
            keep = self.keep_plans and req.obs_key is not None
        except (PhiError, RuntimeError, ValueError) as e:
            res.status = "error"
            res.error = str(e)
        res.done = self.now()
        with self._lock:
            self._in_use -= need
            if plan is not None and keep and not res.plan_reused:
                b = res.device_bytes
                self._resident[req.obs_key] = (plan, b)
                self._resident_bytes += b
                plan = None
            elif res.plan_reused:
                self._resident.move_to_end(req.obs_key)
                plan = None
            if req.obs_key is not None:
                self._busy_keys.discard(req.obs_key)
            self._free_streams.append(sid)
            self._running -= 1
            self._lock.notify_all()
        if plan is not None:
            plan.close()
        fut.set_result(res)


def summarize(results, t_first=None):
    """Throughput and latency percentiles of a finished stream."""
    ok = [r for r in results if r.status == "ok"]
    if not ok:
        return {"ok": 0, "errors": len(results)}
    lat = np.array([r.latency for r in ok])
    t0 = min(r.arrival for r in results) if t_first is None else t_first
    t1 = max(r.done for r in ok)
    nvis = sum(r.n_kept for r in ok)
    errs = collections.Counter(r.error.split(":")[-1].strip() for r in results if r.status != "ok")
    return {"ok": len(ok), "errors": len(results) - len(ok), "error_kinds": dict(errs), "vis": nvis,
            "vis_submitted": sum(r.n_vis for r in ok),
            "makespan_s": t1 - t0, "vis_per_s": nvis / (t1 - t0),
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_max_s": float(lat.max()),
            "plans_reused": sum(r.plan_reused for r in ok)}
