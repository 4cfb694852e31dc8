"""Continuous-batching server for forward transport solves on one GPU.

Requests (grid, order N, optical maps, sources, detectors, step count) arrive
over time. The server admits the next waiting request as soon as a slot is
free and its device footprint (rte_plan_footprint) fits the HBM that the
running requests leave. When one finishes, its slot and memory go to the
next waiting request.

Two ways to run admitted requests:
  - one plan, CUDA stream and host thread per request, so that the device
    work of concurrent requests overlaps;
  - grouping (grouping=True): requests with the same grid and order that run
    at the same time share a group, one host thread and stream per group,
    which advances all its members (up to 8) chunk by chunk with
    rte_step_group, one launch of each step pass for the whole group.
    Requests join a running group of their shape at its next chunk boundary
    and leave it when done.
An autotuner (autotune.Autotuner) may pick each shape's schedule and steps
per step graph; the choice is made once per shape and then pinned.

A request's readouts do not depend on what else runs: every kernel reads and
writes only its plans' buffers, a grouped launch computes each plan's work
items exactly as a launch for that plan alone, and the forward step has no
floating-point atomics; so results are bitwise the same alone, in the mix and
in a group (for the same pinned schedule).

The scheduler is host logic. All transport arithmetic runs in librte's
kernels through the C ABI.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    shape: tuple
    dx: float
    N: int
    c: float
    mua: np.ndarray
    mus: np.ndarray
    g: np.ndarray
    nsteps: int
    pml_cells: int = 0
    pml_mu0: float = 0.0
    pml_mu1: float = 0.0
    src_voxel: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    src_amp: np.ndarray = field(default_factory=lambda: np.zeros(0))
    src_t0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    src_fwhm: np.ndarray = field(default_factory=lambda: np.zeros(0))
    det_voxel: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    arrival: float = 0.0          # seconds after the start of the run
    dt_fraction: float = 0.5      # dt = dt_fraction * the plan's stability limit

    @staticmethod
    def from_workload(rid, wl, arrival=0.0, nsteps=None):
        n = int(nsteps if nsteps is not None else wl.nsteps)
        return Request(rid, tuple(wl.shape), wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, n, wl.pml_width,
                       wl.pml_mu0, wl.pml_mu1, wl.src_voxel, wl.src_amp, wl.src_t0, wl.src_fwhm,
                       wl.det_voxel, arrival, wl.dt_fraction)

    @property
    def updates(self):
        """Moment-voxel updates of the whole request, counted in (N+1)^2 moments."""
        return (self.N + 1) ** 2 * int(np.prod(self.shape)) * self.nsteps


@dataclass
class Result:
    rid: int
    readouts: np.ndarray | None   # [nsteps, ndet], Re psi_00 at the detectors before each step
    dt: float
    arrival: float
    admitted: float
    end: float
    slot: int
    error: str | None = None

    @property
    def latency(self):
        return self.end - self.arrival

    @property
    def ok(self):
        return self.error is None


class Cancelled(Exception):
    pass


def plan_bytes(req: Request, precision: str, real_radiance: bool) -> int:
    """Device bytes of the request's plan for a forward solve."""
    from . import make_desc, plan_footprint
    return plan_footprint(make_desc(req.shape, req.dx, req.N, req.c, req.pml_cells, req.pml_mu0,
                                    req.pml_mu1, precision, real_radiance))


def open_plan(req: Request, precision: str, real_radiance: bool, stream=None, tuner=None):
    """The request's plan on `stream`, with its sources, detectors and (if a
    tuner is given) its shape's pinned schedule; returns (plan, dt)."""
    from . import Plan
    plan = Plan(req.shape, req.dx, req.N, req.c, req.mua, req.mus, req.g, req.pml_cells, req.pml_mu0,
                req.pml_mu1, precision, stream=stream, real_radiance=real_radiance)
    try:
        if tuner is not None:
            tuner.apply(plan, tuner.choice(req.shape, req.N, precision, real_radiance, req.dx, req.c,
                                           req.pml_cells, req.pml_mu0, req.pml_mu1, stream))
        if len(req.src_voxel):
            plan.set_sources(req.src_voxel, np.zeros(len(req.src_voxel)), req.src_amp, req.src_t0,
                             req.src_fwhm)
        if len(req.det_voxel):
            plan.set_detectors(req.det_voxel)
        return plan, req.dt_fraction * plan.stability_limit()
    except Exception:
        plan.close()
        raise


def run_request(req: Request, precision: str, real_radiance: bool, stream=None, chunk: int = 250,
                should_stop=None, tuner=None):
    """Run one request to completion on `stream` (a cudaStream_t as int, or
    None for the legacy default stream); returns (readouts, dt). Between
    chunks of `chunk` steps, `should_stop()` may cancel it."""
    plan, dt = open_plan(req, precision, real_radiance, stream, tuner)
    try:
        parts = []
        done = 0
        while done < req.nsteps:
            if should_stop is not None and should_stop():
                raise Cancelled(f"request {req.rid} cancelled after {done} steps")
            k = min(chunk, req.nsteps - done)
            det, _ = plan.step(dt, k)
            parts.append(det if det is not None else np.zeros((k, 0)))
            done += k
        return np.concatenate(parts, axis=0), dt
    finally:
        plan.close()


class Server:
    """FIFO admission by free slot and HBM footprint.

    Without grouping: one host thread and one CUDA stream per running request.
    runner(req, slot, should_stop) -> (readouts, dt) and sizer(req) -> bytes
    default to a librte plan per request on the slot's stream and to
    rte_plan_footprint; both can be replaced (host-side tests drive the
    scheduler with stand-ins).

    With grouping=True (GPU only): requests of the same grid and order that
    run at the same time share a group thread and stream, stepped together
    by rte_step_group (at most 8 per launch; a larger group steps in turns).
    tuner (autotune.Autotuner or None) pins each shape's schedule."""

    def __init__(self, slots: int = 4, hbm_budget: int | None = None, precision: str = "fp32",
                 real_radiance: bool = True, chunk: int = 250, runner=None, sizer=None, grouping: bool = False,
                 tuner=None):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.slots = int(slots)
        self.hbm_budget = hbm_budget
        self.precision = precision
        self.real = bool(real_radiance)
        self.chunk = int(chunk)
        self.runner = runner
        self.grouping = bool(grouping)
        self.tuner = tuner
        self.sizer = sizer or (lambda r: plan_bytes(r, self.precision, self.real))
        self._cancel = set()
        self._lock = threading.Lock()
        self.stats = {}

    def cancel(self, rid: int):
        """Cancel a request: a waiting one is never admitted, a running one
        stops at its next chunk boundary; its result carries the error."""
        with self._lock:
            self._cancel.add(rid)

    def _cancelled(self, rid):
        with self._lock:
            return rid in self._cancel

    def _gpu_runner(self):
        import torch
        device = torch.cuda.current_device()
        streams = [torch.cuda.Stream(device=device) for _ in range(self.slots)]

        def run(req, slot, should_stop):
            torch.cuda.set_device(device)
            return run_request(req, self.precision, self.real, streams[slot].cuda_stream, self.chunk,
                               should_stop, self.tuner)
        return run

    def run(self, requests):
        """Serve `requests`, whose .arrival times count from this call.
        Returns results ordered by request id; self.stats holds the run's
        makespan, peak concurrency, peak admitted bytes and, with grouping,
        the largest group stepped in one launch."""
        runner = self.runner
        budget = self.hbm_budget
        device = None
        if self.grouping or runner is None or budget is None:
            import torch
            device = torch.cuda.current_device()
            if runner is None and not self.grouping:
                runner = self._gpu_runner()
            if budget is None:
                budget = int(0.9 * torch.cuda.mem_get_info()[0])
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        cv = threading.Condition()
        st = {"mem": 0, "active": 0, "free": list(range(self.slots)), "peak_active": 0, "peak_mem": 0,
              "peak_group": 0}
        results = {}
        groups = {}
        t0 = time.perf_counter()

        def finish(req, slot, nbytes, admitted, det, dt, err):
            end = time.perf_counter() - t0
            with cv:
                results[req.rid] = Result(req.rid, det, dt, req.arrival, admitted, end, slot, err)
                st["mem"] -= nbytes
                st["active"] -= 1
                st["free"].append(slot)
                cv.notify_all()

        def worker(req, slot, nbytes, admitted):
            err, det, dt = None, None, float("nan")
            try:
                det, dt = runner(req, slot, lambda: self._cancelled(req.rid))
            except Exception as e:  # noqa: BLE001 - the failure is the request's result
                err = f"{type(e).__name__}: {e}"
            finish(req, slot, nbytes, admitted, det, dt, err)

        def group_worker(key):
            import torch
            from . import RTEError, step_group
            torch.cuda.set_device(device)
            stream = torch.cuda.Stream(device=device)
            members = []
            while True:
                with cv:
                    incoming = groups[key]
                    groups[key] = []
                    if not members and not incoming:
                        del groups[key]
                        return
                for req, slot, nbytes, admitted in incoming:
                    try:
                        plan, dt = open_plan(req, self.precision, self.real, stream.cuda_stream, self.tuner)
                    except Exception as e:  # noqa: BLE001
                        finish(req, slot, nbytes, admitted, None, float("nan"), f"{type(e).__name__}: {e}")
                        continue
                    members.append({"req": req, "slot": slot, "nbytes": nbytes, "admitted": admitted,
                                    "plan": plan, "dt": dt, "done": 0, "parts": []})
                for mb in list(members):
                    if self._cancelled(mb["req"].rid):
                        mb["plan"].close()
                        members.remove(mb)
                        finish(mb["req"], mb["slot"], mb["nbytes"], mb["admitted"], None, float("nan"),
                               f"Cancelled: request {mb['req'].rid} cancelled after {mb['done']} steps")
                if not members:
                    continue
                batch = members[:8]
                k = min([self.chunk] + [mb["req"].nsteps - mb["done"] for mb in batch])
                try:
                    dets = step_group([mb["plan"] for mb in batch], [mb["dt"] for mb in batch], k)
                    with cv:
                        st["peak_group"] = max(st["peak_group"], len(batch))
                except RTEError as e:
                    if e.status != 8:        # RTE_ERR_UNSUPPORTED: this shape steps plan by plan
                        raise
                    dets = [mb["plan"].step(mb["dt"], k)[0] for mb in batch]
                for mb, d in zip(batch, dets):
                    mb["parts"].append(d if d is not None else np.zeros((k, 0)))
                    mb["done"] += k
                members = members[len(batch):] + batch          # the next turn starts with the others
                for mb in [mb for mb in members if mb["done"] >= mb["req"].nsteps]:
                    mb["plan"].close()
                    members.remove(mb)
                    finish(mb["req"], mb["slot"], mb["nbytes"], mb["admitted"],
                           np.concatenate(mb["parts"], axis=0), mb["dt"], None)

        threads = []
        for req in pending:
            nbytes = int(self.sizer(req))
            if nbytes > budget:
                now = time.perf_counter() - t0
                results[req.rid] = Result(req.rid, None, float("nan"), req.arrival, now, now, -1,
                                          f"rejected: needs {nbytes} bytes, HBM budget is {budget}")
                continue
            with cv:
                while True:
                    now = time.perf_counter() - t0
                    if (now >= req.arrival and st["active"] < self.slots
                            and st["mem"] + nbytes <= budget):
                        break
                    cv.wait(timeout=min(0.05, max(req.arrival - now, 1e-4)))
                if self._cancelled(req.rid):
                    results[req.rid] = Result(req.rid, None, float("nan"), req.arrival, now, now, -1,
                                              "cancelled before admission")
                    continue
                slot = st["free"].pop(0)
                st["mem"] += nbytes
                st["active"] += 1
                st["peak_active"] = max(st["peak_active"], st["active"])
                st["peak_mem"] = max(st["peak_mem"], st["mem"])
                if self.grouping:
                    key = (tuple(req.shape), req.N)
                    start = key not in groups
                    groups.setdefault(key, []).append((req, slot, nbytes, now))
            if self.grouping:
                if start:
                    th = threading.Thread(target=group_worker, args=(key,), daemon=True)
                    th.start()
                    threads.append(th)
                continue
            th = threading.Thread(target=worker, args=(req, slot, nbytes, now), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        self.stats = {"makespan_s": time.perf_counter() - t0, "peak_active": st["peak_active"],
                      "peak_bytes": st["peak_mem"], "budget_bytes": budget}
        if self.grouping:
            self.stats["peak_group"] = st["peak_group"]
        return [results[k] for k in sorted(results)]


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """n arrival times of a Poisson process of `rate` per second, from the
    seeded splitmix64 stream (exponential gaps by inversion)."""
    import synth
    u = synth.Stream(seed).uniform(n, 0.0, 1.0)
    return np.cumsum(-np.log1p(-u) / rate)


def summarize(results, requests, makespan):
    """Latency percentiles over the completed requests, and throughput in
    moment-voxel updates per second over the run."""
    ok = [r for r in results if r.ok]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    done = {r.rid for r in ok}
    ups = sum(q.updates for q in requests if q.rid in done)
    return {"requests": len(results), "completed": len(ok),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "makespan_s": float(makespan),
            "updates_per_s": ups / makespan if makespan > 0 else 0.0}
