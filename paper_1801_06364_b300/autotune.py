"""Autotuner for the explicit step: per (grid, order, precision, layout) it
times the candidate schedules on the GPU and keeps the fastest.

Candidates, all set through rte_set_schedule:
  - schedule: the fused plane path (z pass with the streaming coupling, then
    one fused pass per moment and z plane) where the grid allows it, or the
    split passes;
  - steps per replayed step graph: 2, 4, 8, 16 (fewer launches from the host
    for small grids, where the launch rate limits the step).
Each candidate runs a warm-up and then `repeats` timed runs of `steps` steps
with detector readouts, timed with CUDA events on the plan's stream; the
median decides. Choices are kept in memory and, when a path is given, in a
JSON file, so that a choice made once is pinned for every later request with
the same key (the serving loop relies on that for results that are the same
alone and in a mix).
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

GRAPH_STEPS = (2, 4, 8, 16)


def key_of(shape, N, precision, real_radiance) -> str:
    nz, ny, nx = (int(s) for s in shape)
    return f"{nx}x{ny}x{nz}/N{int(N)}/{precision}/{'real' if real_radiance else 'full'}"


class Autotuner:
    def __init__(self, path: str | None = None, steps: int = 32, repeats: int = 3):
        self.path = path
        self.steps = int(steps)
        self.repeats = int(repeats)
        self.cache: dict = {}
        self._lock = threading.Lock()
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    def choice(self, shape, N, precision="fp32", real_radiance=True, dx=0.25, c=0.214, pml_cells=0,
               pml_mu0=0.0, pml_mu1=0.0, stream=None) -> dict:
        """The pinned choice for this key, tuned on first use."""
        k = key_of(shape, N, precision, real_radiance)
        with self._lock:
            if k in self.cache:
                return self.cache[k]
            cfg = self._tune(shape, N, precision, real_radiance, dx, c, pml_cells, pml_mu0, pml_mu1, stream)
            self.cache[k] = cfg
            if self.path:
                tmp = self.path + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.cache, f, indent=1, sort_keys=True)
                os.replace(tmp, self.path)
            return cfg

    @staticmethod
    def apply(plan, cfg: dict):
        plan.set_schedule(cfg["schedule"], cfg["graph_steps"])

    def _tune(self, shape, N, precision, real, dx, c, pml_cells, pml_mu0, pml_mu1, stream):
        import torch

        from . import RTEError, Plan
        nz, ny, nx = (int(s) for s in shape)
        # a typical tissue-like medium with the request's layer; a pulsed
        # source at the centre and 16 detectors, as the serving requests have
        plan = Plan(shape, dx, N, c, 0.01, 10.0, 0.9, pml_cells, pml_mu0, pml_mu1, precision, stream=stream,
                    real_radiance=real)
        try:
            centre = (nz // 2 * ny + ny // 2) * nx + nx // 2
            plan.set_sources([centre], [0], [1.0], [1.0], [1.0])
            W = max(pml_cells, 1)
            rng = np.random.default_rng(1801063640)
            dets = ((rng.integers(W, nz - W, 16) * ny + rng.integers(W, ny - W, 16)) * nx
                    + rng.integers(W, nx - W, 16))
            plan.set_detectors(dets)
            dt = 0.5 * plan.stability_limit()
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            scheds = ["plane", "split"]
            timings = {}
            for sched in scheds:
                try:
                    plan.set_schedule(sched, 2)
                except RTEError:
                    continue            # the plane path does not take this grid
                for gs in GRAPH_STEPS:
                    plan.set_schedule(sched, gs)
                    plan.step(dt, 2 * gs + 2)        # warm-up, captures the graph
                    runs = []
                    for _ in range(self.repeats):
                        e0.record(st)
                        plan.step(dt, self.steps)
                        e1.record(st)
                        e1.synchronize()
                        runs.append(e0.elapsed_time(e1) / self.steps)
                    timings[f"{sched}/{gs}"] = float(np.median(runs))
            best = min(timings, key=timings.get)
            sched, gs = best.split("/")
            return {"schedule": sched, "graph_steps": int(gs), "ms_per_step": timings[best],
                    "candidates_ms_per_step": timings}
        finally:
            plan.close()
