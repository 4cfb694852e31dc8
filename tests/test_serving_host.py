"""Host logic of the serving loop: admission by slot and HBM footprint, FIFO
order, arrivals, rejection, failures and cancellation, driven with stand-in
runners on the CPU (no GPU, no plan)."""
import threading
import time

import numpy as np
import pytest

import synth
from paper_1801_06364_b300.serving import Request, Server, poisson_arrivals, summarize


def req(rid, arrival=0.0, nsteps=10, n=8, N=1):
    z = np.zeros((n, n, n))
    return Request(rid, (n, n, n), 0.25, N, 0.214, z, z, z, nsteps, arrival=arrival)


class Recorder:
    """Stand-in runner: sleeps, records the concurrency it saw."""

    def __init__(self, seconds=0.05, fail=(), wait_for_cancel=()):
        self.seconds = seconds
        self.fail = set(fail)
        self.wait_for_cancel = set(wait_for_cancel)
        self.lock = threading.Lock()
        self.active = 0
        self.peak = 0
        self.slots_in_use = set()
        self.slot_clash = False
        self.started = {}

    def __call__(self, r, slot, should_stop):
        with self.lock:
            self.active += 1
            self.peak = max(self.peak, self.active)
            if slot in self.slots_in_use:
                self.slot_clash = True
            self.slots_in_use.add(slot)
            self.started[r.rid] = time.perf_counter()
        try:
            if r.rid in self.fail:
                raise RuntimeError("injected failure")
            if r.rid in self.wait_for_cancel:
                for _ in range(400):        # bounded: 4 s at most
                    if should_stop():
                        raise RuntimeError("stopped")
                    time.sleep(0.01)
            time.sleep(self.seconds)
            return np.full((r.nsteps, 2), float(r.rid)), 0.01
        finally:
            with self.lock:
                self.active -= 1
                self.slots_in_use.discard(slot)


def test_slots_bound_concurrency_and_all_complete():
    rec = Recorder(0.05)
    s = Server(slots=3, hbm_budget=1 << 40, runner=rec, sizer=lambda r: 1)
    rs = [req(i) for i in range(9)]
    out = s.run(rs)
    assert [r.rid for r in out] == list(range(9)) and all(r.ok for r in out)
    assert rec.peak == 3 and s.stats["peak_active"] == 3 and not rec.slot_clash
    assert all(np.all(r.readouts == r.rid) for r in out)
    # 9 requests of 50 ms over 3 slots: three waves, not nine
    assert s.stats["makespan_s"] < 9 * 0.05


def test_hbm_budget_limits_admission():
    rec = Recorder(0.03)
    s = Server(slots=8, hbm_budget=100, runner=rec, sizer=lambda r: 40)
    out = s.run([req(i) for i in range(6)])
    assert all(r.ok for r in out)
    assert rec.peak == 2 and s.stats["peak_bytes"] <= 100


def test_oversize_request_rejected_others_served():
    rec = Recorder(0.01)
    sizes = {0: 10, 1: 500, 2: 10}
    s = Server(slots=2, hbm_budget=100, runner=rec, sizer=lambda r: sizes[r.rid])
    out = s.run([req(i) for i in range(3)])
    assert out[0].ok and out[2].ok
    assert not out[1].ok and out[1].error.startswith("rejected")
    assert 1 not in rec.started


def test_arrivals_respected_and_fifo():
    rec = Recorder(0.0)
    arr = [0.0, 0.05, 0.10, 0.15]
    s = Server(slots=1, hbm_budget=1 << 40, runner=rec, sizer=lambda r: 1)
    out = s.run([req(i, a) for i, a in zip((3, 1, 2, 0), arr)])
    for r in out:
        assert r.admitted >= r.arrival - 1e-6
    order = sorted(rec.started, key=rec.started.get)
    assert order == [3, 1, 2, 0]


def test_failure_is_the_requests_result_only():
    rec = Recorder(0.01, fail={2})
    s = Server(slots=2, hbm_budget=1 << 40, runner=rec, sizer=lambda r: 1)
    out = s.run([req(i) for i in range(5)])
    assert [r.ok for r in out] == [True, True, False, True, True]
    assert "injected failure" in out[2].error
    assert s.stats["peak_active"] <= 2


def test_cancel_waiting_and_running_requests():
    rec = Recorder(0.01, wait_for_cancel={0})
    s = Server(slots=1, hbm_budget=1 << 40, runner=rec, sizer=lambda r: 1)
    s.cancel(2)                                   # never admitted
    t = threading.Timer(0.1, s.cancel, args=(0,))  # stops the running one
    t.start()
    out = s.run([req(i) for i in range(3)])
    t.join()
    assert not out[0].ok and "stopped" in out[0].error
    assert out[1].ok
    assert not out[2].ok and out[2].error == "cancelled before admission" and 2 not in rec.started


def test_summary_counts_completed_work():
    rec = Recorder(0.01, fail={1})
    rs = [req(i, nsteps=5, n=8, N=1) for i in range(4)]
    s = Server(slots=4, hbm_budget=1 << 40, runner=rec, sizer=lambda r: 1)
    out = s.run(rs)
    sm = summarize(out, rs, s.stats["makespan_s"])
    assert sm["completed"] == 3 and sm["requests"] == 4
    assert sm["updates_per_s"] == pytest.approx(3 * 4 * 512 * 5 / s.stats["makespan_s"])
    assert sm["p50_latency_s"] <= sm["p99_latency_s"]


def test_poisson_arrivals_are_seeded_and_have_the_rate():
    a = poisson_arrivals(4000, 5.0, 17)
    assert np.all(np.diff(a) >= 0) and np.array_equal(a, poisson_arrivals(4000, 5.0, 17))
    gaps = np.diff(np.concatenate([[0.0], a]))
    # exponential gaps: mean 1/rate, standard deviation 1/rate
    assert abs(gaps.mean() - 0.2) < 4 * 0.2 / np.sqrt(4000)
    assert abs(gaps.std() - 0.2) < 0.02


def test_serving_request_mix_follows_the_recipe():
    seen_n, seen_N = set(), set()
    for i in range(40):
        w = synth.c4_request(i)
        n, N = w.shape[0], w.N
        assert n in (64, 96, 128, 160) and N in (3, 5, 7, 9) and 500 <= w.nsteps <= 3000
        assert w.pml_width == 12 and len(w.det_voxel) == 16 and w.dx == 0.25
        assert 0.005 <= w.mua.min() and w.mua.max() <= 0.1 and 2.0 <= w.mus.min() and w.mus.max() <= 20.0
        assert 0.7 <= w.g.min() and w.g.max() <= 0.95
        seen_n.add(n)
        seen_N.add(N)
        r = Request.from_workload(i, w)
        assert r.updates == (N + 1) ** 2 * n ** 3 * w.nsteps
    assert seen_n == {64, 96, 128, 160} and seen_N == {3, 5, 7, 9}


def test_admission_uses_the_plan_footprint():
    """The default sizer is rte_plan_footprint of the request's plan (host
    call, no GPU): with a budget for one 64^3 P_3 plan, two such requests
    never run together and a 96^3 P_9 request is rejected."""
    from paper_1801_06364_b300.serving import plan_bytes
    small = [Request.from_workload(i, synth.c4_request(i, grids=(64,), orders=(3,), steps_range=(10, 10)))
             for i in range(2)]
    big = Request.from_workload(9, synth.c4_request(9, grids=(96,), orders=(9,), steps_range=(10, 10)))
    b_small = plan_bytes(small[0], "fp32", True)
    b_big = plan_bytes(big, "fp32", True)
    assert b_small > 4 * 10 * 64 ** 3 * 8 and b_big > b_small      # four state buffers of 10 moments at least
    rec = Recorder(0.02)
    s = Server(slots=4, hbm_budget=b_small + b_small // 2, runner=rec)
    out = s.run(small + [big])
    assert [r.ok for r in out] == [True, True, False] and out[2].error.startswith("rejected")
    assert rec.peak == 1 and s.stats["peak_bytes"] == b_small
