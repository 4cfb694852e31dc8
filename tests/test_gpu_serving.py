"""The serving loop on the GPU: each request's readouts are the same alone and
in a mix of concurrent requests of different grids and orders, the FP32 mix
agrees with the one-at-a-time FP64 path to the FP32 tolerance, and sampled
requests agree with the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GRIDS = (32, 40, 48, 64)      # radix 2 (fused plane path) and 2*5, 3*16 (split path)
ORDERS = (2, 3, 4, 5)


def mix(k=8, arrivals=None):
    from paper_1801_06364_b300.serving import Request
    out = []
    for i in range(k):
        w = synth.c4_request(i, grids=GRIDS, orders=ORDERS, steps_range=(60, 180), W=4)
        r = Request.from_workload(i, w, arrival=0.0 if arrivals is None else float(arrivals[i]))
        n = w.shape[0]
        c = n // 2
        # detectors near the source so that every readout carries signal at
        # these short times; pulse early and short
        r.det_voxel = np.array([synth.flat_index(w.shape, c + a, c + b, c + d)
                                for a, b, d in ((0, 0, 1), (0, 2, 0), (3, 0, 0), (1, 1, 1))], np.int64)
        r.src_t0 = np.array([1.0])
        r.src_fwhm = np.array([1.5])
        out.append(r)
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def alone():
    """Every request of the mix run by itself on the legacy default stream."""
    from paper_1801_06364_b300.serving import run_request
    return {r.rid: run_request(r, "fp32", True, None, 50) for r in mix()}


@pytest.mark.parametrize("slots", [3, 8])
def test_results_identical_alone_and_in_the_mix(alone, slots):
    from paper_1801_06364_b300.serving import Server
    rs = mix()
    s = Server(slots=slots, precision="fp32", real_radiance=True, chunk=50)
    out = s.run(rs)
    assert all(r.ok for r in out), [r.error for r in out if not r.ok]
    assert s.stats["peak_active"] == min(slots, len(rs))
    for r in out:
        det, dt = alone[r.rid]
        assert r.dt == dt
        assert r.readouts.shape == det.shape and np.array_equal(r.readouts, det), r.rid


def test_poisson_mix_identical_and_agrees_with_one_at_a_time_fp64(alone):
    from paper_1801_06364_b300.serving import Server, poisson_arrivals
    arr = poisson_arrivals(8, 40.0, 5)
    rs = mix(arrivals=arr)
    out = Server(slots=4, precision="fp32", chunk=50).run(rs)
    ref = Server(slots=1, precision="fp64", real_radiance=False, chunk=50).run(mix())
    for r, q in zip(out, ref):
        assert r.ok and q.ok
        assert r.admitted >= r.arrival - 1e-6
        assert np.array_equal(r.readouts, alone[r.rid][0])
        # the FP32 path against the FP64 path at the same dt (the limit is
        # computed in FP64 on the host for both)
        assert q.dt == pytest.approx(r.dt, rel=1e-12)
        assert rel(r.readouts, q.readouts) < 1e-5, r.rid


def test_sampled_requests_match_the_oracle():
    """The two cheapest requests of the mix, served concurrently with the
    rest, against the FP64 oracle at the dt the plan chose."""
    from paper_1801_06364_b300.serving import Server
    rs = mix()
    cost = sorted(rs, key=lambda r: (r.N + 1) ** 2 * np.prod(r.shape) * r.nsteps)
    pick = {r.rid for r in cost[:2]}
    f32 = Server(slots=8, precision="fp32").run(rs)
    f64 = Server(slots=8, precision="fp64", real_radiance=False).run(mix())
    for r in rs:
        if r.rid not in pick:
            continue
        p = oracle.Problem(r.N, r.shape, r.dx, r.c, r.mua, r.mus, r.g, r.pml_cells, r.pml_mu0, r.pml_mu1)
        src = oracle.Sources(r.src_voxel, np.zeros(1, np.int32), r.src_amp, r.src_t0, r.src_fwhm)
        _, det, _ = oracle.run(p, np.zeros((p.M,) + p.shape), f64[r.rid].dt, r.nsteps, sources=src,
                               det_voxels=r.det_voxel)
        assert rel(f64[r.rid].readouts, det) < 1e-12
        assert rel(f32[r.rid].readouts, det) < 1e-5


def test_concurrent_plans_with_different_shared_memory_sizes():
    """Split-path kernels whose dynamic shared memory differs per grid (FP64,
    80^3 and 96^3 lines, over 48 KB each) launched from four host threads at
    once: the per-function shared-memory limit must not be lowered by one
    plan under another's launch."""
    from paper_1801_06364_b300.serving import Request, Server
    rs = []
    for i, n in enumerate((80, 96, 80, 96)):
        w = synth.c4_request(i, grids=(n,), orders=(5,), steps_range=(120, 120), W=4)
        rs.append(Request.from_workload(i, w))
    out = Server(slots=4, precision="fp64", real_radiance=True, chunk=3).run(rs)
    assert all(r.ok for r in out), [r.error for r in out if not r.ok]
    again = Server(slots=1, precision="fp64", real_radiance=True, chunk=3).run(rs)
    for a, b in zip(out, again):
        assert np.array_equal(a.readouts, b.readouts)


def same_shape_mix(k=6, n=32, N=3):
    """k requests of one grid and order (different media, sources, detectors,
    step counts), for grouping."""
    from paper_1801_06364_b300.serving import Request
    out = []
    for i in range(k):
        w = synth.c4_request(100 + i, grids=(n,), orders=(N,), steps_range=(60, 180), W=4)
        r = Request.from_workload(i, w)
        c = n // 2
        r.det_voxel = np.array([synth.flat_index(w.shape, c + a, c + b, c + d)
                                for a, b, d in ((0, 0, 1), (0, 2, 0), (3, 0, 0))], np.int64)
        r.src_t0 = np.array([1.0])
        r.src_fwhm = np.array([1.5])
        out.append(r)
    return out


def test_grouped_launches_identical_to_each_request_alone():
    """Same-shape requests served with grouping (one launch of each step pass
    for the whole group, rte_step_group) give bitwise the readouts of each
    request run alone, also when the group has more members than one launch
    takes (9 > 8: the group steps in turns) and with a mixed-shape load."""
    from paper_1801_06364_b300.serving import Server, run_request
    rs = same_shape_mix(9) + [r for r in mix(4)]
    for i, r in enumerate(rs):
        r.rid = i
    alone = {r.rid: run_request(r, "fp32", True, None, 50) for r in rs}
    s = Server(slots=13, precision="fp32", real_radiance=True, chunk=50, grouping=True)
    out = s.run(rs)
    assert all(r.ok for r in out), [r.error for r in out if not r.ok]
    assert s.stats["peak_group"] == 8
    for r in out:
        det, dt = alone[r.rid]
        assert r.dt == dt
        assert np.array_equal(r.readouts, det), r.rid


def test_step_group_matches_single_plans_with_states_and_integrals():
    """rte_step_group on three plans with different media and dt against
    rte_step on each: states bitwise equal after 37 steps (an odd count over
    graph replays of 4), readouts equal, plan times advanced by their own dt."""
    import paper_1801_06364_b300 as R
    rs = same_shape_mix(3)
    ref, plans, dts = [], [], []
    import torch
    st = torch.cuda.Stream()
    for r in rs:
        from paper_1801_06364_b300.serving import open_plan
        p, dt = open_plan(r, "fp32", True, st.cuda_stream)
        p.set_schedule("plane", 4)
        plans.append(p)
        dts.append(dt)
        q, dtq = open_plan(r, "fp32", True, None)
        det, _ = q.step(dtq, 37)
        ref.append((det, q.get_state()))
        q.close()
    dets = R.step_group(plans, dts, 37)
    for p, d, (det, state), dt in zip(plans, dets, ref, dts):
        assert np.array_equal(d, det)
        assert np.array_equal(p.get_state(), state)
        assert p.get_time() == pytest.approx(37 * dt, rel=1e-12)
        p.close()


def test_autotuner_pins_one_choice_per_shape(tmp_path):
    """The autotuner times the plane and split schedules and the graph sizes
    for a shape, keeps the fastest, writes it to its file and returns the same
    choice afterwards (also from a new tuner reading the file); a request
    served with the tuned schedule matches the same request run alone with it."""
    from paper_1801_06364_b300.autotune import Autotuner, key_of
    from paper_1801_06364_b300.serving import Server, run_request
    path = str(tmp_path / "tune.json")
    t = Autotuner(path, steps=8, repeats=2)
    c1 = t.choice((32, 32, 32), 3, "fp32", True, 0.25, 0.214, 4, 2.0, 10.0)
    assert c1["schedule"] in ("plane", "split") and c1["graph_steps"] in (2, 4, 8, 16)
    assert set(c1["candidates_ms_per_step"]) >= {"plane/2", "split/2"}
    assert min(c1["candidates_ms_per_step"].values()) == c1["ms_per_step"]
    assert t.choice((32, 32, 32), 3, "fp32", True) is c1
    t2 = Autotuner(path)
    assert t2.cache[key_of((32, 32, 32), 3, "fp32", True)] == c1
    rs = same_shape_mix(3)
    out = Server(slots=3, precision="fp32", real_radiance=True, chunk=50, tuner=t2).run(rs)
    for r in out:
        det, _ = run_request(rs[r.rid], "fp32", True, None, 50, tuner=t2)
        assert r.ok and np.array_equal(r.readouts, det)
