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
