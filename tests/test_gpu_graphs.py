"""Steps replayed from captured CUDA graphs against the same steps launched
kernel by kernel (per-kernel profiling turns the graphs off): bitwise equal
state and readouts, equal kernel counts, and agreement with the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rte():
    import paper_1801_06364_b300 as m
    return m


def make(wl, precision, stream, real=False):
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                   precision, stream=stream, real_radiance=real)
    g.set_sources(wl.src_voxel, [0], [1.0], [0.3], [0.6])
    g.set_detectors(wl.det_voxel)
    return g


@pytest.mark.parametrize("shape", [(16, 32, 32), (20, 24, 40)])      # fused plane path, split path
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("on_torch_stream", [False, True])
def test_graph_replay_equals_plain_launches(shape, precision, on_torch_stream):
    import torch
    m = rte()
    wl = synth.c2(shape=shape, dx=0.4, N=3, W=3, nsteps=0)
    st = torch.cuda.Stream().cuda_stream if on_torch_stream else None
    plain, graph = make(wl, precision, st), make(wl, precision, st)
    plain.profile(True)
    psi = synth.smooth_random_state(wl.N, shape, wl.dx, seed=3, corr=0.8)
    plain.set_state(psi)
    graph.set_state(psi)
    dt = 0.5 * plain.stability_limit()
    for n, f in ((25, 1.0), (8, 1.0), (9, 0.7)):      # reuse of the graph, then a new dt
        l0 = m.kernel_launches()
        dp, _ = plain.step(f * dt, n)
        l1 = m.kernel_launches()
        dg, _ = graph.step(f * dt, n)
        l2 = m.kernel_launches()
        assert np.array_equal(dp, dg)
        assert l1 - l0 == l2 - l1 > 0
    assert np.array_equal(plain.get_state(), graph.get_state())


def test_graph_replay_matches_oracle():
    import torch
    wl = synth.c2(shape=(16, 32, 32), dx=0.4, N=3, W=3, nsteps=0)
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1)
    g = make(wl, "fp64", torch.cuda.Stream().cuda_stream)
    dt = 0.5 * g.stability_limit()
    det, _ = g.step(dt, 30)
    src = oracle.Sources(wl.src_voxel, np.zeros(1, np.int32), np.array([1.0]), np.array([0.3]), np.array([0.6]))
    want, det_w, _ = oracle.run(p, np.zeros((p.M,) + p.shape), dt, 30, sources=src, det_voxels=wl.det_voxel)
    got = g.get_state()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    assert np.linalg.norm(det - det_w) / np.linalg.norm(det_w) < 1e-12
