"""Plans that take their device memory from a caller's allocator
(rte_set_allocator, here PyTorch's caching allocator): the memory shows in
torch's accounting while the plan lives, goes back when it closes, and the
results are bitwise the same as with the library's own cudaMallocAsync."""
import numpy as np
import pytest

import paper_1801_06364_b300 as rte
import synth

pytestmark = pytest.mark.gpu


def _plan(wl, precision, stream):
    g = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                 precision, stream=stream, real_radiance=precision == "fp32")
    g.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, [0.5], [1.0])
    g.set_detectors(wl.det_voxel)
    return g


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_plan_memory_from_torch_caching_allocator(precision):
    import torch
    torch.cuda.set_device(0)
    wl = synth.c2(shape=(32, 32, 32), dx=0.4, N=3, W=3)
    stream = torch.cuda.Stream()
    s = stream.cuda_stream

    ref = _plan(wl, precision, s)
    dt = 0.5 * ref.stability_limit()
    ref.set_state(synth.real_radiance_state(3, wl.shape, wl.dx, seed=3, corr=0.8))
    det_ref, _ = ref.step(dt, 12)
    psi_ref = ref.get_state()
    ref.close()

    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    rte.use_torch_allocator(True)
    try:
        g = _plan(wl, precision, s)
        held = torch.cuda.memory_allocated() - base
        desc = rte.make_desc(wl.shape, wl.dx, wl.N, wl.c, wl.pml_width, wl.pml_mu0, wl.pml_mu1, precision,
                             real_radiance=precision == "fp32")
        assert held >= 0.9 * rte.plan_footprint(desc)
        g.set_state(synth.real_radiance_state(3, wl.shape, wl.dx, seed=3, corr=0.8))
        det, _ = g.step(dt, 12)
        psi = g.get_state()
        # the steady solver grows workspace on first use (and an FP32 plan its
        # FP64 twin): all of it from the same allocator
        before = torch.cuda.memory_allocated()
        g.set_sources(wl.src_voxel, [0], [1.0], [0.0], [0.0])   # constant source
        its, res, ok = g.solve_steady(1e-4, 8, 400)
        assert torch.cuda.memory_allocated() > before
        g.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        rte.use_torch_allocator(False)
    assert np.array_equal(psi, psi_ref)
    assert np.array_equal(det, det_ref)
    # back on the library's own allocator: torch's accounting does not move
    g = _plan(wl, precision, s)
    assert torch.cuda.memory_allocated() == base
    g.close()
