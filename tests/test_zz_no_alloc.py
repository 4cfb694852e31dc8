"""The allocation-free transport entry point, rte_apply_transport_noalloc.

It serves callers that cannot allocate device memory (inside another
framework's memory pool, under a fixed memory budget, or in a plug-in that
may not call cudaMalloc), so it keeps its tables and work buffers in one
device array built into the library. These tests call it through the C ABI
and compare it with the plan-based rte_apply_transport on two calls in a row
(the second call reuses the array the first one filled), at the tolerances
the parity tests use. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _arrays(wl):
    return [np.ascontiguousarray(a, dtype=np.float64) for a in (wl.mua, wl.mus, wl.g)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_plan_entry_point_on_two_calls(precision):
    import torch
    import paper_1801_06364_b300 as rte

    shape, N, W = (12, 20, 24), 3, 3
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    plan = rte.Plan(shape, wl.dx, N, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1, precision)
    desc = plan.desc
    a, s, g = _arrays(wl)
    stream = torch.cuda.current_stream()
    for seed in (11, 12):
        psi = synth.smooth_random_state(N, shape, wl.dx, seed=seed, corr=0.6)
        x = torch.from_numpy(psi.astype(plan.cdtype)).to("cuda")
        want = plan.apply_transport(x)
        got = torch.full_like(x, float("nan"))
        st = rte.lib().rte_apply_transport_noalloc(C.byref(desc), rte._dp(a), rte._dp(s), rte._dp(g),
                                                    C.c_void_p(x.data_ptr()), C.c_void_p(got.data_ptr()),
                                                    C.c_void_p(stream.cuda_stream))
        assert st == rte.RTE_OK, rte.lib().rte_last_error_string()
        w = want.cpu().numpy()
        err = np.linalg.norm(got.cpu().numpy() - w) / np.linalg.norm(w)
        assert err < TOL[precision], err
    plan.close()


def test_noalloc_rejects_problems_beyond_the_scratch_limit():
    import paper_1801_06364_b300 as rte

    desc = rte.make_desc((64, 64, 64), 0.25, 7, 0.214, 4, 2.0, 10.0, "fp64")   # ~0.8 GB of buffers
    a = np.full(64 ** 3, 0.01)
    s = np.full(64 ** 3, 10.0)
    g = np.full(64 ** 3, 0.9)
    st = rte.lib().rte_apply_transport_noalloc(C.byref(desc), rte._dp(a), rte._dp(s), rte._dp(g),
                                                C.c_void_p(16), C.c_void_p(32), None)
    assert st == rte.RTE_ERR_INVALID_ARG
    msg = rte.lib().rte_last_error_string().decode()
    assert "bytes of scratch" in msg and str(32 << 20) in msg
