"""Steady-state GMRES (row a5) and the discrete adjoint (row a6) of the CUDA
path against the oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rte():
    import paper_1801_06364_b300 as m
    return m


def wnorm(N, u):
    wl = np.array([2 * l + 1 for l in range(N + 1) for _ in range(2 * l + 1)], dtype=float)
    return math.sqrt(float(np.sum(wl[:, None] * np.abs(u.reshape(u.shape[0], -1)) ** 2)))


def steady_case(shape=(12, 16, 20), N=3, W=3):
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    p = oracle.Problem(N, shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    q = np.zeros((p.M,) + shape, complex)
    q.reshape(p.M, -1)[0, wl.src_voxel[0]] = 1.0 / wl.dx ** 3
    return wl, p, q


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("shape", [(12, 16, 20), (16, 32, 32)])
@pytest.mark.parametrize("precision,rtol,soltol", [("fp64", 1e-10, 1e-8), ("fp32", 1e-8, 1e-5)])
def test_steady_state_gmres_matches_oracle(precision, rtol, soltol, shape, real):
    """T psi = q for a CW point source in heterogeneous media with the layer.
    FP32 plans refine FP32 GMRES corrections with FP64 residuals, so they
    reach the same rtol; the returned FP32 state then differs from the FP64
    solution by its rounding only."""
    wl, p, q = steady_case(shape)
    want, it, rr, ok = oracle.gmres(p, q, restart=30, max_iter=5000, rtol=1e-12)
    assert ok
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                   wl.pml_mu1, precision, real_radiance=real)
    g.set_sources(wl.src_voxel, [0], [1.0], [0.0], [0.0])
    iters, rel, conv = g.solve_steady(rtol=rtol, restart=30, max_iter=5000)
    assert conv and rel <= rtol
    got = g.get_state()
    # the paper's equation holds when checked with the oracle's FP64 operator: to
    # rtol for FP64; for FP32 the returned state is the refined FP64 solution
    # rounded to FP32, whose residual is that rounding (~6e-8 relative) times
    # |T| |psi| / |q|
    res = q - oracle.apply_T(p, got.astype(complex))
    assert wnorm(p.N, res) / wnorm(p.N, q) < (2 * rtol if precision == "fp64" else 1e-6)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < soltol, (err, iters)


def test_gmres_not_converged_reports_and_plan_stays_usable():
    m = rte()
    wl, p, q = steady_case((8, 8, 8), 2, 2)
    g = m.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1, "fp64")
    g.set_sources(wl.src_voxel, [0], [1.0], [0.0], [0.0])
    it, rel, conv = g.solve_steady(rtol=1e-14, restart=5, max_iter=3)
    assert not conv and it == 3 and rel > 1e-14
    it, rel, conv = g.solve_steady(rtol=1e-9, restart=20, max_iter=4000)
    assert conv


def adjoint_case(shape=(12, 12, 16), N=2, W=2, nsteps=40):
    wl = synth.c5(shape=shape, dx=0.5, N=N, W=W, nsteps=nsteps, nsrc=2, ndet=3)
    t0 = np.array([0.4, 0.7])
    fw = np.array([0.6, 0.6])
    gates = np.array([[0.1, 1.2], [0.5, 2.0], [0.0, 3.0]])
    p = oracle.Problem(N, shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    dt = 0.5 * oracle.stability_limit(p)
    return wl, p, t0, fw, gates, dt


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
@pytest.mark.parametrize("K,shape", [(7, (12, 12, 16)), (40, (12, 12, 16)), (7, (10, 32, 32))])
def test_adjoint_gradient_matches_oracle(precision, tol, K, shape, real):
    """Checkpointed adjoint (every K steps, ragged last segment for K = 7)
    against the oracle's stored-trajectory adjoint, L = sum_d y_d^2. The
    32 x 32 planes take the fused plane kernel for the recomputed segments
    and the adjoint steps (gradient terms in its X2 phase); 12 x 16 planes
    the split passes.

    The two sweeps are checked separately. Forward: each gated readout
    y_d = sum_s w_sd Re psi_00(r_d, t_s) against the oracle, relative to the
    same sum of the field's largest |Re psi_00| (some readouts here are 1e-9
    of the field, so their own relative error measures FP32 rounding of the
    field, not of the method). Adjoint: the gradient against the oracle's
    adjoint driven by the same dL/dy = 2 y, in relative L2."""
    wl, p, t0, fw, gates, dt = adjoint_case(shape)
    ns = 40
    src = oracle.Sources(wl.src_voxel, np.zeros(2, np.int32), wl.src_amp, t0, fw)
    _, det, _ = oracle.run(p, np.zeros((p.M,) + p.shape), dt, ns, sources=src, det_voxels=wl.det_voxel)
    _, field, _ = oracle.run(p, np.zeros((p.M,) + p.shape), dt, ns, sources=src, det_voxels=np.arange(p.V))
    y_w, w = oracle.gated_readouts(det, dt, 0.0, gates)
    scale = (w * np.max(np.abs(field), axis=1)[:, None]).sum(axis=0)
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                   wl.pml_mu1, precision, real_radiance=real)
    g.set_sources(wl.src_voxel, [0, 0], wl.src_amp, t0, fw)
    g.set_detectors(wl.det_voxel)
    y = g.forward(dt, ns, K, gates)
    assert np.max(np.abs(y - y_w) / scale) < (1e-15 if precision == "fp64" else 1e-7)
    if precision == "fp64":
        assert np.linalg.norm(y - y_w) / np.linalg.norm(y_w) < 1e-12
    ga_w, gs_w = oracle.adjoint(p, np.zeros((p.M,) + p.shape), dt, ns, w * (2 * y)[None, :],
                                wl.det_voxel, sources=src)
    ga, gs = g.adjoint(2 * y)
    g.close()
    if precision == "fp32" and np.max(np.abs(y_w) / scale) < 1e-3:
        # Detectors the light barely reaches in 40 steps (readouts under 1e-3
        # of the field scale): the adjoint's source dL/dy is then that small
        # and the gradient, a sum of lambda psi products, cancels to a
        # fraction of their size. Check FP32 on detectors next to the
        # sources instead, where the readouts are of the field's order.
        near = np.array([v + 1 for v in wl.src_voxel] + [v - 1 for v in wl.src_voxel[:1]], dtype=np.int64)
        _, det_n, _ = oracle.run(p, np.zeros((p.M,) + p.shape), dt, ns, sources=src, det_voxels=near)
        y_n, w_n = oracle.gated_readouts(det_n, dt, 0.0, gates)
        assert np.max(np.abs(y_n) / scale) > 1e-2
        g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                       wl.pml_mu1, precision, real_radiance=real)
        g.set_sources(wl.src_voxel, [0, 0], wl.src_amp, t0, fw)
        g.set_detectors(near)
        y = g.forward(dt, ns, K, gates)
        ga_w, gs_w = oracle.adjoint(p, np.zeros((p.M,) + p.shape), dt, ns, w_n * (2 * y)[None, :],
                                    near, sources=src)
        ga, gs = g.adjoint(2 * y)
        g.close()
    ga = ga.cpu().numpy()
    gs = gs.cpu().numpy()
    assert np.linalg.norm(ga - ga_w) / np.linalg.norm(ga_w) < tol
    assert np.linalg.norm(gs - gs_w) / np.linalg.norm(gs_w) < tol
    assert np.all(ga[p.mask.astype(bool)] == 0) and np.all(gs[p.mask.astype(bool)] == 0)


def test_adjoint_gradient_matches_central_differences_fp64():
    """dL/dmu_a and dL/dmu_s at a few voxels against central differences of the
    FP64 GPU forward sweep (h = 1e-4 mu)."""
    m = rte()
    wl, p, t0, fw, gates, dt = adjoint_case()
    ns = 40

    def loss(mua, mus):
        g = m.Plan(wl.shape, wl.dx, wl.N, wl.c, mua, mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1, "fp64")
        g.set_sources(wl.src_voxel, [0, 0], wl.src_amp, t0, fw)
        g.set_detectors(wl.det_voxel)
        y = g.forward(dt, ns, 10, gates)
        return float(np.sum(y * y)), y, g

    L0, y, g = loss(wl.mua, wl.mus)
    ga, gs = g.adjoint(2 * y)
    ga = ga.cpu().numpy()
    gs = gs.cpu().numpy()
    for v in np.argsort(-np.abs(ga).ravel())[:3]:
        idx = np.unravel_index(v, wl.shape)
        for base, grad, which in ((wl.mua, ga, "a"), (wl.mus, gs, "s")):
            h = 1e-4 * base[idx]
            plus, minus = base.copy(), base.copy()
            plus[idx] += h
            minus[idx] -= h
            if which == "a":
                fd = (loss(plus, wl.mus)[0] - loss(minus, wl.mus)[0]) / (2 * h)
            else:
                fd = (loss(wl.mua, plus)[0] - loss(wl.mua, minus)[0]) / (2 * h)
            assert fd == pytest.approx(grad[idx], rel=1e-5, abs=1e-10 * abs(L0))


def test_autograd_function_matches_oracle_gradient():
    import torch
    from paper_1801_06364_b300.autograd import SweepSpec, TransportReadouts
    wl, p, t0, fw, gates, dt = adjoint_case()
    ns = 40
    spec = SweepSpec(wl.shape, wl.dx, wl.N, wl.c, wl.g, dt, ns, 8, wl.src_voxel, wl.src_amp, t0, fw,
                     wl.det_voxel, gates, wl.pml_width, wl.pml_mu0, wl.pml_mu1, "fp64")
    mua = torch.tensor(wl.mua, device="cuda", requires_grad=True)
    mus = torch.tensor(wl.mus, device="cuda", requires_grad=True)
    y = TransportReadouts.apply(mua, mus, spec)
    (y * y).sum().backward()
    src = oracle.Sources(wl.src_voxel, np.zeros(2, np.int32), wl.src_amp, t0, fw)
    _, det, _ = oracle.run(p, np.zeros((p.M,) + p.shape), dt, ns, sources=src, det_voxels=wl.det_voxel)
    y_w, w = oracle.gated_readouts(det, dt, 0.0, gates)
    ga_w, gs_w = oracle.adjoint(p, np.zeros((p.M,) + p.shape), dt, ns, w * (2 * y_w)[None, :],
                                wl.det_voxel, sources=src)
    assert np.linalg.norm(mua.grad.cpu().numpy() - ga_w) / np.linalg.norm(ga_w) < 1e-11
    assert np.linalg.norm(mus.grad.cpu().numpy() - gs_w) / np.linalg.norm(gs_w) < 1e-11


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_preconditioner_cuts_iterations_same_solution(precision, real):
    """The low-order right preconditioner (the default) reaches the same
    solution as plain GMRES, both against the oracle's, in fewer steps."""
    wl, p, q = steady_case((16, 32, 32))
    want, _, _, ok = oracle.gmres(p, q, restart=30, max_iter=5000, rtol=1e-12)
    assert ok
    runs = {}
    for kind in ("none", "low"):
        g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                       wl.pml_mu1, precision, real_radiance=real)
        g.set_sources(wl.src_voxel, [0], [1.0], [0.0], [0.0])
        g.set_preconditioner(kind)
        it, rel, conv = g.solve_steady(rtol=1e-8, restart=20, max_iter=5000)
        assert conv and rel <= 1e-8
        got = g.get_state()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < (1e-6 if precision == "fp64" else 2e-5)
        runs[kind] = it
    # 411 -> 265 Arnoldi steps on this small case; the diffusive 256^3 C3 problem gains far more
    assert runs["low"] < 0.8 * runs["none"], runs


def test_preconditioner_rejects_unknown_kind():
    m = rte()
    wl, p, q = steady_case((8, 8, 8), 2, 2)
    g = m.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1, "fp64")
    st = m.lib().rte_set_preconditioner(g.handle, 7)
    assert st == m.RTE_ERR_INVALID_ARG
