"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over all moments): 1e-12 for FP64 plans, 1e-5 for
FP32 plans, the targets the method's error budget allows: FP64 rounding is
~1e-16 per operation, and an FP32 state carries ~6e-8 relative rounding per
step, which over the few hundred steps tested stays below 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def rte():
    import paper_1801_06364_b300 as m
    return m


def make_pair(wl, precision, pml=True):
    W = wl.pml_width if pml else 0
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1, precision)
    return p, g


SHAPES = [
    ((8, 8, 8), 3, 2),          # (nz, ny, nx), N, layer width
    ((12, 20, 24), 2, 3),       # ragged x tiles (24 = 16 + 8), radix 3 and 5 axes
    ((18, 10, 40), 4, 2),       # 40 = 8 * 5, 18 = 2 * 3 * 3
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,N,W", SHAPES)
def test_state_roundtrip(shape, N, W, precision):
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    _, g = make_pair(wl, precision)
    psi = synth.random_state(N, shape, seed=3)
    g.set_state(psi)
    back = g.get_state()
    assert rel(back, psi) < (1e-14 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,N,W", SHAPES + [((16, 16, 16), 7, 3), ((8, 8, 8), 0, 2)])
def test_apply_transport_matches_oracle(shape, N, W, precision):
    import torch
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    p, g = make_pair(wl, precision)
    psi = synth.smooth_random_state(N, shape, wl.dx, seed=5, corr=0.6)
    want = oracle.apply_T(p, psi)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    x = torch.from_numpy(psi.astype(g.cdtype)).to("cuda")
    got = g.apply_transport(x).cpu().numpy()
    assert rel(got, want) < TOL[precision]


def _run_both(wl, precision, dt, nsteps, psi0=None, integral=False):
    p, g = make_pair(wl, precision)
    if psi0 is None:
        psi0 = np.zeros((wl.M,) + wl.shape, complex)
    src = oracle.Sources(wl.src_voxel, np.zeros(len(wl.src_voxel), np.int32), wl.src_amp, wl.src_t0,
                         wl.src_fwhm)
    want, det_w, int_w = oracle.run(p, psi0, dt, nsteps, sources=src, det_voxels=wl.det_voxel)
    g.set_state(psi0)
    if len(wl.src_voxel):
        g.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, wl.src_t0, wl.src_fwhm)
    if len(wl.det_voxel):
        g.set_detectors(wl.det_voxel)
    det_g, int_g = g.step(dt, nsteps, integral=True)
    return want, det_w, int_w, g.get_state(), det_g, int_g, g


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,N,W", SHAPES)
def test_steps_with_layer_source_detectors_match_oracle(shape, N, W, precision):
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W, nsteps=40)
    wl.src_t0 = np.array([0.6])
    wl.src_fwhm = np.array([0.8])
    p = oracle.Problem(N, shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    dt = 0.5 * oracle.stability_limit(p)
    want, det_w, int_w, got, det_g, int_g, g = _run_both(wl, precision, dt, 40)
    assert g.stability_limit() == pytest.approx(oracle.stability_limit(p), rel=1e-9)
    assert rel(got, want) < TOL[precision]
    assert rel(det_g, det_w) < TOL[precision]
    assert rel(int_g, int_w) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_c1_gaussian_pulse_full_config(precision):
    """32^3 periodic, dx 0.5, P_3, homogeneous (0.01, 1, 0.5), Gaussian pulse
    (sigma 1 mm), 200 steps at 0.5 dt*: all moments and the fluence integral."""
    wl = synth.c1()
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g)
    dt = 0.5 * oracle.stability_limit(p)
    psi0 = synth.gaussian_pulse_state(wl.N, wl.shape, wl.dx, 1.0)
    want, _, int_w = oracle.run(p, psi0, dt, 200)
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, precision=precision)
    g.set_state(psi0)
    _, int_g = g.step(dt, 200, integral=True)
    got = g.get_state()
    assert rel(got, want) < TOL[precision]
    assert rel(int_g, int_w) < TOL[precision]
    # fluence integral decays exactly by (1 - c dt mu_a) per step (periodic, no source)
    r = int_g[1:].real / int_g[:-1].real
    assert np.max(np.abs(r - (1 - wl.c * dt * 0.01))) < (1e-13 if precision == "fp64" else 2e-6)


def test_unstable_dt_rejected_and_plan_stays_usable():
    m = rte()
    wl = synth.c1()
    g = m.Plan((8, 8, 8), 0.5, 3, wl.c, 0.01, 1.0, 0.5, precision="fp32")
    dts = g.stability_limit()
    with pytest.raises(m.RTEError) as e:
        g.step(1.5 * dts, 1)
    assert e.value.status == m.RTE_ERR_UNSTABLE_DT
    g.step(0.5 * dts, 2)            # still usable
    g.step(1.5 * dts, 1, allow_unstable=True)


def test_sources_rejected_in_layer_and_out_of_range():
    m = rte()
    g = m.Plan((12, 12, 12), 0.4, 2, 0.214, 0.01, 10.0, 0.9, 3, 2.0, 10.0, "fp32")
    with pytest.raises(m.RTEError):
        g.set_sources([0], [0], [1.0], [0.0], [1.0])          # corner voxel is in the layer
    with pytest.raises(m.RTEError):
        g.set_sources([12 ** 3], [0], [1.0], [0.0], [1.0])
    with pytest.raises(m.RTEError):
        g.set_sources([6 * 144 + 6 * 12 + 6], [9], [1.0], [0.0], [1.0])   # moment 9 > M-1 = 8
    g.set_sources([6 * 144 + 6 * 12 + 6] * 2, [0, 3], [1.0, 2.0], [0.0, 0.0], [0.0, 0.0])


def test_repeated_and_higher_moment_sources_match_oracle():
    shape, N = (8, 12, 16), 2
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=2)
    p, g = make_pair(wl, "fp64")
    v = int(synth.flat_index(shape, 4, 6, 8))
    vox = np.array([v, v, v + 1])
    mom = np.array([0, 0, 5])
    amp = np.array([1.0, 0.5, 2.0])
    t0 = np.array([0.2, 0.4, 0.0])
    fw = np.array([0.5, 0.0, 0.3])
    src = oracle.Sources(vox, mom, amp, t0, fw)
    dt = 0.5 * oracle.stability_limit(p)
    want, _, _ = oracle.run(p, np.zeros((p.M,) + shape), dt, 15, sources=src)
    g.set_sources(vox, mom, amp, t0, fw)
    g.step(dt, 15, readouts=False)
    assert rel(g.get_state(), want) < 1e-12


def test_step_continues_across_calls_and_time():
    shape, N = (8, 8, 8), 3
    wl = synth.c2(shape=shape, dx=0.5, N=N, W=2)
    wl.src_t0 = np.array([0.3])
    wl.src_fwhm = np.array([0.4])
    p, g = make_pair(wl, "fp64")
    dt = 0.5 * oracle.stability_limit(p)
    src = oracle.Sources(wl.src_voxel, np.zeros(1, np.int32), wl.src_amp, wl.src_t0, wl.src_fwhm)
    want, det_w, _ = oracle.run(p, np.zeros((p.M,) + shape), dt, 20, sources=src, det_voxels=wl.det_voxel)
    g.set_sources(wl.src_voxel, [0], wl.src_amp, wl.src_t0, wl.src_fwhm)
    g.set_detectors(wl.det_voxel)
    d1, _ = g.step(dt, 7)
    d2, _ = g.step(dt, 13)
    assert g.get_time() == pytest.approx(20 * dt)
    assert rel(np.concatenate([d1, d2]), det_w) < 1e-12
    assert rel(g.get_state(), want) < 1e-12


def test_n0_is_pure_local_decay():
    """P_0 has no streaming term: each voxel decays by (1 - c dt mu_a)."""
    shape = (8, 8, 8)
    wl = synth.c2(shape=shape, dx=0.5, N=0, W=2)
    p, g = make_pair(wl, "fp64")
    psi = synth.random_state(0, shape, seed=9)
    g.set_state(psi)
    dt = 0.01
    g.step(dt, 3, allow_unstable=True)
    mua = p.effective_media[0]
    want = psi * (1 - wl.c * dt * mua) ** 3
    assert rel(g.get_state(), want) < 1e-13


# Shapes that take the fixed-size kernels (fused plane for nx, ny in {32, 64,
# 128}; fixed z pass for nz in {32, 64, 128}) next to runtime-size axes.
FIXED_SHAPES = [
    ((24, 32, 64), 3, 3),       # plane 64 x 32, runtime z (24)
    ((64, 32, 32), 2, 4),       # plane 32 x 32, fixed z 64
    ((32, 128, 32), 1, 2),      # plane 32 x 128, fixed z 32
    ((12, 96, 96), 2, 3),       # plane 96 x 96 (12 x 8 transforms), runtime z
    ((10, 160, 160), 1, 3),     # plane 160 x 160 (20 x 8; FP64 takes the split path), runtime z
    ((96, 32, 32), 1, 2),       # fixed z 96
    ((160, 32, 32), 1, 2),      # fixed z 160
    ((256, 8, 16), 1, 2),       # fixed z 256 (16 x 16), runtime planes
    ((6, 256, 256), 1, 2),      # 256 x 256 planes: fixed-size Y and X line passes (no plane kernel)
    ((10, 32, 96), 2, 3),       # 96 x 32 planes: fixed line passes (the plane kernel takes 96 only square)
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,N,W", FIXED_SHAPES)
def test_fixed_size_kernels_match_oracle(shape, N, W, precision):
    import torch
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W, nsteps=25)
    wl.src_t0 = np.array([0.5])
    wl.src_fwhm = np.array([0.8])
    p, g = make_pair(wl, precision)
    psi = synth.smooth_random_state(N, shape, wl.dx, seed=21, corr=0.6)
    want = oracle.apply_T(p, psi)
    got = g.apply_transport(torch.from_numpy(psi.astype(g.cdtype)).to("cuda")).cpu().numpy()
    assert rel(got, want) < TOL[precision]
    dt = 0.5 * oracle.stability_limit(p)
    want, det_w, int_w, got, det_g, int_g, _ = _run_both(wl, precision, dt, 25, psi0=psi)
    assert rel(got, want) < TOL[precision]
    assert rel(det_g, det_w) < TOL[precision]
    assert rel(int_g, int_w) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_benchmark_workload_one_step(precision):
    """The benchmark workload at full size (128^3, P_7, layer 12, 8 spheres,
    pulsed source, 16 detectors) and in the launch configuration bench.py
    times: one explicit step from a smooth random state against one oracle
    step, all moments compared."""
    wl = synth.c2()
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1)
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                   precision)
    dt = 0.5 * g.stability_limit()
    psi0 = synth.smooth_random_state(wl.N, wl.shape, wl.dx, seed=5, corr=1.0).astype(g.cdtype)
    src = oracle.Sources(wl.src_voxel, np.zeros(1, np.int32), wl.src_amp, np.array([0.0]), np.array([10.0]))
    want, det_w, _ = oracle.run(p, psi0.astype(complex), dt, 2, sources=src, det_voxels=wl.det_voxel)
    g.set_state(psi0)
    g.set_sources(wl.src_voxel, [0], wl.src_amp, [0.0], [10.0])
    g.set_detectors(wl.det_voxel)
    det_g, _ = g.step(dt, 2)
    got = g.get_state()
    assert rel(got, want) < TOL[precision]
    assert rel(det_g, det_w) < TOL[precision]
    g.close()


def test_full_size_uniform_field_decays_per_l():
    """Property at full size: a spatially uniform state in a homogeneous
    periodic 128^3 P_7 medium is multiplied per step by 1 - c dt D_l exactly
    (k = 0 only), in the fixed-size kernels' FP32 arithmetic."""
    m = rte()
    shape, N = (128, 128, 128), 7
    g = m.Plan(shape, 0.25, N, synth.C_LIGHT, 0.01, 10.0, 0.9, precision="fp32")
    rng = np.random.default_rng(0)
    amp = (rng.normal(size=(N + 1) ** 2) + 1j * rng.normal(size=(N + 1) ** 2)).astype(np.complex64)
    g.set_state(np.broadcast_to(amp[:, None, None, None], ((N + 1) ** 2,) + shape).copy())
    dt = 0.5 * g.stability_limit()
    g.step(dt, 3)
    out = g.get_state()
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    want = amp * (1 - synth.C_LIGHT * dt * (0.01 + 10.0 * (1 - 0.9 ** ls))) ** 3
    assert np.max(np.abs(out[:, 7, 60, 99] - want) / np.abs(want)) < 1e-5
    assert np.max(np.abs(out - out[:, :1, :1, :1])) < 1e-5 * np.max(np.abs(amp))


# ---------------------------------------------------------------- real radiance
# Plans with real_radiance=1 store the m >= 0 moments only; the oracle runs
# the full (N+1)^2 moments with the mirrored sources made explicit.

def _real_pair_sources(wl, N):
    """moment 0 at the source voxel plus the real-radiance pair (1, +-1)."""
    v = int(wl.src_voxel[0])
    full = oracle.Sources(np.array([v, v + 1, v + 1]), np.array([0, 3, 1]), np.array([1.0, 0.4, -0.4]),
                          np.array([0.5, 0.3, 0.3]), np.array([0.8, 0.6, 0.6]))
    half = ([v, v + 1], [0, 3], [1.0, 0.4], [0.5, 0.3], [0.8, 0.6])
    return full, half


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,N,W", [((24, 32, 64), 3, 3), ((12, 20, 24), 2, 3), ((32, 32, 32), 4, 2)])
def test_real_radiance_layout_matches_oracle(shape, N, W, precision):
    import torch
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    p = oracle.Problem(N, shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    g = rte().Plan(shape, wl.dx, N, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1, precision,
                   real_radiance=True)
    psi = synth.real_radiance_state(N, shape, wl.dx, seed=31, corr=0.6)
    want = oracle.apply_T(p, psi)
    got = g.apply_transport(torch.from_numpy(psi.astype(g.cdtype)).to("cuda")).cpu().numpy()
    assert rel(got, want) < TOL[precision]
    full, half = _real_pair_sources(wl, N)
    dt = 0.5 * oracle.stability_limit(p)
    want, det_w, int_w = oracle.run(p, psi, dt, 30, sources=full, det_voxels=wl.det_voxel)
    g.set_state(psi)
    g.set_sources(*half)
    g.set_detectors(wl.det_voxel)
    det_g, int_g = g.step(dt, 30, integral=True)
    assert rel(g.get_state(), want) < TOL[precision]
    assert rel(det_g, det_w) < TOL[precision]
    assert rel(int_g, int_w) < TOL[precision]
    import torch as _t
    out = _t.empty(g.field_shape, dtype=_t.complex128 if precision == "fp64" else _t.complex64, device="cuda")
    assert rel(g.get_state(out).cpu().numpy(), want) < TOL[precision]


def test_real_radiance_rejects_negative_m_sources():
    m = rte()
    g = m.Plan((8, 8, 8), 0.5, 2, 0.214, 0.01, 1.0, 0.5, precision="fp32", real_radiance=True)
    with pytest.raises(m.RTEError):
        g.set_sources([100], [1], [1.0], [0.0], [1.0])      # moment 1 = (l=1, m=-1)
    g.set_sources([100], [3], [1.0], [0.0], [1.0])          # (1, +1) is accepted


def test_full_size_benchmark_workload_real_radiance_fp32():
    """The benchmark workload in the real-radiance layout: two steps from a
    smooth random real radiance against the full-moment oracle."""
    wl = synth.c2()
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1)
    g = rte().Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                   "fp32", real_radiance=True)
    dt = 0.5 * g.stability_limit()
    psi0 = synth.real_radiance_state(wl.N, wl.shape, wl.dx, seed=6, corr=1.0)
    src = oracle.Sources(wl.src_voxel, np.zeros(1, np.int32), wl.src_amp, np.array([0.0]), np.array([10.0]))
    want, det_w, _ = oracle.run(p, psi0, dt, 2, sources=src, det_voxels=wl.det_voxel)
    g.set_state(psi0)
    g.set_sources(wl.src_voxel, [0], wl.src_amp, [0.0], [10.0])
    g.set_detectors(wl.det_voxel)
    det_g, _ = g.step(dt, 2)
    assert rel(g.get_state(), want) < TOL["fp32"]
    assert rel(det_g, det_w) < TOL["fp32"]
    g.close()


@pytest.mark.parametrize("precision,real", [("fp64", False), ("fp32", True)])
def test_high_order_p21_matches_oracle(precision, real):
    """P_21 (484 moments, the order of the paper's transient run, Sec. IV A)
    on 32 x 32 planes: T psi and 6 explicit steps against the oracle."""
    import torch
    shape, N, W = (6, 32, 32), 21, 2
    wl = synth.c2(shape=shape, dx=0.5, N=N, W=W)
    p = oracle.Problem(N, shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    g = rte().Plan(shape, wl.dx, N, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1, precision,
                   real_radiance=real)
    psi = synth.real_radiance_state(N, shape, wl.dx, seed=41, corr=0.8)
    want = oracle.apply_T(p, psi)
    got = g.apply_transport(torch.from_numpy(psi.astype(g.cdtype)).to("cuda")).cpu().numpy()
    assert rel(got, want) < TOL[precision]
    # the oracle's limit for this case is 0.1378 ps (dense 484 x 484
    # eigenproblems, minutes on the CPU, so not recomputed here)
    dt = 0.06
    want, _, _ = oracle.run(p, psi, dt, 6)
    g.set_state(psi)
    g.step(dt, 6, readouts=False)
    assert rel(g.get_state(), want) < TOL[precision]
