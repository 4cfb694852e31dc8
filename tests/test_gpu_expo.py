"""Exponential step for a homogeneous medium (the arbitrary-step scheme the
paper names for homogeneous media) against the oracle's per-wavevector expm."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rte():
    import paper_1801_06364_b300 as m
    return m


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


MEDIUM = dict(mua=0.02, mus=1.5, g=0.7)


def plan_pair(shape, N, dx, precision, real=False):
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, MEDIUM["mua"], MEDIUM["mus"], MEDIUM["g"])
    g = rte().Plan(shape, dx, N, synth.C_LIGHT, MEDIUM["mua"], MEDIUM["mus"], MEDIUM["g"], precision=precision,
                   real_radiance=real)
    return p, g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("shape,N", [((32, 8, 12), 3), ((64, 6, 4), 2)])
def test_exponential_step_matches_oracle(shape, N, precision, tol):
    dx = 0.5
    p, g = plan_pair(shape, N, dx, precision)
    psi0 = synth.smooth_random_state(N, shape, dx, seed=13, corr=0.8)
    dt = 5.0 * g.stability_limit()          # beyond the explicit limit
    want = oracle.exp_step(p, psi0, dt, 3)
    g.set_state(psi0)
    g.step_exponential(dt, 3)
    assert rel(g.get_state(), want) < tol
    assert g.get_time() == pytest.approx(3 * dt)


def test_exponential_steps_compose_and_mix_with_explicit_steps():
    shape, N, dx = (32, 8, 8), 2, 0.5
    _, g = plan_pair(shape, N, dx, "fp64")
    psi0 = synth.smooth_random_state(N, shape, dx, seed=4, corr=0.8)
    g.set_state(psi0)
    g.step_exponential(0.6, 2)
    two = g.get_state()
    g.set_state(psi0)
    g.step_exponential(1.2, 1)              # a new dt rebuilds E_k
    assert rel(g.get_state(), two) < 1e-12
    # an explicit step from the result (the state is back in the mixed layout)
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, MEDIUM["mua"], MEDIUM["mus"], MEDIUM["g"])
    dte = 0.5 * g.stability_limit()
    want, _, _ = oracle.run(p, two, dte, 3)
    g.step(dte, 3)
    assert rel(g.get_state(), want) < 1e-12


def test_exponential_step_rejects_unsupported_problems():
    m = rte()
    shape, N, dx = (32, 8, 8), 1, 0.5
    psi0 = synth.real_radiance_state(N, shape, dx, seed=2, corr=0.8)   # also valid for the real layout
    cases = []
    mua = np.full(shape, 0.02)
    mua[0, 0, 0] = 0.03
    cases.append(m.Plan(shape, dx, N, synth.C_LIGHT, mua, 1.5, 0.7, precision="fp64"))               # heterogeneous
    cases.append(m.Plan(shape, dx, N, synth.C_LIGHT, 0.02, 1.5, 0.7, 2, 1.0, 2.0, "fp64"))            # layer
    cases.append(m.Plan((20, 8, 8), dx, N, synth.C_LIGHT, 0.02, 1.5, 0.7, precision="fp64"))          # nz
    cases.append(m.Plan(shape, dx, N, synth.C_LIGHT, 0.02, 1.5, 0.7, precision="fp32", real_radiance=True))
    src = m.Plan(shape, dx, N, synth.C_LIGHT, 0.02, 1.5, 0.7, precision="fp64")
    src.set_sources([100], [0], [1.0], [0.0], [0.0])
    cases.append(src)
    for g in cases:
        f = np.zeros(g.field_shape) if g.shape != shape else psi0
        g.set_state(f)
        with pytest.raises(m.RTEError) as e:
            g.step_exponential(0.5, 1)
        assert e.value.status == m.RTE_ERR_UNSUPPORTED
        # unchanged up to the round trip through the xy transforms
        assert np.allclose(g.get_state(), f, rtol=0, atol=(1e-12 if g.fp64 else 1e-6) * max(1.0, np.abs(f).max()))
