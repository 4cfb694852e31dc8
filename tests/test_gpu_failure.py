"""Failure detection on the GPU without a GPU fault: a NaN or an infinity put
into the state from the host (rte_set_state) must come back as
RTE_ERR_NONFINITE, and the plan must stay usable afterwards."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rte():
    import paper_1801_06364_b300 as m
    return m


# (shape, precision, real layout): the fused plane path, and the split path
# (nz = 40 has no fixed-size z transform, so the step takes the line passes)
CASES = [((32, 32, 32), "fp32", True), ((40, 32, 32), "fp64", False)]


@pytest.mark.parametrize("shape,precision,real", CASES)
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_state_is_reported_and_the_plan_stays_usable(shape, precision, real, bad):
    R = rte()
    N, W = 3, 3
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    p = oracle.Problem(N, shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1)
    dt = 0.5 * oracle.stability_limit(p)
    psi0 = synth.real_radiance_state(N, shape, wl.dx, seed=4, corr=0.8)
    g = R.Plan(shape, wl.dx, N, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1, precision,
               real_radiance=real)
    g.set_detectors(wl.det_voxel)
    poisoned = psi0.copy()
    poisoned[7, shape[0] // 2, 7, 9] = bad          # one moment (l = 2, m = 1) at one voxel
    g.set_state(poisoned)
    with pytest.raises(R.RTEError) as err:
        g.step(dt, 2)                                # readouts requested: the call synchronises
    assert err.value.status == R.RTE_ERR_NONFINITE
    # reported once: a further call on a finite state succeeds
    g.set_state(psi0)
    det, _ = g.step(dt, 6)
    want, det_w, _ = oracle.run(p, psi0, dt, 6, det_voxels=wl.det_voxel)
    got = g.get_state()
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert np.all(np.isfinite(det))
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
    assert np.linalg.norm(det - det_w) / np.linalg.norm(det_w) < tol
    g.close()


def test_nonfinite_flag_reaches_a_later_synchronising_call():
    """A run without outputs does not synchronise; the flag it raised is
    reported by the next call that does (here rte_get_state), which still
    returns the state."""
    R = rte()
    shape, N, W = (32, 32, 32), 3, 3
    wl = synth.c2(shape=shape, dx=0.4, N=N, W=W)
    g = R.Plan(shape, wl.dx, N, wl.c, wl.mua, wl.mus, wl.g, W, wl.pml_mu0, wl.pml_mu1, "fp32",
               real_radiance=True)
    dt = 0.5 * g.stability_limit()
    psi = synth.real_radiance_state(N, shape, wl.dx, seed=5, corr=0.8)
    psi[0, 3, 4, 5] = np.nan
    g.set_state(psi)
    g.step(dt, 4, readouts=False)
    with pytest.raises(R.RTEError) as err:
        g.get_state()
    assert err.value.status == R.RTE_ERR_NONFINITE
    out = np.empty(g.field_shape, np.complex64)
    assert R.lib().rte_get_state(g.handle, out.ctypes.data_as(R.C.c_void_p), R.RTE_HOST) == R.RTE_OK
    g.close()
