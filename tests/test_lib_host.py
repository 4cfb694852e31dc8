"""Host-side checks of librte that need no GPU: the library loads, exports
every symbol include/rte.h declares, validates arguments, and its host-only
stability limit (its own complex QR eigenvalue solver on the z-blocks of
S(k)) agrees with the oracle's dense eigvals along another direction."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_1801_06364_b300 as rte
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rte.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rte_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = rte.lib()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    bound = {s[0] for s in rte.SIGNATURES}
    assert set(names) == bound
    assert "sm_103a" in rte.version()


def test_status_strings():
    L = rte.lib()
    assert L.rte_status_string(0) == b"ok"
    assert b"stability" in L.rte_status_string(3)


@pytest.mark.parametrize("shape,N", [((8, 8, 8), 3), ((12, 10, 16), 2), ((20, 24, 18), 5)])
def test_stability_limit_matches_oracle(shape, N):
    wl = synth.c2(shape=shape, dx=0.25, N=N, W=2)
    desc = rte.make_desc(shape, 0.25, N, synth.C_LIGHT, 2, 2.0, 10.0)
    got = rte.stability_limit_media(desc, wl.mua, wl.mus, wl.g)
    p = oracle.Problem(N, shape, 0.25, synth.C_LIGHT, wl.mua, wl.mus, wl.g, 2, 2.0, 10.0)
    want = oracle.stability_limit(p)
    assert got == pytest.approx(want, rel=1e-9)


def test_stability_limit_periodic_and_published_values():
    # C1 (32^3, dx 0.5, P_3, homogeneous (0.01, 1, 0.5)): the oracle's value
    desc = rte.make_desc((32, 32, 32), 0.5, 3, synth.C_LIGHT)
    got = rte.stability_limit_media(desc, 0.01, 1.0, 0.5)
    want = oracle.stability_limit(oracle.Problem(3, (32, 32, 32), 0.5, synth.C_LIGHT, 0.01, 1.0, 0.5))
    assert got == pytest.approx(want, rel=1e-10)
    # uniform damping closed form 2 d / (c (d^2 + kmax^2 xmax^2))
    from scipy.special import roots_legendre
    d = 1.7
    desc = rte.make_desc((16, 16, 16), 0.25, 7, synth.C_LIGHT)
    got = rte.stability_limit_media(desc, d, 0.0, 0.9)
    kmax = np.sqrt(3) * 2 * np.pi * 7 / (16 * 0.25)
    xmax = np.max(roots_legendre(8)[0])
    assert got == pytest.approx(2 * d / (synth.C_LIGHT * (d * d + kmax * kmax * xmax * xmax)), rel=1e-10)


def test_invalid_descriptors_rejected_without_gpu():
    bad = [
        rte.make_desc((7, 8, 8), 0.5, 3, 0.2),       # 7 is not a 2/3/5 product
        rte.make_desc((8, 8, 8), 0.5, 22, 0.2),      # N too large
        rte.make_desc((8, 8, 8), -1.0, 3, 0.2),      # dx
        rte.make_desc((8, 8, 8), 0.5, 3, 0.2, pml_cells=4, pml_mu0=1, pml_mu1=2),  # layer too thick
    ]
    for d in bad:
        with pytest.raises(rte.RTEError) as e:
            rte.plan_footprint(d)
        assert e.value.status == rte.RTE_ERR_INVALID_ARG
    h = C.c_void_p()
    a = np.zeros(512)
    st = rte.lib().rte_plan_create(C.byref(bad[0]), rte._dp(a), rte._dp(a), rte._dp(a), None, C.byref(h))
    assert st == rte.RTE_ERR_INVALID_ARG and not h.value


def test_footprint_counts_four_state_buffers():
    d = rte.make_desc((128, 128, 128), 0.25, 7, 0.214, 12, 2.0, 10.0, "fp32")
    b = rte.plan_footprint(d)
    state = 64 * 128 ** 3 * 8
    # four state-sized buffers, the media and (fixed-size xy axes) D_l per l in slot order
    extra = 128 ** 3 * 16 + 8 * 128 ** 3 * 4
    assert 4 * state + extra <= b < 4 * state + extra + 10 ** 6
    # 96 x 96 FP32 planes take the plane kernel too (75 KB of shared memory), so D_l is kept per l
    d = rte.make_desc((96, 96, 96), 0.25, 3, 0.214, 12, 2.0, 10.0, "fp32")
    state = 16 * 96 ** 3 * 8
    extra = 96 ** 3 * 16 + 4 * 96 ** 3 * 4
    assert 4 * state + extra <= rte.plan_footprint(d) < 4 * state + extra + 10 ** 6
    # 80-point axes and FP64 planes over 64 points per axis (the plane kernel's
    # register DFTs stop at 16 FP64 points) have no D_l copy
    for shape in ((80, 80, 80), (160, 160, 16), (96, 96, 96)):
        d = rte.make_desc(shape, 0.25, 3, 0.214, 4, 2.0, 10.0, "fp64")
        V = int(np.prod(shape))
        state = 16 * V * 16
        assert 4 * state + V * 32 <= rte.plan_footprint(d) < 4 * state + V * 32 + 10 ** 6


def test_product_has_no_oracle_import():
    """The CUDA path's package never imports the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_1801_06364_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "rte_oracle" not in text, f


def test_set_allocator_takes_both_callbacks_or_neither():
    L = rte.lib()
    fn = rte._ALLOC_FN(lambda n, s, c: None)
    st = L.rte_set_allocator(C.cast(fn, C.c_void_p), None, None)
    assert st == rte.RTE_ERR_INVALID_ARG
    assert L.rte_set_allocator(None, None, None) == rte.RTE_OK


def test_torch_allocator_binding_registers_and_keeps_its_callbacks():
    """use_torch_allocator registers a callback pair with the library and keeps
    every pair it registered alive (plans created under one keep calling it
    until they close); enable=False goes back to cudaMallocAsync. No plan is
    created, so no GPU is needed."""
    n0 = len(rte._ALLOCATORS)
    try:
        rte.use_torch_allocator(True)
        rte.use_torch_allocator(True)
        assert len(rte._ALLOCATORS) == n0 + 2
        alloc, free = rte._ALLOCATORS[-1]
        assert isinstance(alloc, rte._ALLOC_FN) and isinstance(free, rte._FREE_FN)
    finally:
        rte.use_torch_allocator(False)
    assert len(rte._ALLOCATORS) == n0 + 2          # still alive after the switch back
