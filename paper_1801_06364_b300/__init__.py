"""Python binding of librte: the pseudospectral P_N radiative-transport
method of Powell, Cox & Arridge (arXiv:1801.06364) on one B300 GPU.

This module only marshals arguments into the C ABI declared in
``include/rte.h``; every step of the method runs in the CUDA kernels of
``librte.so``. There is no CPU fallback: importing works without a GPU (the
host-only entry points such as the stability limit stay usable), but every
device call fails loudly when CUDA is unavailable.

Fields are complex arrays of shape (M, nz, ny, nx), M = (N+1)^2, moment index
l*l + l + m; complex64 for FP32 plans, complex128 for FP64 plans.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

RTE_OK = 0
RTE_ERR_INVALID_ARG = 1
RTE_ERR_OOM = 2
RTE_ERR_UNSTABLE_DT = 3
RTE_ERR_NONFINITE = 4
RTE_ERR_NOT_CONVERGED = 5
RTE_ERR_TIMEOUT = 6
RTE_ERR_CUDA = 7
RTE_ERR_UNSUPPORTED = 8
RTE_ERR_STATE = 9
RTE_FP32 = 0
RTE_FP64 = 1
RTE_HOST = 0
RTE_DEVICE = 1
RTE_PREC_NONE = 0
RTE_PREC_LOW_ORDER = 1
RTE_SCHED_AUTO = 0
RTE_SCHED_PLANE = 1
RTE_SCHED_SPLIT = 2

LIB_PATH = _build.LIB


class RTEError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx_mm", C.c_double),
                ("N", C.c_int), ("c_mm_per_ps", C.c_double), ("pml_cells", C.c_int),
                ("pml_mu0", C.c_double), ("pml_mu1", C.c_double), ("precision", C.c_int),
                ("real_radiance", C.c_int)]


# (name, restype, argtypes) of every symbol include/rte.h declares
_VP, _D, _I, _DP, _IP = C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)
_I64P = C.POINTER(C.c_int64)
SIGNATURES = [
    ("rte_status_string", C.c_char_p, [_I]),
    ("rte_last_error_string", C.c_char_p, []),
    ("rte_version", C.c_char_p, []),
    ("rte_plan_create", _I, [C.POINTER(GridDesc), _DP, _DP, _DP, _VP, C.POINTER(_VP)]),
    ("rte_plan_destroy", _I, [_VP]),
    ("rte_set_allocator", _I, [_VP, _VP, _VP]),
    ("rte_plan_footprint", _I, [C.POINTER(GridDesc), C.POINTER(C.c_uint64)]),
    ("rte_stability_limit_media", _I, [C.POINTER(GridDesc), _DP, _DP, _DP, _DP]),
    ("rte_stability_limit", _I, [_VP, _DP]),
    ("rte_set_state", _I, [_VP, _VP, _I]),
    ("rte_get_state", _I, [_VP, _VP, _I]),
    ("rte_set_time", _I, [_VP, _D]),
    ("rte_get_time", _I, [_VP, _DP]),
    ("rte_set_sources", _I, [_VP, _I, _I64P, _IP, _DP, _DP, _DP]),
    ("rte_set_detectors", _I, [_VP, _I, _I64P]),
    ("rte_step", _I, [_VP, _D, _I, _I, _DP, _DP]),
    ("rte_apply_transport", _I, [_VP, _VP, _VP]),
    ("rte_solve_steady", _I, [_VP, _D, _I, _I, _IP, _DP]),
    ("rte_set_preconditioner", _I, [_VP, _I]),
    ("rte_set_schedule", _I, [_VP, _I, _I]),
    ("rte_step_group", _I, [C.POINTER(_VP), _I, _DP, _I, C.POINTER(_DP)]),
    ("rte_step_exponential", _I, [_VP, _D, _I]),
    ("rte_forward", _I, [_VP, _D, _I, _I, _DP, _DP, _DP]),
    ("rte_adjoint", _I, [_VP, _DP, _VP, _VP]),
    ("rte_profile_enable", _I, [_VP, _I]),
    ("rte_profile_read", _I, [_VP, _I, C.c_char_p, _IP, _DP, _IP]),
    ("rte_apply_transport_noalloc", _I, [C.POINTER(GridDesc), _DP, _DP, _DP, _VP, _VP, _VP]),
    ("rte_fma_peak", _I, [_I, _DP]),
    ("rte_kernel_launch_count", C.c_uint64, []),
]

_LIB = None
_LIB_LOCK = threading.Lock()


def lib():
    """Load librte.so (building it first if it is missing); safe to call from
    several threads at once (the serving loop drives plans from many)."""
    global _LIB
    if _LIB is None:
        with _LIB_LOCK:
            if _LIB is None:
                if not os.path.exists(LIB_PATH) or os.environ.get("RTE_REBUILD"):
                    _build.build()
                L = C.CDLL(LIB_PATH)
                for name, res, args in SIGNATURES:
                    f = getattr(L, name)
                    f.restype = res
                    f.argtypes = args
                _LIB = L
    return _LIB


def _check(status, where):
    if status != RTE_OK:
        L = lib()
        raise RTEError(status, where, L.rte_last_error_string().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def version() -> str:
    return lib().rte_version().decode()


def kernel_launches() -> int:
    return int(lib().rte_kernel_launch_count())


def fma_peak(precision="fp64") -> float:
    """FMA throughput (FLOP/s) of the current device in FP32 or FP64, from the
    library's own kernel (see rte.h)."""
    out = C.c_double(0.0)
    prec = RTE_FP64 if precision in ("fp64", RTE_FP64) else RTE_FP32
    _check(lib().rte_fma_peak(prec, C.byref(out)), "rte_fma_peak")
    return out.value


def make_desc(shape, dx, N, c, pml_cells=0, pml_mu0=0.0, pml_mu1=0.0, precision="fp32",
              real_radiance=False) -> GridDesc:
    nz, ny, nx = (int(s) for s in shape)
    prec = RTE_FP64 if precision in ("fp64", RTE_FP64, "f64", np.float64) else RTE_FP32
    return GridDesc(nx, ny, nz, float(dx), int(N), float(c), int(pml_cells), float(pml_mu0), float(pml_mu1), prec,
                    int(bool(real_radiance)))


def stability_limit_media(desc: GridDesc, mua, mus, g) -> float:
    """Host-only dt* of the explicit step for the given maps (see rte.h)."""
    shp = (desc.nz, desc.ny, desc.nx)
    a = np.ascontiguousarray(np.broadcast_to(mua, shp), dtype=np.float64)
    s = np.ascontiguousarray(np.broadcast_to(mus, shp), dtype=np.float64)
    gg = np.ascontiguousarray(np.broadcast_to(g, shp), dtype=np.float64)
    out = C.c_double(0.0)
    _check(lib().rte_stability_limit_media(C.byref(desc), _dp(a), _dp(s), _dp(gg), C.byref(out)),
           "rte_stability_limit_media")
    return out.value


def plan_footprint(desc: GridDesc) -> int:
    out = C.c_uint64(0)
    _check(lib().rte_plan_footprint(C.byref(desc), C.byref(out)), "rte_plan_footprint")
    return int(out.value)


def _torch():
    import torch
    return torch


# rte_alloc_fn / rte_free_fn of include/rte.h
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_ALLOCATORS = []    # every callback pair ever registered: plans keep theirs until they close


def use_torch_allocator(enable=True):
    """Plans created from now on take their device memory from PyTorch's caching
    allocator (on the plan's stream) instead of cudaMallocAsync, so that it shows
    in torch.cuda.memory_allocated() and is pooled with the caller's tensors.
    Plans created earlier keep their allocator. enable=False returns to
    cudaMallocAsync. The plan's memory goes back to the pool at Plan.close()."""
    if not enable:
        _check(lib().rte_set_allocator(None, None, None), "rte_set_allocator")
        return
    torch = _torch()

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None      # NULL: the library reports RTE_ERR_OOM

    def free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (_ALLOC_FN(alloc), _FREE_FN(free))
    _ALLOCATORS.append(cbs)
    _check(lib().rte_set_allocator(C.cast(cbs[0], C.c_void_p), C.cast(cbs[1], C.c_void_p), None),
           "rte_set_allocator")


def step_group(plans, dts, nsteps, readouts=True):
    """nsteps explicit steps of same-shape plans in one launch of each step
    pass (rte_step_group); returns each plan's readouts [nsteps, ndet] or None."""
    n = len(plans)
    hs = (_VP * n)(*[p._h.value for p in plans])
    d = np.ascontiguousarray(dts, dtype=np.float64)
    dets = [np.zeros((nsteps, max(p.ndet, 1))) if (readouts and p.ndet) else None for p in plans]
    ptrs = (_DP * n)(*[_dp(x) if x is not None else None for x in dets])
    _check(lib().rte_step_group(hs, n, _dp(d), int(nsteps), ptrs), "rte_step_group")
    return [x[:, :p.ndet] if x is not None else None for x, p in zip(dets, plans)]


class Plan:
    """One problem on the GPU: grid, order, media, layer, state, sources."""

    def __init__(self, shape, dx, N, c, mua, mus, g, pml_cells=0, pml_mu0=0.0, pml_mu1=0.0,
                 precision="fp32", stream=None, real_radiance=False):
        """real_radiance=True stores the m >= 0 moments only (valid for real
        radiance, psi_l^{-m} = (-1)^m conj(psi_l^m)); fields in and out keep
        the full (N+1)^2-moment layout."""
        self.desc = make_desc(shape, dx, N, c, pml_cells, pml_mu0, pml_mu1, precision, real_radiance)
        self.real_radiance = bool(real_radiance)
        self.shape = tuple(int(s) for s in shape)
        self.N = int(N)
        self.M = (self.N + 1) ** 2
        self.V = int(np.prod(self.shape))
        self.fp64 = self.desc.precision == RTE_FP64
        self.cdtype = np.complex128 if self.fp64 else np.complex64
        a = np.ascontiguousarray(np.broadcast_to(mua, self.shape), dtype=np.float64)
        s = np.ascontiguousarray(np.broadcast_to(mus, self.shape), dtype=np.float64)
        gg = np.ascontiguousarray(np.broadcast_to(g, self.shape), dtype=np.float64)
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream is not None else None
        _check(lib().rte_plan_create(C.byref(self.desc), _dp(a), _dp(s), _dp(gg), st, C.byref(h)),
               "rte_plan_create")
        self._h = h
        self.ndet = 0

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rte_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def field_shape(self):
        return (self.M,) + self.shape

    def stability_limit(self) -> float:
        out = C.c_double(0.0)
        _check(lib().rte_stability_limit(self._h, C.byref(out)), "rte_stability_limit")
        return out.value

    # --- state -----------------------------------------------------------
    def set_state(self, psi):
        """psi: numpy array (host) or torch CUDA tensor (device), complex."""
        if isinstance(psi, np.ndarray):
            a = np.ascontiguousarray(psi, dtype=self.cdtype)
            assert a.shape == self.field_shape
            _check(lib().rte_set_state(self._h, a.ctypes.data_as(C.c_void_p), RTE_HOST), "rte_set_state")
        else:
            t = psi.contiguous()
            assert tuple(t.shape) == self.field_shape
            where = RTE_DEVICE if t.is_cuda else RTE_HOST
            _check(lib().rte_set_state(self._h, C.c_void_p(t.data_ptr()), where), "rte_set_state")

    def get_state(self, out=None):
        if out is None:
            a = np.empty(self.field_shape, dtype=self.cdtype)
            _check(lib().rte_get_state(self._h, a.ctypes.data_as(C.c_void_p), RTE_HOST), "rte_get_state")
            return a
        assert out.is_contiguous() and tuple(out.shape) == self.field_shape
        where = RTE_DEVICE if out.is_cuda else RTE_HOST
        _check(lib().rte_get_state(self._h, C.c_void_p(out.data_ptr()), where), "rte_get_state")
        return out

    def set_time(self, t):
        _check(lib().rte_set_time(self._h, float(t)), "rte_set_time")

    def get_time(self):
        out = C.c_double(0.0)
        _check(lib().rte_get_time(self._h, C.byref(out)), "rte_get_time")
        return out.value

    # --- sources / detectors ---------------------------------------------
    def set_sources(self, voxel, moment, amp, t0, fwhm):
        v = np.ascontiguousarray(voxel, dtype=np.int64)
        m = np.ascontiguousarray(moment, dtype=np.int32)
        a = np.ascontiguousarray(amp, dtype=np.float64)
        t = np.ascontiguousarray(t0, dtype=np.float64)
        f = np.ascontiguousarray(fwhm, dtype=np.float64)
        n = v.size
        _check(lib().rte_set_sources(self._h, n, v.ctypes.data_as(_I64P), m.ctypes.data_as(_IP),
                                     _dp(a), _dp(t), _dp(f)), "rte_set_sources")

    def set_detectors(self, voxel):
        v = np.ascontiguousarray(voxel, dtype=np.int64)
        _check(lib().rte_set_detectors(self._h, v.size, v.ctypes.data_as(_I64P)), "rte_set_detectors")
        self.ndet = v.size

    # --- time stepping ----------------------------------------------------
    def step(self, dt, nsteps, allow_unstable=False, readouts=True, integral=False):
        """nsteps explicit steps; returns (det_series[nsteps, ndet] or None,
        integral[nsteps] complex or None) read before each step."""
        det = np.zeros((nsteps, max(self.ndet, 1))) if (readouts and self.ndet) else None
        integ = np.zeros((nsteps, 2)) if integral else None
        _check(lib().rte_step(self._h, float(dt), int(nsteps), int(bool(allow_unstable)),
                              _dp(det) if det is not None else None,
                              _dp(integ) if integ is not None else None), "rte_step")
        return (det[:, :self.ndet] if det is not None else None,
                (integ[:, 0] + 1j * integ[:, 1]) if integ is not None else None)

    def step_exponential(self, dt, nsteps=1):
        """nsteps exponential steps of any dt (uniform medium without a layer
        or sources, full layout): psi^(k) <- expm(-c dt (S(k) + D)) psi^(k)."""
        _check(lib().rte_step_exponential(self._h, float(dt), int(nsteps)), "rte_step_exponential")

    def apply_transport(self, psi_in, psi_out=None):
        """T psi for torch CUDA tensors (complex64 / complex128)."""
        torch = _torch()
        x = psi_in.contiguous()
        if psi_out is None:
            psi_out = torch.empty_like(x)
        _check(lib().rte_apply_transport(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(psi_out.data_ptr())),
               "rte_apply_transport")
        return psi_out

    def set_schedule(self, schedule="auto", graph_steps=2):
        """Step schedule ("auto", "plane" or "split") and steps per replayed
        step graph (even, 2..64, or 0 for none); see rte_set_schedule."""
        k = {"auto": RTE_SCHED_AUTO, "plane": RTE_SCHED_PLANE, "split": RTE_SCHED_SPLIT}[schedule]
        _check(lib().rte_set_schedule(self._h, k, int(graph_steps)), "rte_set_schedule")

    def set_preconditioner(self, kind):
        """GMRES right preconditioner: "low" (l <= 1 mean-medium inverse, the
        default) or "none"."""
        k = {"none": RTE_PREC_NONE, "low": RTE_PREC_LOW_ORDER}[kind]
        _check(lib().rte_set_preconditioner(self._h, k), "rte_set_preconditioner")

    def solve_steady(self, rtol=1e-6, restart=20, max_iter=2000):
        it = C.c_int(0)
        rr = C.c_double(0.0)
        st = lib().rte_solve_steady(self._h, float(rtol), int(restart), int(max_iter), C.byref(it), C.byref(rr))
        if st not in (RTE_OK, RTE_ERR_NOT_CONVERGED):
            _check(st, "rte_solve_steady")
        return it.value, rr.value, st == RTE_OK

    # --- per-kernel timing ---------------------------------------------------
    def profile(self, enable=True):
        _check(lib().rte_profile_enable(self._h, int(bool(enable))), "rte_profile_enable")

    def profile_read(self):
        """{kernel name: (launches, total ms)} from CUDA events on the plan's stream."""
        mx = 64
        names = C.create_string_buffer(64 * mx)
        cnt = (C.c_int * mx)()
        ms = (C.c_double * mx)()
        n = C.c_int(0)
        _check(lib().rte_profile_read(self._h, mx, names, cnt, ms, C.byref(n)), "rte_profile_read")
        out = {}
        for i in range(min(n.value, mx)):
            nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (int(cnt[i]), float(ms[i]))
        return out

    # --- adjoint -----------------------------------------------------------
    def forward(self, dt, nsteps, ckpt_every, gates):
        g = np.asarray(gates, dtype=np.float64).reshape(-1, 2)
        lo = np.ascontiguousarray(g[:, 0])
        hi = np.ascontiguousarray(g[:, 1])
        y = np.zeros(max(self.ndet, 1))
        _check(lib().rte_forward(self._h, float(dt), int(nsteps), int(ckpt_every), _dp(lo), _dp(hi), _dp(y)),
               "rte_forward")
        return y[:self.ndet]

    def adjoint(self, dL_dy):
        """Returns (dL/dmu_a, dL/dmu_s) as float64 torch CUDA tensors of the grid shape."""
        torch = _torch()
        d = np.ascontiguousarray(dL_dy, dtype=np.float64)
        ga = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        gs = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        _check(lib().rte_adjoint(self._h, _dp(d), C.c_void_p(ga.data_ptr()), C.c_void_p(gs.data_ptr())),
               "rte_adjoint")
        return ga, gs
