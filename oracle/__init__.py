"""FP64 CPU oracle for the pseudospectral P_N transport method
(Powell, Cox & Arridge, arXiv:1801.06364).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the CUDA library never does, and the
two share no code. The arithmetic lives in ``rte_oracle.c`` (plain C, FP64,
its own DFT/FFT); this module marshals numpy arrays into it and adds the
stability-limit routine, which uses ``numpy.linalg.eigvals`` as a library step.

Every function cites the part of the paper it follows:
  Eq. 3-6   moment expansion, HG scattering diagonal, alpha/beta recurrence
  Eq. 7-10  Fourier transform and the k-space streaming term
  Eq. 11    explicit time step (signs read so that the scheme decays)
  Eq. 12    perfectly matched layer (mu_s = 0, q = 0, isotropic loss mu_b)
  Sec. II.A steady state via a Krylov method on the implicit operator
  Sec. II.A stability of the explicit step (asserted there, derived here)

Arrays: fields are complex128 of shape (M, nz, ny, nx), M = (N+1)^2, moment
index l*l + l + m; media are float64 of shape (nz, ny, nx).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_alpha.restype = C.c_double
        L.orc_alpha.argtypes = [C.c_int, C.c_int]
        L.orc_beta.restype = C.c_double
        L.orc_beta.argtypes = [C.c_int, C.c_int]
        L.orc_wavenumber.restype = C.c_double
        L.orc_wavenumber.argtypes = [C.c_int, C.c_int, C.c_double]
        L.orc_streaming_matrix.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_void_p]
        L.orc_kspace_streaming.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.orc_dft_naive.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.orc_fft.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.orc_fft3d.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_dft3d_naive.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_pml_profile.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_void_p, C.c_void_p]
        L.orc_apply_streaming.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_apply_T.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_apply_T_adjoint.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_source_density.restype = C.c_double
        L.orc_source_density.argtypes = [C.c_double] * 5
        L.orc_run.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_double,
                              C.c_int, ip, ip, dp, dp, dp, C.c_int, ip, dp, dp]
        L.orc_gmres.restype = C.c_int
        L.orc_gmres.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                ip, dp]
        L.orc_adjoint.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_double,
                                  C.c_int, ip, ip, dp, dp, dp, C.c_int, ip, dp, dp, dp]
        _LIB = L
    return _LIB


class _Medium(C.Structure):
    _fields_ = [("N", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("c", C.c_double),
                ("mua", C.c_void_p), ("mus", C.c_void_p), ("g", C.c_void_p)]


def _ptr(a, ctype=None):
    if a is None:
        return None
    if ctype is None:
        return a.ctypes.data_as(C.c_void_p)
    return a.ctypes.data_as(C.POINTER(ctype))


def num_moments(N: int) -> int:
    return (N + 1) ** 2


def moment_index(l: int, m: int) -> int:
    return l * l + l + m


def alpha(l: int, m: int) -> float:
    """alpha_l^m of Eq. 6."""
    return lib().orc_alpha(l, m)


def beta(l: int, m: int) -> float:
    """beta_l^m of Eq. 6."""
    return lib().orc_beta(l, m)


def wavenumber(i: int, n: int, dx: float) -> float:
    """DFT wavenumber of index i (Nyquist index mapped to 0)."""
    return lib().orc_wavenumber(i, n, dx)


def wavenumbers(n: int, dx: float) -> np.ndarray:
    return np.array([wavenumber(i, n, dx) for i in range(n)])


def streaming_matrix(N: int, k) -> np.ndarray:
    """Dense (M, M) matrix S(k) of the k-space streaming term (Eq. 10, d -> +ik)."""
    M = num_moments(N)
    out = np.zeros((M, M), dtype=np.complex128)
    lib().orc_streaming_matrix(N, float(k[0]), float(k[1]), float(k[2]), _ptr(out))
    return out


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    lib().orc_fft(_ptr(x), _ptr(out), x.size, sign)
    return out


def dft_naive(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    lib().orc_dft_naive(_ptr(x), _ptr(out), x.size, sign)
    return out


def fft3d(f: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT of a (nz, ny, nx) field (Eq. 8 on the grid)."""
    g = np.array(f, dtype=np.complex128, order="C", copy=True)
    nz, ny, nx = g.shape
    lib().orc_fft3d(_ptr(g), nx, ny, nz, sign)
    return g


def dft3d_naive(f: np.ndarray, sign: int = -1) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.complex128)
    nz, ny, nx = f.shape
    out = np.empty_like(f)
    lib().orc_dft3d_naive(_ptr(f), _ptr(out), nx, ny, nz, sign)
    return out


def pml_profile(shape, width: int, mu0: float, mu1: float):
    """Half-cosine PML loss mu_b and the layer mask (Sec. II.B, Eq. 12)."""
    nz, ny, nx = shape
    mub = np.zeros(shape, dtype=np.float64)
    mask = np.zeros(shape, dtype=np.uint8)
    lib().orc_pml_profile(nx, ny, nz, int(width), float(mu0), float(mu1), _ptr(mub), _ptr(mask))
    return mub, mask


@dataclass
class Problem:
    """A P_N problem on a periodic grid, with the PML folded into the media:
    inside the layer mu_a -> mu_b and mu_s -> 0 (Eq. 12)."""
    N: int
    shape: tuple          # (nz, ny, nx)
    dx: float             # mm
    c: float              # mm/ps
    mua: np.ndarray
    mus: np.ndarray
    g: np.ndarray
    pml_width: int = 0
    pml_mu0: float = 0.0
    pml_mu1: float = 0.0
    mask: np.ndarray = field(default=None, repr=False)
    _eff: tuple = field(default=None, repr=False)

    def __post_init__(self):
        shp = tuple(int(s) for s in self.shape)
        self.shape = shp
        mua = np.broadcast_to(np.asarray(self.mua, dtype=np.float64), shp).copy()
        mus = np.broadcast_to(np.asarray(self.mus, dtype=np.float64), shp).copy()
        g = np.broadcast_to(np.asarray(self.g, dtype=np.float64), shp).copy()
        self.mua, self.mus, self.g = mua, mus, g
        mub, mask = pml_profile(shp, self.pml_width, self.pml_mu0, self.pml_mu1)
        self.mask = mask
        inl = mask.astype(bool)
        mua_e = np.where(inl, mub, mua)
        mus_e = np.where(inl, 0.0, mus)
        self._eff = (np.ascontiguousarray(mua_e), np.ascontiguousarray(mus_e), np.ascontiguousarray(g))

    @property
    def M(self):
        return num_moments(self.N)

    @property
    def V(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    @property
    def effective_media(self):
        return self._eff

    def _struct(self):
        nz, ny, nx = self.shape
        a, s, g = self._eff
        return _Medium(self.N, nx, ny, nz, float(self.dx), float(self.c),
                       a.ctypes.data, s.ctypes.data, g.ctypes.data)

    def damping(self):
        """D_l(r) = mu_a + mu_s (1 - g^l) (Eq. 6, 11), shape (N+1, nz, ny, nx)."""
        a, s, g = self._eff
        return np.stack([a + s * (1.0 - g ** l) for l in range(self.N + 1)])


def _field(prob: Problem, psi) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    assert psi.shape == (prob.M,) + prob.shape, psi.shape
    return psi


def apply_streaming(prob: Problem, psi) -> np.ndarray:
    """F^-1[S(k) F psi] (stage 1 of the operator, Sec. III; Eq. 10)."""
    psi = _field(prob, psi)
    out = np.empty_like(psi)
    st = prob._struct()
    lib().orc_apply_streaming(C.byref(st), _ptr(psi), _ptr(out))
    return out


def apply_T(prob: Problem, psi) -> np.ndarray:
    """T psi = F^-1[psidot] + D psi (stages 1-2, Sec. III)."""
    psi = _field(prob, psi)
    out = np.empty_like(psi)
    st = prob._struct()
    lib().orc_apply_T(C.byref(st), _ptr(psi), _ptr(out))
    return out


def apply_T_adjoint(prob: Problem, psi) -> np.ndarray:
    """T^H psi in the plain Euclidean inner product."""
    psi = _field(prob, psi)
    out = np.empty_like(psi)
    st = prob._struct()
    lib().orc_apply_T_adjoint(C.byref(st), _ptr(psi), _ptr(out))
    return out


def source_density(t, amp, t0, fwhm, dx) -> float:
    """Gaussian pulse (or constant for fwhm <= 0) source density per mm^3."""
    return lib().orc_source_density(float(t), float(amp), float(t0), float(fwhm), float(dx))


@dataclass
class Sources:
    voxel: np.ndarray      # flat voxel index z*ny*nx + y*nx + x
    moment: np.ndarray
    amp: np.ndarray
    t0: np.ndarray
    fwhm: np.ndarray

    @staticmethod
    def none():
        z = np.zeros(0)
        return Sources(np.zeros(0, np.int32), np.zeros(0, np.int32), z, z, z)

    def arrays(self):
        return (np.ascontiguousarray(self.voxel, dtype=np.int32),
                np.ascontiguousarray(self.moment, dtype=np.int32),
                np.ascontiguousarray(self.amp, dtype=np.float64),
                np.ascontiguousarray(self.t0, dtype=np.float64),
                np.ascontiguousarray(self.fwhm, dtype=np.float64))


def run(prob: Problem, psi0, dt: float, nsteps: int, t_start: float = 0.0,
        sources: Sources | None = None, det_voxels=None):
    """nsteps explicit steps of Eq. 11. Returns (psi, det_series[nsteps, ndet],
    integral[nsteps] complex): readouts of the state each step starts from."""
    psi = np.array(_field(prob, psi0), copy=True)
    src = (sources or Sources.none()).arrays()
    dv = np.ascontiguousarray(np.zeros(0) if det_voxels is None else det_voxels, dtype=np.int32)
    ndet = dv.size
    det = np.zeros((nsteps, max(ndet, 1)), dtype=np.float64)
    integ = np.zeros((nsteps, 2), dtype=np.float64)
    st = prob._struct()
    I_ = C.c_int
    lib().orc_run(C.byref(st), _ptr(psi), float(dt), int(nsteps), float(t_start),
                  len(src[0]), _ptr(src[0], I_), _ptr(src[1], I_), _ptr(src[2], C.c_double),
                  _ptr(src[3], C.c_double), _ptr(src[4], C.c_double),
                  ndet, _ptr(dv, I_), _ptr(det, C.c_double), _ptr(integ, C.c_double))
    return psi, det[:, :ndet], integ[:, 0] + 1j * integ[:, 1]


def gmres(prob: Problem, q, restart: int = 20, max_iter: int = 2000, rtol: float = 1e-10):
    """Steady state T psi = q by restarted GMRES in the (2l+1)-weighted inner
    product (Sec. II.A). Returns (psi, iterations, relative residual, converged)."""
    q = _field(prob, q)
    x = np.zeros_like(q)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = prob._struct()
    rc = lib().orc_gmres(C.byref(st), _ptr(q), _ptr(x), int(restart), int(max_iter), float(rtol),
                         C.byref(it), C.byref(rr))
    return x, it.value, rr.value, rc == 0


def adjoint(prob: Problem, psi0, dt: float, nsteps: int, weights, det_voxels,
            sources: Sources | None = None, t_start: float = 0.0):
    """Discrete adjoint of nsteps explicit steps. weights[n, d] = dL/dRe psi_00(r_d)
    at the pre-step state n. Returns (dL/dmu_a, dL/dmu_s) on the grid."""
    psi0 = _field(prob, psi0)
    src = (sources or Sources.none()).arrays()
    dv = np.ascontiguousarray(det_voxels, dtype=np.int32)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    assert w.shape == (nsteps, dv.size)
    ga = np.zeros(prob.shape)
    gs = np.zeros(prob.shape)
    mask = np.ascontiguousarray(prob.mask, dtype=np.uint8)
    st = prob._struct()
    I_ = C.c_int
    lib().orc_adjoint(C.byref(st), _ptr(mask), _ptr(psi0), float(dt), int(nsteps), float(t_start),
                      len(src[0]), _ptr(src[0], I_), _ptr(src[1], I_), _ptr(src[2], C.c_double),
                      _ptr(src[3], C.c_double), _ptr(src[4], C.c_double),
                      dv.size, _ptr(dv, I_), _ptr(w, C.c_double), _ptr(ga, C.c_double), _ptr(gs, C.c_double))
    return ga, gs


def exp_step(prob: Problem, psi0, dt: float, nsteps: int = 1):
    """Exponential integrator for a homogeneous medium on the periodic grid,
    the arbitrary-step scheme the paper names for homogeneous media (Sec. V):
    per wavevector k, psi^(k) <- expm(-c dt (S(k) + D)) psi^(k), with S(k)
    the streaming matrix of Eq. 10 and D = diag(mu_a + mu_s (1 - g^l)),
    applied nsteps times, between the grid's 3D DFT and its inverse (Eq. 7-8).
    The medium must be uniform and have no layer; there are no sources."""
    from scipy.linalg import expm
    a, s, g = prob.effective_media
    if prob.pml_width or np.ptp(a) or np.ptp(s) or np.ptp(g):
        raise ValueError("exp_step needs a uniform medium without a layer")
    N, M = prob.N, prob.M
    nz, ny, nx = prob.shape
    psi = _field(prob, psi0)
    hat = np.stack([fft3d(psi[j], -1) for j in range(M)])
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    D = np.diag(a.flat[0] + s.flat[0] * (1.0 - g.flat[0] ** ls))
    kx, ky, kz = wavenumbers(nx, prob.dx), wavenumbers(ny, prob.dx), wavenumbers(nz, prob.dx)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                E = expm(-prob.c * dt * (streaming_matrix(N, (kx[ix], ky[iy], kz[iz])) + D))
                v = hat[:, iz, iy, ix]
                for _ in range(nsteps):
                    v = E @ v
                hat[:, iz, iy, ix] = v
    out = np.stack([fft3d(hat[j], +1) for j in range(M)]) / (nx * ny * nz)
    return out


def gated_readouts(det_series, dt, t_start, gates):
    """y_d = sum_s dt * Re psi_00(r_d, t_s) over pre-step states t_s in [lo_d, hi_d]."""
    ns = det_series.shape[0]
    t = t_start + dt * np.arange(ns)
    y = np.zeros(det_series.shape[1])
    w = np.zeros_like(det_series)
    for d, (lo, hi) in enumerate(gates):
        sel = (t >= lo) & (t <= hi)
        w[:, d] = np.where(sel, dt, 0.0)
        y[d] = np.sum(w[:, d] * det_series[:, d])
    return y, w


# --------------------------------------------------------------------------
# Stability limit of the explicit step (Sec. II.A asserts conditional
# stability; the bound below is the standard amplification-factor condition).
# --------------------------------------------------------------------------

STAB_NK = 256            # |k| samples in (0, k_max]
STAB_MAX_CLASSES = 1024  # distinct interior media beyond which the extreme class is used


def media_classes(prob: Problem):
    """Distinct (mu_a, mu_s, g) triples of the folded media. If the interior
    holds more than STAB_MAX_CLASSES, the interior is represented by the single
    least-damped triple (min mu_a, min mu_s, max g); layer classes are kept."""
    a, s, g = prob._eff
    inl = prob.mask.astype(bool)
    interior = np.unique(np.stack([a[~inl], s[~inl], g[~inl]], axis=1), axis=0)
    layer = np.unique(np.stack([a[inl], s[inl], g[inl]], axis=1), axis=0) if inl.any() else np.zeros((0, 3))
    if interior.shape[0] > STAB_MAX_CLASSES:
        interior = np.array([[interior[:, 0].min(), interior[:, 1].min(), interior[:, 2].max()]])
    return np.concatenate([interior, layer], axis=0)


def k_max(prob: Problem) -> float:
    nz, ny, nx = prob.shape
    km = [np.max(np.abs(wavenumbers(n, prob.dx))) for n in (nx, ny, nz)]
    return float(np.sqrt(np.sum(np.square(km))))


def stability_limit(prob: Problem, direction=(1.0, 1.0, 1.0)) -> float:
    """dt* = min over media classes and |k| in {k_max j / STAB_NK, j = 0..STAB_NK} of
    min over eigenvalues lam of M_k = -c (S(k) + D) of 2 Re(-lam) / |lam|^2,
    so that every Fourier mode of a frozen-coefficient medium satisfies
    |1 + dt lam| <= 1. The spectrum of S(k) depends on |k| only; the oracle
    evaluates it along `direction` with the full (N+1)^2 matrix."""
    N = prob.N
    u = np.asarray(direction, dtype=np.float64)
    u = u / np.linalg.norm(u)
    kmax = k_max(prob)
    ks = kmax * np.arange(0, STAB_NK + 1) / STAB_NK
    Sunit = streaming_matrix(N, u)          # S is linear in k
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)], dtype=np.float64)
    best = math.inf
    for (mua, mus, g) in media_classes(prob):
        Dd = mua + mus * (1.0 - g ** ls)
        mats = -prob.c * (ks[:, None, None] * Sunit[None] + np.diag(Dd)[None])
        lam = np.linalg.eigvals(mats).ravel()
        lam = lam[np.abs(lam) > 0]
        re = -lam.real
        if np.any(re <= 0):
            return 0.0
        best = min(best, float(np.min(2.0 * re / np.abs(lam) ** 2)))
    return best
