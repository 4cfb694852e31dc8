"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the
oracle: optical maps, initial states, source and detector placements.

This module holds none of the transport method's arithmetic (no transforms,
no coefficients, no time stepping); it only draws inputs. Random numbers come
from a splitmix64 stream (Steele, Lea & Flood, OOPSLA 2014), so that every
array is reproducible from its seed on any machine.

Workloads (all lengths in mm, times in ps, coefficients in 1/mm):
  C1  32^3, dx 0.5, P_3, homogeneous (0.01, 1, 0.5), periodic, Gaussian pulse
  C2  128^3, dx 0.25, P_7, PML 12, background (0.01, 10, 0.9) + 8 spheres
  C3  256^3, dx 0.2, P_5, PML 16, three z-slabs with log-normal mu_s
  C4  serving: grids {64,96,128,160}^3, N in {3,5,7,9}, 1-6 spheres
  C5  128^3, dx 0.25, P_5, PML 12, Gaussian-random-field media, 4 sources
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1801063640
C_LIGHT = 0.214          # mm/ps, the speed used throughout the workloads
PML_MU0 = 2.0            # 1/mm at the inner edge of the layer
PML_MU1 = 10.0           # 1/mm at the outer boundary

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of splitmix64 from `seed`, starting at stream position `offset`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential draws from one splitmix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int = 1, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller pairs."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi)."""
        return lo + np.floor(self.uniform(n) * (hi - lo)).astype(np.int64)


def coords(n: int, dx: float) -> np.ndarray:
    """Cell-centre coordinates x_j = (j - n/2) dx: the grid centre is index n/2."""
    return (np.arange(n) - n // 2) * dx


def flat_index(shape, z, y, x):
    nz, ny, nx = shape
    return (np.asarray(z) * ny + np.asarray(y)) * nx + np.asarray(x)


def gaussian_pulse_state(N: int, shape, dx: float, sigma: float = 1.0) -> np.ndarray:
    """Isotropic Gaussian exp(-|r|^2 / 2 sigma^2) at the grid centre in the
    l = 0 moment; all other moments zero. Shape (M, nz, ny, nx), complex128."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(coords(nz, dx), coords(ny, dx), coords(nx, dx), indexing="ij")
    psi = np.zeros(((N + 1) ** 2, nz, ny, nx), dtype=np.complex128)
    psi[0] = np.exp(-(x * x + y * y + z * z) / (2.0 * sigma * sigma))
    return psi


def random_state(N: int, shape, seed: int, real_radiance: bool = False) -> np.ndarray:
    """Unit-variance complex Gaussian noise in every moment (parity fixtures)."""
    M = (N + 1) ** 2
    V = int(np.prod(shape))
    s = Stream(seed)
    re = s.normal(M * V).reshape((M,) + tuple(shape))
    im = s.normal(M * V).reshape((M,) + tuple(shape))
    return re + 1j * im


def smooth_random_state(N: int, shape, dx: float, seed: int, corr: float = 1.5) -> np.ndarray:
    """Band-limited random moments: white noise filtered by exp(-|k|^2 corr^2/4)."""
    raw = random_state(N, shape, seed)
    return np.stack([_filter(raw[j], dx, corr) for j in range(raw.shape[0])])


def real_radiance_state(N: int, shape, dx: float, seed: int, corr: float = 1.0) -> np.ndarray:
    """Smooth random moments of a real radiance: psi_l^0 real and
    psi_l^{-m} = (-1)^m conj(psi_l^m) (complex harmonics, Condon-Shortley phase)."""
    psi = smooth_random_state(N, shape, dx, seed, corr)
    for l in range(N + 1):
        j0 = l * l + l
        psi[j0] = psi[j0].real
        for m in range(1, l + 1):
            psi[j0 - m] = (-1) ** m * np.conj(psi[j0 + m])
    return psi


def _filter(f, dx, corr):
    nz, ny, nx = f.shape
    kz = 2 * np.pi * np.fft.fftfreq(nz, dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, dx)
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    return np.fft.ifftn(np.fft.fftn(f) * np.exp(-K2 * corr * corr / 4.0))


@dataclass
class Workload:
    name: str
    N: int
    shape: tuple
    dx: float
    mua: np.ndarray
    mus: np.ndarray
    g: np.ndarray
    pml_width: int = 0
    pml_mu0: float = PML_MU0
    pml_mu1: float = PML_MU1
    c: float = C_LIGHT
    src_voxel: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    src_amp: np.ndarray = field(default_factory=lambda: np.zeros(0))
    src_t0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    src_fwhm: np.ndarray = field(default_factory=lambda: np.zeros(0))
    det_voxel: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    det_gate: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    nsteps: int = 0
    dt_fraction: float = 0.5

    @property
    def M(self):
        return (self.N + 1) ** 2

    @property
    def V(self):
        return int(np.prod(self.shape))


def _interior_bounds(n, W):
    return W, n - W        # Omega is [W, n-W) on each axis


def _paint_spheres(stream, shape, dx, W, count, r_lo, r_hi, mua, mus, g,
                   mua_rng, mus_rng, g_rng=None, r_is_fraction=False):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    side = (min(shape) - 2 * W) * dx
    for _ in range(count):
        r = stream.uniform(1, r_lo, r_hi)[0]
        if r_is_fraction:
            r *= side
        c = []
        for n in (nz, ny, nx):
            lo, hi = _interior_bounds(n, W)
            a, b = lo * dx + r, hi * dx - r
            if b <= a:
                a = b = 0.5 * (lo + hi) * dx
            c.append(stream.uniform(1, a, b)[0])
        sa = stream.uniform(1, *mua_rng)[0]
        ss = stream.uniform(1, *mus_rng)[0]
        sg = stream.uniform(1, *g_rng)[0] if g_rng is not None else None
        inside = ((z + 0.5) * dx - c[0]) ** 2 + ((y + 0.5) * dx - c[1]) ** 2 + ((x + 0.5) * dx - c[2]) ** 2 <= r * r
        mua[inside] = sa
        mus[inside] = ss
        if sg is not None:
            g[inside] = sg


def _interior_voxels(stream, shape, W, count):
    nz, ny, nx = shape
    zs = stream.integers(count, W, nz - W)
    ys = stream.integers(count, W, ny - W)
    xs = stream.integers(count, W, nx - W)
    return flat_index(shape, zs, ys, xs).astype(np.int64)


def c1() -> Workload:
    """32^3 periodic grid, dx 0.5, P_3, homogeneous medium, Gaussian pulse."""
    shape = (32, 32, 32)
    return Workload("C1: 32^3 P_3 periodic, Gaussian pulse", 3, shape, 0.5,
                    np.full(shape, 0.01), np.full(shape, 1.0), np.full(shape, 0.5),
                    pml_width=0, nsteps=200)


def c2(shape=(128, 128, 128), dx=0.25, N=7, W=12, nsteps=2000) -> Workload:
    """128^3, dx 0.25, P_7, PML 12, background + 8 seeded spheres, pulsed l=0
    point source at the grid centre (FWHM 10 ps, t0 15 ps), 16 detectors."""
    s = Stream(BASE_SEED + 2)
    mua = np.full(shape, 0.01)
    mus = np.full(shape, 10.0)
    g = np.full(shape, 0.9)
    _paint_spheres(s, shape, dx, W, 8, 2.0, 6.0, mua, mus, g, (0.005, 0.1), (5.0, 20.0))
    nz, ny, nx = shape
    src = np.array([flat_index(shape, nz // 2, ny // 2, nx // 2)], dtype=np.int64)
    det = _interior_voxels(s, shape, W, 16)
    return Workload(f"C2: {nx}^3 P_{N} PML {W}, 8 spheres, pulsed source", N, shape, dx, mua, mus, g,
                    pml_width=W, src_voxel=src, src_amp=np.array([1.0]), src_t0=np.array([15.0]),
                    src_fwhm=np.array([10.0]), det_voxel=det, nsteps=nsteps)


def c3(shape=(256, 256, 256), dx=0.2, N=5, W=16) -> Workload:
    """256^3, dx 0.2, P_5, PML 16, three z-slabs, mu_s *= exp(0.2 Z - 0.02),
    continuous-wave l=0 source at the grid centre."""
    s = Stream(BASE_SEED + 3)
    nz, ny, nx = shape
    mua = np.empty(shape)
    mus = np.empty(shape)
    g = np.full(shape, 0.8)
    z = np.arange(nz)
    lo, hi = _interior_bounds(nz, W)
    slab = np.clip(((z - lo) * 3) // max(hi - lo, 1), 0, 2)
    for k, (a, b) in enumerate([(0.02, 8.0), (0.01, 12.0), (0.05, 6.0)]):
        mua[slab == k] = a
        mus[slab == k] = b
    mus *= np.exp(0.2 * s.normal(mus.size).reshape(shape) - 0.02)
    src = np.array([flat_index(shape, nz // 2, ny // 2, nx // 2)], dtype=np.int64)
    return Workload(f"C3: {nx}^3 P_{N} PML {W}, layered log-normal, CW source", N, shape, dx,
                    mua, mus, g, pml_width=W, src_voxel=src, src_amp=np.array([1.0]),
                    src_t0=np.array([0.0]), src_fwhm=np.array([0.0]))


def c4_request(i: int, grids=(64, 96, 128, 160), orders=(3, 5, 7, 9), steps_range=(500, 3000),
               W: int = 12) -> Workload:
    """One request of the serving workload: grid drawn from {64,96,128,160}^3,
    dx 0.25, N from {3,5,7,9}, 500-3000 steps, PML 12, 1-6 spheres. The
    keyword arguments draw a scaled-down mix from the same recipe."""
    s = Stream(BASE_SEED + 4 + 1000 * i)
    n = int(grids[s.integers(1, 0, len(grids))[0]])
    N = int(orders[s.integers(1, 0, len(orders))[0]])
    steps = int(s.integers(1, steps_range[0], steps_range[1] + 1)[0])
    shape = (n, n, n)
    mua = np.full(shape, s.uniform(1, 0.005, 0.1)[0])
    mus = np.full(shape, s.uniform(1, 2.0, 20.0)[0])
    g = np.full(shape, s.uniform(1, 0.7, 0.95)[0])
    count = int(s.integers(1, 1, 7)[0])
    _paint_spheres(s, shape, 0.25, W, count, 0.1, 0.25, mua, mus, g, (0.005, 0.1), (2.0, 20.0),
                   (0.7, 0.95), r_is_fraction=True)
    src = np.array([flat_index(shape, n // 2, n // 2, n // 2)], dtype=np.int64)
    det = _interior_voxels(s, shape, W, 16)
    return Workload(f"C4 request {i}: {n}^3 P_{N}", N, shape, 0.25, mua, mus, g, pml_width=W,
                    src_voxel=src, src_amp=np.array([1.0]), src_t0=np.array([15.0]),
                    src_fwhm=np.array([10.0]), det_voxel=det, nsteps=steps)


def e1(n: int = 64) -> Workload:
    """The paper's transient run without PML (Sec. IV A): a 50 mm cube on an
    n^3 grid, mu_a 0.01, mu_s 1.0, g 0.9, mu_s 5.0 where x <= 15 mm (x from 0
    at the cube face), P_21, 400 steps; the initial state is an isotropic
    Gaussian of 1/e diameter 1.5 mm at the centre (gaussian_pulse_state with
    sigma = 0.75 / sqrt(2) mm)."""
    shape = (n, n, n)
    dx = 50.0 / n
    mua = np.full(shape, 0.01)
    mus = np.full(shape, 1.0)
    g = np.full(shape, 0.9)
    x = (np.arange(n) + 0.5) * dx
    mus[:, :, x <= 15.0] = 5.0
    return Workload(f"E1: {n}^3 P_21, 50 mm cube, mu_s step at x = 15 mm", 21, shape, dx, mua, mus, g,
                    pml_width=0, nsteps=400)


def e2(n: int = 64) -> Workload:
    """The paper's steady-state run with PML (Sec. IV B): a 50 mm cube on an
    n^3 grid holding a 35.5 mm cube of mu_a 0.01, mu_s 10, g 0.95 inside a
    half-cosine layer rising from 0.01 to 1.0 /mm (the layer 7.25 mm, whole
    cells); P_7; a constant isotropic source 8 mm from the centre along x (a
    point source: the 1.5 mm Gaussian spans about two cells); 25 000 steps."""
    shape = (n, n, n)
    dx = 50.0 / n
    W = int(round(7.25 / dx))
    mua = np.full(shape, 0.01)
    mus = np.full(shape, 10.0)
    g = np.full(shape, 0.95)
    c = n // 2
    src = np.array([flat_index(shape, c, c, c + int(round(8.0 / dx)))], dtype=np.int64)
    return Workload(f"E2: {n}^3 P_7, 35.5 mm cube in a 50 mm layer box, CW source", 7, shape, dx, mua, mus, g,
                    pml_width=W, pml_mu0=0.01, pml_mu1=1.0, src_voxel=src, src_amp=np.array([1.0]),
                    src_t0=np.array([0.0]), src_fwhm=np.array([0.0]), nsteps=25000)


def c5(shape=(128, 128, 128), dx=0.25, N=5, W=12, nsteps=1500, nsrc=4, ndet=32) -> Workload:
    """Gaussian random field media (correlation 3 mm) about mu_a 0.01, mu_s 10,
    g 0.9; pulsed sources with staggered t0 and time-gated detectors."""
    s = Stream(BASE_SEED + 5)
    G1 = _unit_grf(s, shape, dx, 3.0)
    G2 = _unit_grf(s, shape, dx, 3.0)
    mua = 0.01 * np.exp(0.2 * G1 - 0.02)
    mus = 10.0 * np.exp(0.2 * G2 - 0.02)
    g = np.full(shape, 0.9)
    src = _interior_voxels(s, shape, W, nsrc)
    t0 = 15.0 + 5.0 * np.arange(nsrc)
    det = _interior_voxels(s, shape, W, ndet)
    tlo = s.uniform(ndet, 5.0, 15.0)
    gates = np.stack([tlo, tlo + 20.0], axis=1)
    return Workload(f"C5: {shape[2]}^3 P_{N} PML {W}, GRF media, {nsrc} sources", N, shape, dx,
                    mua, mus, g, pml_width=W, src_voxel=src, src_amp=np.ones(nsrc),
                    src_t0=t0, src_fwhm=np.full(nsrc, 10.0), det_voxel=det, det_gate=gates,
                    nsteps=nsteps)


def _unit_grf(stream, shape, dx, corr):
    white = stream.normal(int(np.prod(shape))).reshape(shape)
    f = np.real(_filter(white, dx, corr))
    return (f - f.mean()) / f.std()
