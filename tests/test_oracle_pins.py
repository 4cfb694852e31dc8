"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle routine against something independent of the
oracle's own code: sphere quadrature with SciPy's spherical harmonics, textbook
DFT identities, closed-form decay laws, Legendre roots, the diffusion limit of
P_1, dense per-k solves, brute force and finite differences.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.special import roots_legendre, sph_harm_y

import oracle
import synth


# ---------------------------------------------------------------- helpers

def ylm_table(N, nth, nph):
    """Y_l^m on a Gauss-Legendre x trapezoid grid; returns (Y[M, P], w[P], s[3, P])."""
    x, wx = roots_legendre(nth)
    theta = np.arccos(x)
    phi = 2 * np.pi * np.arange(nph) / nph
    T, P = np.meshgrid(theta, phi, indexing="ij")
    W = np.outer(wx, np.full(nph, 2 * np.pi / nph))
    Y = []
    for l in range(N + 1):
        for m in range(-l, l + 1):
            Y.append(sph_harm_y(l, m, T, P).ravel())
    s = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)]).reshape(3, -1)
    return np.array(Y), W.ravel(), s


def quadrature_streaming(N, k):
    """S(k)[LM, lm] = (c_l / c_L) * i * sum_j k_j <Y_LM, s_j Y_lm> by quadrature,
    the projection of s.grad applied to phi = c_l exp(i k.r) Y_lm (Eq. 1, 3)."""
    Y, w, s = ylm_table(N, 2 * N + 6, 4 * N + 10)
    c = np.array([math.sqrt((2 * l + 1) / (4 * math.pi)) for l in range(N + 1) for _ in range(2 * l + 1)])
    ks = np.tensordot(np.asarray(k, dtype=float), s, axes=1)       # k . s at each node
    G = (np.conj(Y) * w) @ (Y * ks).T                                 # <Y_L, (k.s) Y_l>
    return 1j * G * c[None, :] / c[:, None]


def kgrid(shape, dx):
    """Wavenumbers with the Nyquist index set to zero, written out independently."""
    out = []
    for n in shape:
        i = np.arange(n)
        ip = np.where(2 * i < n, i, i - n)
        ip = np.where(2 * i == n, 0, ip)
        out.append(2 * np.pi * ip / (n * dx))
    kz, ky, kx = np.meshgrid(*out, indexing="ij")
    return kx, ky, kz


def wdot(N, u, v):
    wl = np.array([2 * l + 1 for l in range(N + 1) for _ in range(2 * l + 1)], dtype=float)
    return np.sum(wl[:, None] * np.conj(u.reshape(u.shape[0], -1)) * v.reshape(v.shape[0], -1))


# ---------------------------------------------------------------- Eq. 6 / Eq. 10

@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_streaming_matrix_matches_sphere_quadrature(N):
    """alpha/beta recurrence and the +ik reading of Eq. 10 against brute-force
    projection of s.grad onto the orthonormal complex harmonics (Eq. 3, 6)."""
    rng = np.random.default_rng(N)
    for k in [(0, 0, 1.0), (1.0, 0, 0), (0, 1.0, 0), tuple(rng.normal(size=3))]:
        S = oracle.streaming_matrix(N, k)
        Q = quadrature_streaming(N, k)
        assert np.max(np.abs(S - Q)) < 1e-13, (k, np.max(np.abs(S - Q)))


def test_alpha_beta_values():
    """Eq. 6 closed forms at a few indices."""
    assert oracle.alpha(3, 1) == pytest.approx(math.sqrt(4 * 2))
    assert oracle.alpha(2, 2) == 0.0
    assert oracle.beta(3, 1) == pytest.approx(math.sqrt(4 * 3))
    assert oracle.beta(2, -1) == 0.0
    assert oracle.beta(1, -1) == 0.0


@pytest.mark.parametrize("N", [2, 5, 7])
def test_streaming_spectrum_legendre_roots_and_isotropy(N):
    """The m = 0 block of the z-streaming matrix has eigenvalues i * roots of
    P_{N+1}; the full spectrum of S(k) depends only on |k|."""
    S = oracle.streaming_matrix(N, (0, 0, 1.0))
    idx0 = [oracle.moment_index(l, 0) for l in range(N + 1)]
    ev = np.sort(np.linalg.eigvals(S[np.ix_(idx0, idx0)] / 1j).real)
    roots = np.sort(roots_legendre(N + 1)[0])
    assert np.max(np.abs(ev - roots)) < 1e-12
    ez = np.sort_complex(np.round(np.linalg.eigvals(S), 10))
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    ed = np.sort_complex(np.round(np.linalg.eigvals(oracle.streaming_matrix(N, d)), 10))
    assert np.max(np.abs(ez - ed)) < 1e-9


# ---------------------------------------------------------------- DFT

@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8, 10, 12, 15, 16, 24, 96, 7, 14])
def test_fft_matches_naive_dft_and_identities(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    X = oracle.fft(x, -1)
    assert np.max(np.abs(X - oracle.dft_naive(x, -1))) < 1e-12 * max(1, n)
    # round trip
    assert np.max(np.abs(oracle.fft(X, +1) / n - x)) < 1e-13 * max(1, n)
    # closed forms: DFT of exp(2 pi i k0 j / n) is n delta_{k, k0}; of a delta is all ones
    for k0 in {0, n // 2, n - 1}:
        e = np.exp(2j * np.pi * k0 * np.arange(n) / n)
        want = np.zeros(n, complex)
        want[k0] = n
        assert np.max(np.abs(oracle.fft(e, -1) - want)) < 1e-12 * n
    d = np.zeros(n, complex)
    d[0] = 1
    assert np.max(np.abs(oracle.fft(d, -1) - 1)) < 1e-14


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 5), (4, 3, 8)])
def test_fft3d_matches_brute_force(shape):
    rng = np.random.default_rng(1)
    f = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    F = oracle.fft3d(f, -1)
    assert np.max(np.abs(F - oracle.dft3d_naive(f, -1))) < 1e-11
    assert np.max(np.abs(oracle.fft3d(F, +1) / f.size - f)) < 1e-13
    # separable plane wave -> single nonzero bin
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k0 = (1 % nz, 2 % ny, 3 % nx)
    e = np.exp(-2j * np.pi * (k0[0] * z / nz + k0[1] * y / ny + k0[2] * x / nx))
    E = oracle.fft3d(e, +1)
    want = np.zeros(shape, complex)
    want[k0] = f.size
    assert np.max(np.abs(E - want)) < 1e-10


# ---------------------------------------------------------------- Eq. 11 closed forms

def _homog(N, shape, dx, mua, mus, g, **kw):
    return oracle.Problem(N, shape, dx, synth.C_LIGHT, mua, mus, g, **kw)


def test_uniform_fields_decay_per_l_exactly():
    """A spatially uniform field has only k = 0: each step multiplies psi_l^m by
    exactly 1 - c dt (mu_a + mu_s (1 - g^l)); the continuous limit is
    exp(-c (mu_a + mu_s (1 - g^l)) t), reached at first order in dt."""
    N, shape, dx = 3, (4, 6, 5), 0.5
    mua, mus, g = 0.02, 3.0, 0.7
    p = _homog(N, shape, dx, mua, mus, g)
    rng = np.random.default_rng(3)
    amp = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
    psi0 = amp[:, None, None, None] * np.ones((p.M,) + shape)
    dt, n = 0.01, 7
    psi, _, _ = oracle.run(p, psi0, dt, n)
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    D = mua + mus * (1 - g ** ls)
    want = amp * (1 - synth.C_LIGHT * dt * D) ** n
    assert np.max(np.abs(psi[:, 0, 0, 0] - want) / np.abs(want)) < 1e-14
    assert np.max(np.abs(psi - psi[:, :1, :1, :1])) < 1e-14
    # first-order convergence to the exponential
    T = 0.4
    errs = []
    for dt in (0.02, 0.01, 0.005):
        psi, _, _ = oracle.run(p, psi0, dt, int(round(T / dt)))
        errs.append(np.max(np.abs(psi[:, 0, 0, 0] - amp * np.exp(-synth.C_LIGHT * D * T))))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_single_fourier_mode_matches_matrix_power_and_expm():
    """psi = v exp(i k.r) with k on the grid evolves as (I + dt M_k)^n v with
    M_k = -c (S(k) + D) (Eq. 10-11); against expm(n dt M_k) the error is O(dt)."""
    from scipy.linalg import expm
    N, shape, dx = 3, (8, 8, 8), 0.5
    mua, mus, g = 0.01, 1.0, 0.5
    p = _homog(N, shape, dx, mua, mus, g)
    nz, ny, nx = shape
    ik = (1, 2, 3)                          # (kz, ky, kx) indices
    kx, ky, kz = kgrid(shape, dx)
    kvec = (kx[ik], ky[ik], kz[ik])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wave = np.exp(2j * np.pi * (ik[0] * z / nz + ik[1] * y / ny + ik[2] * x / nx))
    rng = np.random.default_rng(5)
    v = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
    psi0 = v[:, None, None, None] * wave[None]
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    Mk = -synth.C_LIGHT * (quadrature_streaming(N, kvec) + np.diag(mua + mus * (1 - g ** ls)))
    dt, n = 0.02, 25
    psi, _, _ = oracle.run(p, psi0, dt, n)
    want = np.linalg.matrix_power(np.eye(p.M) + dt * Mk, n) @ v
    got = psi[:, 2, 3, 4] / wave[2, 3, 4]
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    assert np.max(np.abs(psi - got[:, None, None, None] * wave[None])) < 1e-12
    T = 0.8
    errs = []
    for dt in (0.04, 0.02, 0.01):
        psi, _, _ = oracle.run(p, psi0, dt, int(round(T / dt)))
        errs.append(np.max(np.abs(psi[:, 2, 3, 4] / wave[2, 3, 4] - expm(T * Mk) @ v)))
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_integral_of_fluence_decays_with_mu_a_only():
    """In a periodic homogeneous medium without sources the k = 0 row of the
    streaming term vanishes, so sum_r psi_00 is multiplied per step by exactly
    1 - c dt mu_a."""
    N, shape, dx = 3, (8, 8, 8), 0.5
    p = _homog(N, shape, dx, 0.01, 1.0, 0.5)
    psi0 = synth.smooth_random_state(N, shape, dx, seed=11)
    dt, n = 0.03, 20
    _, _, integ = oracle.run(p, psi0, dt, n)
    ratio = integ[1:] / integ[:-1]
    assert np.max(np.abs(ratio - (1 - synth.C_LIGHT * dt * 0.01))) < 1e-13


def test_point_source_injects_c_dt_q():
    """With zero state and zero media one step adds exactly c dt q(t_0) at the
    source voxel and moment (Eq. 11 with the source term read as c dt q)."""
    N, shape, dx = 2, (4, 4, 4), 0.5
    p = _homog(N, shape, dx, 0.0, 0.0, 0.0)
    src = oracle.Sources(np.array([21]), np.array([0]), np.array([2.0]), np.array([1.0]), np.array([3.0]))
    dt = 0.05
    psi, _, _ = oracle.run(p, np.zeros((p.M,) + shape), dt, 1, t_start=0.4, sources=src)
    q = 2.0 * math.exp(-4 * math.log(2) * ((0.4 - 1.0) / 3.0) ** 2) / dx ** 3
    flat = psi.reshape(p.M, -1)
    assert flat[0, 21] == pytest.approx(synth.C_LIGHT * dt * q, rel=1e-15)
    flat[0, 21] = 0
    assert np.max(np.abs(flat)) == 0.0


def test_real_radiance_symmetry_and_cubic_invariance():
    """psi_l^{-m} = (-1)^m conj(psi_l^m) is preserved, and psi_00 of the centred
    isotropic pulse is invariant under the 48 symmetries of the cubic grid."""
    N, n, dx = 3, 16, 0.5
    shape = (n, n, n)
    p = _homog(N, shape, dx, 0.01, 1.0, 0.5)
    psi0 = synth.gaussian_pulse_state(N, shape, dx, 1.0)
    psi, _, _ = oracle.run(p, psi0, 0.03, 12)
    for l in range(N + 1):
        for m in range(1, l + 1):
            a = psi[oracle.moment_index(l, -m)]
            b = (-1) ** m * np.conj(psi[oracle.moment_index(l, m)])
            assert np.max(np.abs(a - b)) < 1e-13
    f = psi[0].real
    assert np.max(np.abs(psi[0].imag)) < 1e-13
    refl = np.concatenate([[0], np.arange(n - 1, 0, -1)])   # j -> (n - j) mod n about index n/2
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product([False, True], repeat=3):
            g = np.transpose(f, perm)
            for ax, fl in enumerate(flips):
                if fl:
                    g = np.take(g, refl, axis=ax)
            assert np.max(np.abs(g - f)) < 1e-13


def test_streaming_sign_gives_outward_flux():
    """After a few steps the centred pulse carries J_z = psi_1^0 > 0 above the
    centre and < 0 below it: radiance streams away from the source."""
    N, n, dx = 3, 16, 0.5
    shape = (n, n, n)
    p = _homog(N, shape, dx, 0.01, 1.0, 0.5)
    psi, _, _ = oracle.run(p, synth.gaussian_pulse_state(N, shape, dx, 1.0), 0.03, 10)
    jz = psi[oracle.moment_index(1, 0)].real[:, n // 2, n // 2]
    c = n // 2
    assert np.all(jz[c + 1:c + 4] > 0) and np.all(jz[c - 3:c] < 0)
    assert abs(jz[c]) < 1e-12 * np.max(np.abs(jz))


# ---------------------------------------------------------------- PML and stability

def test_pml_profile_closed_form():
    """Half-cosine profile mu0 -> mu1 over W cells (Sec. II.B), max over axes in
    edges and corners, zero inside Omega."""
    W, mu0, mu1 = 3, 0.5, 4.0
    mub, mask = oracle.pml_profile((10, 12, 11), W, mu0, mu1)
    prof = lambda d: mu0 + (mu1 - mu0) * (1 - np.cos(np.pi * d / W)) / 2
    assert mub[5, 6, 0] == pytest.approx(prof(W - 0.5))
    assert mub[5, 6, 2] == pytest.approx(prof(0.5))
    assert mub[5, 6, 10] == pytest.approx(prof(W - 0.5))
    assert mub[5, 6, 8] == pytest.approx(prof(0.5))
    assert mub[0, 1, 5] == pytest.approx(max(prof(W - 0.5), prof(W - 1.5)))
    assert mask[5, 6, 5] == 0 and mub[5, 6, 5] == 0
    assert mask.sum() == 10 * 12 * 11 - 4 * 6 * 5


def test_stability_limit_uniform_damping_closed_form():
    """With the same damping d for every l (mu_s = 0), the eigenvalues are
    -c (d + i |k| x_j), x_j the roots of P_{N+1}, so
    dt* = 2 d / (c (d^2 + k_max^2 x_max^2))."""
    for N in (1, 3, 7):
        shape, dx, d = (16, 12, 10), 0.25, 1.3
        p = _homog(N, shape, dx, d, 0.0, 0.9)
        kx, ky, kz = kgrid(shape, dx)
        kmax = math.sqrt(np.max(np.abs(kx)) ** 2 + np.max(np.abs(ky)) ** 2 + np.max(np.abs(kz)) ** 2)
        xmax = np.max(roots_legendre(N + 1)[0])
        want = 2 * d / (synth.C_LIGHT * (d * d + kmax * kmax * xmax * xmax))
        assert oracle.stability_limit(p) == pytest.approx(want, rel=1e-9)
        assert oracle.stability_limit(p, (0, 0, 1)) == pytest.approx(want, rel=1e-9)


def _damping_only_limit(d, kmax, N):
    """Closed form of the explicit-step limit for one medium class with the same
    damping d in every l (mu_s = 0): the eigenvalues of -c (S(k) + d) are
    -c (d +- i |k| x_j) with x_j the roots of P_{N+1}, so the class allows
    dt = 2 d / (c (d^2 + k_max^2 x_max^2))."""
    xmax = np.max(roots_legendre(N + 1)[0])
    return 2 * d / (synth.C_LIGHT * (d * d + kmax * kmax * xmax * xmax))


def _kmax(shape, dx):
    kx, ky, kz = kgrid(shape, dx)
    return math.sqrt(np.max(np.abs(kx)) ** 2 + np.max(np.abs(ky)) ** 2 + np.max(np.abs(kz)) ** 2)


def test_stability_limit_takes_the_minimum_over_media_classes():
    """Two interior regions without scattering: the limit is the smaller of the
    two closed forms (here the weaker absorber, because both lie below the
    turning point d = k_max x_max of 2d / (d^2 + K^2)). Taking the largest class,
    the first or the last would give another value."""
    N, shape, dx = 3, (12, 14, 16), 0.25
    kmax = _kmax(shape, dx)
    a1, a2 = 0.05, 0.4
    mua = np.full(shape, a2)
    mua[:, :, :8] = a1
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, mua, 0.0, 0.8)
    cls = oracle.media_classes(p)
    assert sorted(cls[:, 0].tolist()) == [a1, a2] and np.all(cls[:, 1] == 0)
    f1, f2 = _damping_only_limit(a1, kmax, N), _damping_only_limit(a2, kmax, N)
    assert f1 < 0.5 * f2
    assert oracle.stability_limit(p) == pytest.approx(f1, rel=1e-9)
    # swap the regions: same answer (the minimum does not depend on the order)
    p2 = oracle.Problem(N, shape, dx, synth.C_LIGHT, mua[:, :, ::-1].copy(), 0.0, 0.8)
    assert oracle.stability_limit(p2) == pytest.approx(f1, rel=1e-9)


def test_stability_limit_counts_every_layer_level():
    """Interior damping near the turning point and a strongly absorbing layer
    (Eq. 12, mu_s = 0 there): the largest layer level, mu_b at depth W - 1/2,
    sets the limit by the closed form. Dropping the layer classes, or keeping
    only its first level, gives a larger value."""
    N, shape, dx, W = 2, (12, 12, 14), 0.25, 2
    kmax = _kmax(shape, dx)
    xmax = np.max(roots_legendre(N + 1)[0])
    K = kmax * xmax
    a1, a2 = 0.9 * K, 1.2 * K
    mu0, mu1 = 8 * K, 20 * K
    mua = np.full(shape, a1)
    mua[:6] = a2
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, mua, 0.0, 0.9, pml_width=W, pml_mu0=mu0, pml_mu1=mu1)
    prof = lambda d: mu0 + (mu1 - mu0) * (1 - np.cos(np.pi * d / W)) / 2
    levels = [prof(j + 0.5) for j in range(W)]
    cls = oracle.media_classes(p)
    for lv in levels:
        assert np.any(np.isclose(cls[:, 0], lv, rtol=1e-14) & (cls[:, 1] == 0))
    want = min(_damping_only_limit(d, kmax, N) for d in [a1, a2] + levels)
    assert want == pytest.approx(_damping_only_limit(levels[-1], kmax, N), rel=1e-15)
    interior_only = min(_damping_only_limit(d, kmax, N) for d in (a1, a2))
    assert want < 0.5 * interior_only
    assert _damping_only_limit(levels[0], kmax, N) > 1.5 * want
    assert oracle.stability_limit(p) == pytest.approx(want, rel=1e-9)


def test_stability_limit_collapses_many_classes_to_the_least_damped_triple():
    """More than 1024 distinct interior triples are represented by one class,
    (min mu_a, min mu_s, max g).
    - Without scattering the closed form applies: the limit is that of the
      smallest mu_a (both extremes lie below the turning point, where the
      limit grows with damping).
    - With scattering: the limit equals that of a uniform medium made of the
      triple, and differs from the uniform media made of each of the three
      swapped extremes (max mu_a, max mu_s or min g), so a swap fails here."""
    N, shape, dx = 2, (12, 12, 12), 0.25
    kmax = _kmax(shape, dx)
    rng = np.random.default_rng(11)
    mua = rng.uniform(0.05, 0.3, size=shape)
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, mua, 0.0, 0.9)
    cls = oracle.media_classes(p)
    assert cls.shape[0] == 1 and cls[0, 0] == mua.min()
    assert oracle.stability_limit(p) == pytest.approx(_damping_only_limit(mua.min(), kmax, N), rel=1e-9)
    assert _damping_only_limit(mua.max(), kmax, N) > 2 * _damping_only_limit(mua.min(), kmax, N)

    mus = rng.uniform(2.0, 12.0, size=shape)
    g = rng.uniform(0.3, 0.95, size=shape)
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, mua, mus, g)
    cls = oracle.media_classes(p)
    assert cls.shape[0] == 1
    assert tuple(cls[0]) == (mua.min(), mus.min(), g.max())
    uni = lambda a, s, gg: oracle.stability_limit(_homog(N, shape, dx, a, s, gg))
    want = uni(mua.min(), mus.min(), g.max())
    got = oracle.stability_limit(p)
    assert got == pytest.approx(want, rel=1e-12)
    for swapped in ((mua.max(), mus.min(), g.max()), (mua.min(), mus.max(), g.max()),
                    (mua.min(), mus.min(), g.min())):
        assert abs(uni(*swapped) - want) > 1e-3 * want


def test_stability_limit_bounds_growth():
    """Stepping the most unstable Fourier mode of a homogeneous medium at 0.99 dt*
    does not grow; at 1.3 dt* it does."""
    N, shape, dx = 3, (8, 8, 8), 0.5
    p = _homog(N, shape, dx, 0.01, 1.0, 0.5)
    dts = oracle.stability_limit(p)
    kx, ky, kz = kgrid(shape, dx)
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    k = (kx[3, 3, 3], ky[3, 3, 3], kz[3, 3, 3])
    Mk = -synth.C_LIGHT * (quadrature_streaming(N, k) + np.diag(0.01 + 1.0 * (1 - 0.5 ** ls)))
    rho = lambda dt: np.max(np.abs(np.linalg.eigvals(np.eye(p.M) + dt * Mk)))
    assert rho(0.99 * dts) <= 1 + 1e-12
    kmaxv = (kx[3, 3, 3], ky[3, 3, 3], kz[3, 3, 3])
    assert np.linalg.norm(kmaxv) == pytest.approx(oracle.k_max(p))
    assert rho(1.3 * dts) > 1


# ---------------------------------------------------------------- steady state

def test_p1_steady_state_is_diffusion():
    """N = 1, homogeneous, periodic: psi_00^(k) = q^(k) / (mu_a + |k|^2 / (3 (mu_a + mu_s (1-g))))."""
    N, shape, dx = 1, (8, 8, 8), 0.5
    mua, mus, g = 0.05, 2.0, 0.6
    p = _homog(N, shape, dx, mua, mus, g)
    q = np.zeros((p.M,) + shape, complex)
    q[0, 4, 4, 4] = 1.0
    q[0, 1, 2, 6] = 0.5
    x, it, rr, ok = oracle.gmres(p, q, restart=30, max_iter=3000, rtol=1e-12)
    assert ok
    kx, ky, kz = kgrid(shape, dx)
    K2 = kx ** 2 + ky ** 2 + kz ** 2
    qh = np.fft.fftn(q[0])
    want = np.fft.ifftn(qh / (mua + K2 / (3 * (mua + mus * (1 - g)))))
    assert np.max(np.abs(x[0] - want)) < 1e-9 * np.max(np.abs(want))


def test_gmres_matches_dense_per_k_solve():
    """Homogeneous periodic medium, any N: psi^(k) = (S(k) + D)^-1 q^(k)."""
    N, shape, dx = 3, (6, 8, 5), 0.5
    mua, mus, g = 0.03, 1.5, 0.8
    p = _homog(N, shape, dx, mua, mus, g)
    q = synth.random_state(N, shape, seed=21)
    x, it, rr, ok = oracle.gmres(p, q, restart=40, max_iter=4000, rtol=1e-12)
    assert ok and rr <= 1e-12
    kx, ky, kz = kgrid(shape, dx)
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    D = np.diag(mua + mus * (1 - g ** ls))
    qh = np.fft.fftn(q, axes=(1, 2, 3))
    xh = np.empty_like(qh)
    for idx in np.ndindex(shape):
        A = quadrature_streaming(N, (kx[idx], ky[idx], kz[idx])) + D
        xh[(slice(None),) + idx] = np.linalg.solve(A, qh[(slice(None),) + idx])
    want = np.fft.ifftn(xh, axes=(1, 2, 3))
    assert np.max(np.abs(x - want)) < 1e-8 * np.max(np.abs(want))


def test_heterogeneous_T_is_streaming_plus_local_damping():
    """T psi - F^-1[S F psi] = D_l(r) psi pointwise, with the PML folded in
    (mu_a -> mu_b, mu_s -> 0, Eq. 12) written out here independently."""
    N, shape, dx, W = 2, (12, 10, 14), 0.4, 3
    wl = synth.c2(shape=shape, dx=dx, N=N, W=W)
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, wl.mua, wl.mus, wl.g, W, 2.0, 10.0)
    psi = synth.random_state(N, shape, seed=4)
    diff = oracle.apply_T(p, psi) - oracle.apply_streaming(p, psi)
    mub, mask = oracle.pml_profile(shape, W, 2.0, 10.0)
    inl = mask.astype(bool)
    for l in range(N + 1):
        D = np.where(inl, mub, wl.mua + wl.mus * (1 - wl.g ** l))
        for m in range(-l, l + 1):
            j = oracle.moment_index(l, m)
            assert np.max(np.abs(diff[j] - D * psi[j])) < 1e-12


def test_gmres_heterogeneous_residual():
    N, shape, dx, W = 2, (12, 12, 12), 0.4, 3
    wl = synth.c2(shape=shape, dx=dx, N=N, W=W)
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, wl.mua, wl.mus, wl.g, W, 2.0, 10.0)
    q = np.zeros((p.M,) + shape, complex)
    q[0, 6, 6, 6] = 1.0 / dx ** 3
    x, it, rr, ok = oracle.gmres(p, q, restart=20, max_iter=3000, rtol=1e-10)
    assert ok
    r = q - oracle.apply_T(p, x)
    assert math.sqrt(wdot(N, r, r).real / wdot(N, q, q).real) <= 1.01e-10


# ---------------------------------------------------------------- adjoint

def test_adjoint_operator_dot_product():
    """<T^H u, v> = <u, T v> in the Euclidean inner product."""
    N, shape, dx, W = 3, (8, 10, 6), 0.5, 2
    wl = synth.c2(shape=shape, dx=dx, N=N, W=W)
    p = oracle.Problem(N, shape, dx, synth.C_LIGHT, wl.mua, wl.mus, wl.g, W, 2.0, 10.0)
    u = synth.random_state(N, shape, seed=7)
    v = synth.random_state(N, shape, seed=8)
    lhs = np.vdot(oracle.apply_T_adjoint(p, u), v)
    rhs = np.vdot(u, oracle.apply_T(p, v))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_adjoint_gradient_matches_central_differences():
    """dL/dmu_a and dL/dmu_s of L = sum_d y_d^2 (gated readouts) against central
    finite differences of the forward oracle."""
    N, shape, dx, W = 2, (8, 8, 8), 0.5, 2
    wl = synth.c5(shape=shape, dx=dx, N=N, W=W, nsteps=40, nsrc=2, ndet=3)
    dt, ns = 0.05, 40
    src = oracle.Sources(wl.src_voxel, np.zeros(2, np.int32), wl.src_amp, np.array([0.5, 0.8]),
                         np.array([0.6, 0.6]))
    gates = np.array([[0.2, 1.5], [0.5, 2.0], [0.0, 2.0]])

    def loss(mua, mus):
        p = oracle.Problem(N, shape, dx, synth.C_LIGHT, mua, mus, wl.g, W, 2.0, 10.0)
        _, det, _ = oracle.run(p, np.zeros((p.M,) + shape), dt, ns, sources=src, det_voxels=wl.det_voxel)
        y, w = oracle.gated_readouts(det, dt, 0.0, gates)
        return np.sum(y * y), y, w, p

    L0, y, w, p = loss(wl.mua, wl.mus)
    weights = w * (2 * y)[None, :]
    ga, gs = oracle.adjoint(p, np.zeros((p.M,) + shape), dt, ns, weights, wl.det_voxel, sources=src)
    flat = np.argsort(-np.abs(ga).ravel())[:4]
    for v in flat:
        idx = np.unravel_index(v, shape)
        for which, grad in (("a", ga), ("s", gs)):
            base = (wl.mua if which == "a" else wl.mus)
            h = 1e-4 * base[idx]
            plus = base.copy(); plus[idx] += h
            minus = base.copy(); minus[idx] -= h
            if which == "a":
                fd = (loss(plus, wl.mus)[0] - loss(minus, wl.mus)[0]) / (2 * h)
            else:
                fd = (loss(wl.mua, plus)[0] - loss(wl.mua, minus)[0]) / (2 * h)
            assert fd == pytest.approx(grad[idx], rel=1e-6, abs=1e-12 * abs(L0)), (which, idx)
    assert np.all(ga[p.mask.astype(bool)] == 0)


def test_exp_step_uniform_field_decays_exactly():
    """exp_step on a spatially uniform field (k = 0 only): each moment decays
    as exp(-c D_l t) for any dt, with D_l = mu_a + mu_s (1 - g^l)."""
    N, shape, dx = 3, (8, 8, 8), 0.5
    mua, mus, g = 0.02, 1.5, 0.7
    p = _homog(N, shape, dx, mua, mus, g)
    rng = np.random.default_rng(11)
    v = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
    psi0 = v[:, None, None, None] * np.ones(shape)[None]
    dt = 3.0                                # far beyond the explicit limit
    psi = oracle.exp_step(p, psi0, dt, 2)
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    want = v * np.exp(-synth.C_LIGHT * (mua + mus * (1 - g ** ls)) * 2 * dt)
    assert np.max(np.abs(psi - want[:, None, None, None])) < 1e-13 * np.max(np.abs(v))


def test_exp_step_single_mode_matches_quadrature_expm():
    """A single Fourier mode evolves with expm(t M_k), M_k = -c (S(k) + D),
    S(k) built here by sphere quadrature, independently of the oracle's S."""
    from scipy.linalg import expm
    N, shape, dx = 3, (8, 8, 8), 0.5
    mua, mus, g = 0.01, 1.0, 0.5
    p = _homog(N, shape, dx, mua, mus, g)
    nz, ny, nx = shape
    ik = (1, 2, 3)
    kx, ky, kz = kgrid(shape, dx)
    kvec = (kx[ik], ky[ik], kz[ik])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wave = np.exp(2j * np.pi * (ik[0] * z / nz + ik[1] * y / ny + ik[2] * x / nx))
    rng = np.random.default_rng(5)
    v = rng.normal(size=p.M) + 1j * rng.normal(size=p.M)
    ls = np.array([l for l in range(N + 1) for _ in range(2 * l + 1)])
    Mk = -synth.C_LIGHT * (quadrature_streaming(N, kvec) + np.diag(mua + mus * (1 - g ** ls)))
    psi = oracle.exp_step(p, v[:, None, None, None] * wave[None], 0.4, 2)
    want = expm(0.8 * Mk) @ v
    assert np.max(np.abs(psi - want[:, None, None, None] * wave[None])) < 1e-11 * np.max(np.abs(want))


def test_exp_step_is_the_limit_of_the_explicit_step():
    """On a smooth field, explicit steps of dt converge to exp_step at first
    order (error halves with dt), and exp_step composes: two steps of t/2
    equal one step of t."""
    N, shape, dx = 2, (8, 8, 8), 0.5
    p = _homog(N, shape, dx, 0.01, 2.0, 0.8)
    psi0 = synth.smooth_random_state(N, shape, dx, seed=9, corr=1.0)
    T = 0.4
    want = oracle.exp_step(p, psi0, T, 1)
    assert np.max(np.abs(oracle.exp_step(p, psi0, T / 2, 2) - want)) < 1e-12 * np.max(np.abs(want))
    errs = []
    for n in (20, 40, 80):
        psi, _, _ = oracle.run(p, psi0, T / n, n)
        errs.append(np.max(np.abs(psi - want)))
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_exp_step_rejects_layered_or_heterogeneous_media():
    p = _homog(1, (8, 8, 8), 0.5, 0.01, 1.0, 0.5, pml_width=2, pml_mu0=1.0, pml_mu1=2.0)
    with pytest.raises(ValueError):
        oracle.exp_step(p, np.zeros((4, 8, 8, 8)), 0.1)


def test_gated_readouts_rectangle_rule_by_hand():
    """y_d = dt * sum of Re psi_00 over the pre-step times inside [lo, hi]
    (closed gate), checked on a series whose sums are known by hand."""
    dt = 0.5
    series = np.column_stack([np.arange(8.0), np.ones(8), np.arange(8.0) ** 2])
    # times 0, 0.5, ..., 3.5 (t_start 0); gates [1, 2], [0, 10], [3.5, 3.5]
    y, w = oracle.gated_readouts(series, dt, 0.0, [(1.0, 2.0), (0.0, 10.0), (3.5, 3.5)])
    assert y[0] == pytest.approx(0.5 * (2 + 3 + 4))        # t = 1.0, 1.5, 2.0 -> indices 2, 3, 4
    assert y[1] == pytest.approx(0.5 * 8)
    assert y[2] == pytest.approx(0.5 * 49)                 # only t = 3.5 (index 7)
    assert np.array_equal(w[:, 0] > 0, (np.arange(8) >= 2) & (np.arange(8) <= 4))
    y2, _ = oracle.gated_readouts(series, dt, 1.0, [(1.0, 2.0), (0.0, 10.0), (3.5, 3.5)])
    assert y2[0] == pytest.approx(0.5 * (0 + 1 + 2))       # shifted start: indices 0, 1, 2
