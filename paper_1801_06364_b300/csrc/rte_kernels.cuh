// rte_kernels.cuh -- the device kernels of one explicit step / one operator
// application of the pseudospectral P_N method (Powell, Cox & Arridge,
// arXiv:1801.06364, Sec. II-III).
//
// State representation. The plan keeps psi~ = F_xy psi: every moment field
// transformed along x and y (unnormalised DFT, exp(-i k.r)) and left in real
// space along z. Layout [M][nz][ny][nx] (kx fastest), complex, plan precision.
// With the state in this form one step needs:
//   Z    per-moment spectral z-derivative  Dz = F_z^-1[i kz F_z psi~]
//   Y^-1 inverse y-DFT of psi~ (columns)                        -> T1
//   X    inverse x-DFT, pointwise stage, forward x-DFT (rows)    -> T1
//   Y+   forward y-DFT of T1, plus a psi~ + coefS * S~(psi~, Dz)  -> psi~'
// where S~ is the streaming term of Eq. 10 in the mixed (kx, ky, z) space:
//   S~_lm = 1/(2l+1) [ a_{l+1}^m Dz_{l+1,m} + a_l^m Dz_{l-1,m}
//           - 1/2 (i kx + ky)(b_l^m psi~_{l-1,m-1} - b_{l+1}^{1-m} psi~_{l+1,m-1})
//           - 1/2 (i kx - ky)(-b_l^{-m} psi~_{l-1,m+1} + b_{l+1}^{m+1} psi~_{l+1,m+1}) ].
// The pointwise stage (paper stages 2-3) computes in real space
//   inc = coefD * D_l(r) psi + injections,   D_l = mu_a + mu_s (1 - g^l),
// so that a step (coefD = -c dt, a = 1, coefS = -c dt) gives
//   psi~' = psi~ - c dt (S~ + F_xy[D psi]) + F_xy[c dt q],
// the update of Eq. 11 written as state + increment, and an operator
// application (coefD = 1, a = 0, coefS = 1) gives T psi~.
#pragma once
#include "rte_fft.cuh"

namespace rte {

template <typename R> struct Geo {
    using T = typename cvec<R>::type;
    int nx, ny, nz, M;
    FftPlan px, py, pz;
    const T *twx, *twy, *twz;     // exp(-2 pi i j / n) per axis
    const R *kx, *ky, *kz;        // wavenumbers (Nyquist -> 0)
    // set to 1 by the pass that writes the updated state when an output of
    // the kx = 0 column is not finite (one non-finite value anywhere in a
    // plane reaches every kx of it through the x transform within a step)
    int *nonfinite;
};

// flag a non-finite value (see Geo::nonfinite)
template <typename T> __device__ __forceinline__ void flag_nonfinite(int *flag, const T &v) {
    if (flag && !(isfinite(v.x) && isfinite(v.y))) atomicOr(flag, 1);
}

template <typename R> struct Media4;
template <> struct Media4<float> { using type = float4; };
template <> struct Media4<double> { using type = double4_32a; };

// Arguments of the X pass.
template <typename R> struct XArgs {
    using T = typename cvec<R>::type;
    int inv_in;            // apply the inverse x-DFT to the loaded rows
    int pointwise;         // apply the pointwise stage
    int fwd_out;           // apply the forward x-DFT before storing
    R coefD;               // multiplies D_l psi
    const typename Media4<R>::type *med;   // (mu_a, mu_s, g, interior) per voxel
    const int *lof;        // l of each moment
    const int *step;       // device step counter (readouts, injections)
    // pre-step readouts of Re psi_00 at detector voxels
    int ndet;
    const int4 *det;       // (x, y, z, unused)
    double *det_out;       // [step][ndet]
    // injections: amp[step * ninj + i] added to moment inj.w at voxel (x, y, z)
    int ninj;
    const int4 *inj;
    const R *inj_amp;
    // real-space record of psi (adjoint forward segment) and gradient terms
    T *rec_out;            // [M][V] or null
    const T *rec_in;       // psi_n in real space for the gradient, or null
    double *grad_a, *grad_s;
    R grad_scale;          // -c dt
    const R *wl;           // c_l^2 = (2l+1)/4pi per moment, for the adjoint gradient
};

template <typename T> __device__ __forceinline__ T czero() { return mk<T>(0, 0); }

// Shared-memory tiles: two buffers of `elems` complex values each (the FFT
// ping-pongs between them).
template <typename T> __device__ __forceinline__ T *tile0() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<T *>(smem_raw);
}
template <typename T> __device__ __forceinline__ T *other(T *r, T *s0, T *s1) { return r == s0 ? s1 : s0; }

constexpr int kMaxThreads = 512;

// ---------------------------------------------------------------- Z pass
// One CTA: moment m, row ky, TX consecutive kx columns, all z.
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_zderiv(const typename cvec<R>::type *__restrict__ in,
                                                        typename cvec<R>::type *__restrict__ out, Geo<R> g, int TX) {
    using T = typename cvec<R>::type;
    const int P = TX + 1;
    T *s0 = tile0<T>(), *s1 = s0 + g.nz * P;
    const int x0 = blockIdx.x * TX, y = blockIdx.y, m = blockIdx.z;
    const size_t plane = (size_t)g.ny * g.nx;
    const size_t base = (size_t)m * g.nz * plane + (size_t)y * g.nx + x0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int cnt = g.nz * TX;
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / TX, b = i - e * TX;
        s0[e * P + b] = (x0 + b < g.nx) ? in[base + e * plane + b] : czero<T>();
    }
    __syncthreads();
    T *r = fft_lines<T>(s0, s1, g.pz, TX, P, 1, g.twz, tid, nthr);
    const R inv = R(1) / R(g.nz);
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / TX, b = i - e * TX;
        const T v = r[e * P + b];
        const R k = g.kz[e] * inv;
        // conj(i k v): the inverse DFT is taken as conj(FFT(conj(.)))
        r[e * P + b] = mk<T>(-k * v.y, -k * v.x);
    }
    __syncthreads();
    r = fft_lines<T>(r, other(r, s0, s1), g.pz, TX, P, 1, g.twz, tid, nthr);
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / TX, b = i - e * TX;
        if (x0 + b < g.nx) out[base + e * plane + b] = cconj(r[e * P + b]);
    }
}

// ---------------------------------------------------------------- Y passes
// One CTA: moment m, plane z, TX consecutive kx columns, all y.
// inverse != 0: out = F_y^-1 in. Otherwise out = F_y in, and when psi_in is
// given: out = a psi_in + F_y in + coefS * S~(psi_in, dz).
// in and out may alias (each CTA reads its whole tile first); psi_in and dz
// must not alias out.
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_ypass(const typename cvec<R>::type *in, typename cvec<R>::type *out,
                                                       Geo<R> g, int TX, int inverse,
                                                       const typename cvec<R>::type *__restrict__ psi_in,
                                                       const typename cvec<R>::type *__restrict__ dz, R a, R coefS,
                                                       const CouplingRow *__restrict__ coup) {
    using T = typename cvec<R>::type;
    const int P = TX + 1;
    T *s0 = tile0<T>(), *s1 = s0 + g.ny * P;
    const int x0 = blockIdx.x * TX, z = blockIdx.y, m = blockIdx.z;
    const size_t V = (size_t)g.nz * g.ny * g.nx;
    const size_t base = ((size_t)m * g.nz + z) * g.ny * g.nx + x0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int cnt = g.ny * TX;
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / TX, b = i - e * TX;
        T v = (x0 + b < g.nx) ? in[base + (size_t)e * g.nx + b] : czero<T>();
        s0[e * P + b] = inverse ? cconj(v) : v;
    }
    __syncthreads();
    const T *r = fft_lines<T>(s0, s1, g.py, TX, P, 1, g.twy, tid, nthr);
    if (inverse) {
        const R inv = R(1) / R(g.ny);
        for (int i = tid; i < cnt; i += nthr) {
            const int e = i / TX, b = i - e * TX;
            if (x0 + b < g.nx) out[base + (size_t)e * g.nx + b] = cscale(cconj(r[e * P + b]), inv);
        }
        return;
    }
    if (psi_in == nullptr) {
        for (int i = tid; i < cnt; i += nthr) {
            const int e = i / TX, b = i - e * TX;
            if (x0 + b < g.nx) out[base + (size_t)e * g.nx + b] = r[e * P + b];
        }
        return;
    }
    const CouplingRow cr = coup[m];
    const size_t zoff = (size_t)z * g.ny * g.nx;
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / TX, b = i - e * TX;
        const int x = x0 + b;
        if (x >= g.nx) continue;
        const size_t pos = zoff + (size_t)e * g.nx + x;   // (z, ky, kx) within a moment
        const R kx = g.kx[x], ky = g.ky[e];
        R sr = 0, si = 0;
        for (int t = 0; t < cr.n; ++t) {
            const R c = (R)cr.coef[t];
            const size_t src = (size_t)cr.src[t] * V + pos;
            if (cr.type[t] == 0) {
                const T d = dz[src];
                sr += c * d.x;
                si += c * d.y;
            } else {
                T u;
                if (cr.type[t] >= 3) {        // conj(psi~(-kx, -ky)), real-radiance layout
                    const int mx = x == 0 ? 0 : g.nx - x, my = e == 0 ? 0 : g.ny - e;
                    u = cconj(psi_in[(size_t)cr.src[t] * V + zoff + (size_t)my * g.nx + mx]);
                } else {
                    u = psi_in[src];
                }
                if (cr.type[t] == 1 || cr.type[t] == 3) {        // (i kx + ky)(u.x + i u.y)
                    sr += c * (ky * u.x - kx * u.y);
                    si += c * (kx * u.x + ky * u.y);
                } else {                      // (i kx - ky)(u.x + i u.y)
                    sr += c * (-ky * u.x - kx * u.y);
                    si += c * (kx * u.x - ky * u.y);
                }
            }
        }
        const T self = psi_in[(size_t)m * V + pos];
        const T f = r[e * P + b];
        const T o = mk<T>(a * self.x + f.x + coefS * sr, a * self.y + f.y + coefS * si);
        if (x == 0) flag_nonfinite(g.nonfinite, o);
        out[base + (size_t)e * g.nx + b] = o;
    }
}

// ---------------------------------------------------------------- X pass
// One CTA: MC moments (m0 .. m0+MC-1) of row (y, z), all x. in and out may alias.
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_xpass(const typename cvec<R>::type *in, typename cvec<R>::type *out,
                                                       Geo<R> g, int MC, XArgs<R> xa) {
    using T = typename cvec<R>::type;
    __shared__ int step_s;
    const int nx = g.nx, P = nx + 1;
    T *s0 = tile0<T>(), *s1 = s0 + MC * P;
    const int y = blockIdx.x, z = blockIdx.y, m0 = blockIdx.z * MC;
    const int mc = min(MC, g.M - m0);
    if (mc <= 0) return;
    const size_t V = (size_t)g.nz * g.ny * nx;
    const size_t row = ((size_t)z * g.ny + y) * nx;           // voxel index of x = 0
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int cnt = mc * nx;
    for (int i = tid; i < cnt; i += nthr) {
        const int b = i / nx, e = i - b * nx;
        T v = in[(size_t)(m0 + b) * V + row + e];
        s0[b * P + e] = xa.inv_in ? cconj(v) : v;
    }
    if (tid == 0) step_s = xa.step ? *xa.step : 0;
    __syncthreads();
    T *r = s0;
    if (xa.inv_in) {
        r = fft_lines<T>(s0, s1, g.px, mc, 1, P, g.twx, tid, nthr);
        const R inv = R(1) / R(nx);
        for (int i = tid; i < cnt; i += nthr) {
            const int b = i / nx, e = i - b * nx;
            r[b * P + e] = cscale(cconj(r[b * P + e]), inv);
        }
        __syncthreads();
    }
    if (xa.pointwise) {
        const int step = step_s;
        // pre-step readouts of Re psi_00
        if (m0 == 0) {
            for (int d = tid; d < xa.ndet; d += nthr) {
                const int4 p = xa.det[d];
                if (p.y == y && p.z == z) xa.det_out[(size_t)step * xa.ndet + d] = (double)r[p.x].x;
            }
        }
        if (xa.grad_a) {
            // adjoint gradient: this row holds lambda~_{n+1} in real space and
            // rec_in holds psi_n; sum over the moments of this chunk.
            for (int e = tid; e < nx; e += nthr) {
                const size_t v = row + e;
                const typename Media4<R>::type md = xa.med[v];
                if (md.w == R(0)) continue;
                double ga = 0.0, gs = 0.0;
                for (int b = 0; b < mc; ++b) {
                    const int m = m0 + b;
                    const T lam = r[b * P + e];
                    const T ps = xa.rec_in[(size_t)m * V + v];
                    const double pr = (double)xa.wl[m] * ((double)lam.x * ps.x + (double)lam.y * ps.y);
                    double gl = 1.0;
                    for (int q = 0; q < xa.lof[m]; ++q) gl *= (double)md.z;
                    ga += pr;
                    gs += (1.0 - gl) * pr;
                }
                atomicAdd(xa.grad_a + v, (double)xa.grad_scale * ga);
                atomicAdd(xa.grad_s + v, (double)xa.grad_scale * gs);
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += nthr) {
            const int b = i / nx, e = i - b * nx;
            const int m = m0 + b;
            const size_t v = row + e;
            const typename Media4<R>::type md = xa.med[v];
            R gl = 1;
            const int l = xa.lof[m];
            for (int q = 0; q < l; ++q) gl *= md.z;
            const R D = md.x + md.y * (R(1) - gl);
            const T p = r[b * P + e];
            if (xa.rec_out) xa.rec_out[(size_t)m * V + v] = p;
            r[b * P + e] = cscale(p, xa.coefD * D);
        }
        __syncthreads();
        if (tid == 0 && xa.ninj > 0) {
            for (int q = 0; q < xa.ninj; ++q) {
                const int4 p = xa.inj[q];
                if (p.y == y && p.z == z && p.w >= m0 && p.w < m0 + mc) {
                    T &t = r[(p.w - m0) * P + p.x];
                    t.x += xa.inj_amp[(size_t)step * xa.ninj + q];
                }
            }
        }
        __syncthreads();
    }
    if (xa.fwd_out) r = fft_lines<T>(r, other(r, s0, s1), g.px, mc, 1, P, g.twx, tid, nthr);
    for (int i = tid; i < cnt; i += nthr) {
        const int b = i / nx, e = i - b * nx;
        out[(size_t)(m0 + b) * V + row + e] = r[b * P + e];
    }
}

// ---------------------------------------------------------------- step end
// integral[2 step + {0,1}] = dx^3 sum_r psi_00 = dx^3 sum_z psi~_00(kx=0, ky=0, z)
// of the pre-step state, then step += delta. One warp.
template <typename R>
__global__ void k_advance(const typename cvec<R>::type *__restrict__ psi_t, int nx, int ny, int nz,
                          int *step, double *integral, double vol, int delta) {
    const int lane = threadIdx.x;
    if (integral) {
        double re = 0.0, im = 0.0;
        for (int z = lane; z < nz; z += 32) {
            const auto v = psi_t[(size_t)z * ny * nx];
            re += (double)v.x;
            im += (double)v.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            const int s = *step;
            integral[2 * s] = re * vol;
            integral[2 * s + 1] = im * vol;
        }
    }
    __syncwarp();
    if (lane == 0) *step += delta;
}

// g[v] = 0 on layer voxels (interior flag med.w == 0): the mu_a gradient is
// defined on the interior only
template <typename R>
__global__ void k_zero_layer(double *__restrict__ g, const typename Media4<R>::type *__restrict__ med, size_t V) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x)
        if (med[v].w == R(0)) g[v] = 0.0;
}

// ---------------------------------------------------------------- steady-state preconditioner
// Right preconditioner P^-1 of the steady operator T = S + D for GMRES (the
// method's steady problem, Sec. II.A, solved by a Krylov method). For a
// homogeneous medium with D_l = Dbar_l, T is block diagonal in k; P keeps the
// l <= 1 block of that operator exactly, (Dbar + S^(k)) on the moments
// (0,0), (1,-1), (1,0), (1,1), and D_l alone for l >= 2. The l <= 1 block
// carries the slowly decaying diffusive modes (D_0 = mu_a is small), which
// is where unpreconditioned GMRES spends its iterations.
struct PrecLow {
    int nterm;             // couplings among the l <= 1 moments (full layout, index l*l + l + m)
    int o[16], s[16], type[16];
    double coef[16];
    double d0, d1;         // Dbar_0, Dbar_1
};

// One CTA: row ky, TX consecutive kx columns, all z, the four l <= 1
// moments (element e of moment m, column b at s[e P4 + m TX + b]). Forward
// z-DFT of all four, a 4 x 4 solve per (kx, ky, kz), inverse z-DFT.
// real != 0: `in`/`out` hold the m >= 0 moments only ((0,0), (1,0), (1,1)
// at 0, 1, 2); (1,-1) is read as -conj(psi~_{1,1}(-kx, -ky, z)).
// out must not alias in.
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_prec_low(const typename cvec<R>::type *__restrict__ in,
                                                          typename cvec<R>::type *__restrict__ out, Geo<R> g, int TX,
                                                          int real, PrecLow pl) {
    using T = typename cvec<R>::type;
    const int L = 4 * TX, P4 = L + 1;
    T *s0 = tile0<T>(), *s1 = s0 + g.nz * P4;
    const int x0 = blockIdx.x * TX, y = blockIdx.y;
    const size_t plane = (size_t)g.ny * g.nx, V = plane * g.nz;
    const int ym = (g.ny - y) % g.ny;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int cnt = g.nz * L;
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / L, r = i - e * L, m = r / TX, b = r - m * TX, x = x0 + b;
        T v = czero<T>();
        if (x < g.nx) {
            if (!real) {
                v = in[(size_t)m * V + e * plane + (size_t)y * g.nx + x];
            } else if (m != 1) {
                v = in[(size_t)(m == 0 ? 0 : m - 1) * V + e * plane + (size_t)y * g.nx + x];
            } else {
                const T u = in[2 * V + e * plane + (size_t)ym * g.nx + (g.nx - x) % g.nx];
                v = mk<T>(-u.x, u.y);
            }
        }
        s0[e * P4 + r] = v;
    }
    __syncthreads();
    T *q = fft_lines<T>(s0, s1, g.pz, L, P4, 1, g.twz, tid, nthr);
    const R inv = R(1) / R(g.nz);
    for (int i = tid; i < g.nz * TX; i += nthr) {
        const int e = i / TX, b = i - e * TX, x = x0 + b;
        const R kx = x < g.nx ? g.kx[x] : R(0), ky = g.ky[y], kz = g.kz[e];
        // A = Dbar + S^(k) on the l <= 1 moments; S^: type 0 i kz, type 1 (i kx + ky), type 2 (i kx - ky)
        R ar[4][4], ai[4][4], br[4], bi[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < 4; ++c) ar[r][c] = ai[r][c] = R(0);
            ar[r][r] = (R)(r == 0 ? pl.d0 : pl.d1);
            const T v = q[e * P4 + r * TX + b];
            br[r] = v.x;
            bi[r] = v.y;
        }
        for (int t = 0; t < pl.nterm; ++t) {
            const R c = (R)pl.coef[t];
            const int ty = pl.type[t];
            const R fr = ty == 0 ? R(0) : (ty == 1 ? ky : -ky);
            const R fi = ty == 0 ? kz : kx;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                    if (r == pl.o[t] && cc == pl.s[t]) {
                        ar[r][cc] += c * fr;
                        ai[r][cc] += c * fi;
                    }
        }
        // Gaussian elimination with partial pivoting (complex 4 x 4)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int piv = k;
            R best = ar[k][k] * ar[k][k] + ai[k][k] * ai[k][k];
#pragma unroll
            for (int r = k + 1; r < 4; ++r) {
                const R m2 = ar[r][k] * ar[r][k] + ai[r][k] * ai[r][k];
                if (m2 > best) {
                    best = m2;
                    piv = r;
                }
            }
#pragma unroll
            for (int r = k + 1; r < 4; ++r)
                if (r == piv) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const R tr = ar[k][c], ti = ai[k][c];
                        ar[k][c] = ar[r][c];
                        ai[k][c] = ai[r][c];
                        ar[r][c] = tr;
                        ai[r][c] = ti;
                    }
                    const R tr = br[k], ti = bi[k];
                    br[k] = br[r];
                    bi[k] = bi[r];
                    br[r] = tr;
                    bi[r] = ti;
                }
            // 1 / pivot
            const R den = ar[k][k] * ar[k][k] + ai[k][k] * ai[k][k];
            const R pr = ar[k][k] / den, pi = -ai[k][k] / den;
#pragma unroll
            for (int r = k + 1; r < 4; ++r) {
                const R fr = ar[r][k] * pr - ai[r][k] * pi, fi = ar[r][k] * pi + ai[r][k] * pr;
#pragma unroll
                for (int c = k; c < 4; ++c) {
                    ar[r][c] -= fr * ar[k][c] - fi * ai[k][c];
                    ai[r][c] -= fr * ai[k][c] + fi * ar[k][c];
                }
                br[r] -= fr * br[k] - fi * bi[k];
                bi[r] -= fr * bi[k] + fi * br[k];
            }
        }
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            R sr = br[k], si = bi[k];
#pragma unroll
            for (int c = k + 1; c < 4; ++c) {
                sr -= ar[k][c] * br[c] - ai[k][c] * bi[c];
                si -= ar[k][c] * bi[c] + ai[k][c] * br[c];
            }
            const R den = ar[k][k] * ar[k][k] + ai[k][k] * ai[k][k];
            br[k] = (sr * ar[k][k] + si * ai[k][k]) / den;
            bi[k] = (si * ar[k][k] - sr * ai[k][k]) / den;
        }
        // inverse z-DFT as conj(F conj(.)) / nz
#pragma unroll
        for (int r = 0; r < 4; ++r) q[e * P4 + r * TX + b] = mk<T>(br[r] * inv, -bi[r] * inv);
    }
    __syncthreads();
    q = fft_lines<T>(q, other(q, s0, s1), g.pz, L, P4, 1, g.twz, tid, nthr);
    for (int i = tid; i < cnt; i += nthr) {
        const int e = i / L, r = i - e * L, m = r / TX, b = r - m * TX, x = x0 + b;
        if (x >= g.nx || (real && m == 1)) continue;
        const int mo = real ? (m == 0 ? 0 : m - 1) : m;
        out[(size_t)mo * V + e * plane + (size_t)y * g.nx + x] = cconj(q[e * P4 + r]);
    }
}

// out[m] = scale[m] in[m] per stored moment (the l >= 2 part of P^-1);
// grid (chunks, moments)
template <typename R>
__global__ void k_scale_moments(const typename cvec<R>::type *__restrict__ in, typename cvec<R>::type *__restrict__ out,
                                size_t V, const R *__restrict__ scale) {
    const R c = scale[blockIdx.y];
    const size_t off = (size_t)blockIdx.y * V;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
        const auto v = in[off + i];
        out[off + i] = mk<typename cvec<R>::type>(c * v.x, c * v.y);
    }
}

// ---------------------------------------------------------------- vectors
// FP64 weighted dot products for GMRES: res[i] = sum mw[moment] conj(B_i) w
// over ncol basis vectors B_i (stored contiguously, stride n); mw = 2l+1, and
// twice that for m > 0 in the real-radiance layout. Per-block partial sums go
// to part[blockIdx.x * ncol + i]; k_sum_parts adds them.
// Columns are taken 8 at a time so that w is read once per group. Columns
// ncolb..ncol-1 (at most one) stand for w itself, giving |w|^2 in the same pass.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2)
    k_wdot_multi(const typename cvec<R>::type *__restrict__ basis, size_t n, int ncolb, int ncol,
                             const typename cvec<R>::type *__restrict__ w, size_t V,
                             const double *__restrict__ mw, double2 *part) {
    // grid (chunks, moments): every block sees one moment, so its weight is uniform
    constexpr int G = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *red = reinterpret_cast<double2 *>(smem_raw);   // [ncol][32]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int mom = blockIdx.y;
    const double wgt = mw[mom];
    const size_t off = (size_t)mom * V;
    const auto *ww = w + off;
    for (int c0 = 0; c0 < ncol; c0 += G) {
        const int g = min(G, ncol - c0);
        double re[G], im[G];
        if constexpr (sizeof(R) == 4) {
            // FP32 products with compensated (Kahan) FP32 sums per thread; the
            // per-thread sums and everything after are FP64. B300's FP64 rate
            // is a small fraction of FP32, so per-element FP64 would bound it.
            float sr[G], cr[G], si[G], ci[G];
#pragma unroll
            for (int j = 0; j < G; ++j) sr[j] = cr[j] = si[j] = ci[j] = 0.f;
            for (size_t i = (size_t)blockIdx.x * blockDim.x + tid; i < V; i += (size_t)gridDim.x * blockDim.x) {
                // all operands of the group are requested before any arithmetic,
                // so that each thread keeps G + 1 loads in flight
                const auto v = ww[i];
                typename cvec<R>::type uu[G];
#pragma unroll
                for (int j = 0; j < G; ++j)
                    uu[j] = j < g && c0 + j < ncolb ? basis[(size_t)(c0 + j) * n + off + i] : v;
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    if (j >= g) break;
                    const auto u = uu[j];
                    const float pr = fmaf(u.x, v.x, u.y * v.y) - cr[j];
                    const float tr = sr[j] + pr;
                    cr[j] = (tr - sr[j]) - pr;
                    sr[j] = tr;
                    const float pi = fmaf(u.x, v.y, -(u.y * v.x)) - ci[j];
                    const float ti = si[j] + pi;
                    ci[j] = (ti - si[j]) - pi;
                    si[j] = ti;
                }
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                re[j] = (double)sr[j] - (double)cr[j];
                im[j] = (double)si[j] - (double)ci[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j) re[j] = im[j] = 0.0;
            for (size_t i = (size_t)blockIdx.x * blockDim.x + tid; i < V; i += (size_t)gridDim.x * blockDim.x) {
                const auto v = ww[i];
                typename cvec<R>::type uu[G];
#pragma unroll
                for (int j = 0; j < G; ++j)
                    uu[j] = j < g && c0 + j < ncolb ? basis[(size_t)(c0 + j) * n + off + i] : v;
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    if (j >= g) break;
                    const auto u = uu[j];
                    re[j] += (double)u.x * v.x + (double)u.y * v.y;
                    im[j] += (double)u.x * v.y - (double)u.y * v.x;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (j >= g) break;
            double a = re[j], bb = im[j];
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, o);
                bb += __shfl_down_sync(0xffffffffu, bb, o);
            }
            if (lane == 0) red[(c0 + j) * 32 + wid] = make_double2(wgt * a, wgt * bb);
        }
    }
    __syncthreads();
    const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int c = tid; c < ncol; c += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int q = 0; q < nw; ++q) {
            re += red[c * 32 + q].x;
            im += red[c * 32 + q].y;
        }
        part[blk * ncol + c] = make_double2(re, im);
    }
}

static __global__ void k_sum_parts(const double2 *__restrict__ part, int nblk, int ncol, double2 *res) {
    const int c = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        re += part[(size_t)b * ncol + c].x;
        im += part[(size_t)b * ncol + c].y;
    }
    __shared__ double sr[32], si[32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sr[wid] = re;
        si[wid] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += sr[q];
            b += si[q];
        }
        res[c] = make_double2(a, b);
    }
}

// out = scale (w - sum_i h_i B_i)  (h in FP64, device; out may be w)
// (element arithmetic in the plan precision: the result is stored in it)
template <typename R>
__global__ void k_sub_multi(const typename cvec<R>::type *__restrict__ basis, size_t n, int ncol,
                            const double2 *__restrict__ h, const typename cvec<R>::type *w,
                            typename cvec<R>::type *out, R scale) {
    __shared__ R hr[64], hi[64];
    for (int c = threadIdx.x; c < ncol && c < 64; c += blockDim.x) {
        hr[c] = (R)h[c].x;
        hi[c] = (R)h[c].y;
    }
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        R re = w[i].x, im = w[i].y;
        for (int c = 0; c < ncol; ++c) {
            const auto u = basis[(size_t)c * n + i];
            re -= hr[c] * u.x - hi[c] * u.y;
            im -= hr[c] * u.y + hi[c] * u.x;
        }
        out[i].x = scale * re;
        out[i].y = scale * im;
    }
}

// y += sum_i c_i B_i (FP64 coefficients)
template <typename R, typename Q>
__global__ void k_add_multi(const typename cvec<Q>::type *__restrict__ basis, size_t n, int ncol,
                            const double2 *__restrict__ c, typename cvec<R>::type *y) {
    __shared__ R cr[64], ci[64];
    for (int q = threadIdx.x; q < ncol && q < 64; q += blockDim.x) {
        cr[q] = (R)c[q].x;
        ci[q] = (R)c[q].y;
    }
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        R re = y[i].x, im = y[i].y;
        for (int q = 0; q < ncol; ++q) {
            const auto u = basis[(size_t)q * n + i];
            re += cr[q] * (R)u.x - ci[q] * (R)u.y;
            im += cr[q] * (R)u.y + ci[q] * (R)u.x;
        }
        y[i].x = re;
        y[i].y = im;
    }
}

// y = alpha * x + beta * y with complex FP64 alpha, beta (x may be null)
template <typename R, typename Q>
__global__ void k_axpby(const typename cvec<Q>::type *__restrict__ x, typename cvec<R>::type *y, size_t n,
                        double ar, double ai, double br, double bi) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(R) == 4 && sizeof(Q) == 4) {
            float xr = 0.f, xi = 0.f, yr = 0.f, yi = 0.f;
            if (x) {
                xr = x[i].x;
                xi = x[i].y;
            }
            if (br != 0.0 || bi != 0.0) {
                yr = y[i].x;
                yi = y[i].y;
            }
            const float a0 = (float)ar, a1 = (float)ai, b0 = (float)br, b1 = (float)bi;
            y[i].x = a0 * xr - a1 * xi + b0 * yr - b1 * yi;
            y[i].y = a0 * xi + a1 * xr + b0 * yi + b1 * yr;
            continue;
        }
        double xr = 0.0, xi = 0.0, yr = 0.0, yi = 0.0;
        if (x) {
            xr = x[i].x;
            xi = x[i].y;
        }
        if (br != 0.0 || bi != 0.0) {      // y is not read when beta = 0
            yr = y[i].x;
            yi = y[i].y;
        }
        y[i].x = (R)(ar * xr - ai * xi + br * yr - bi * yi);
        y[i].y = (R)(ar * xi + ai * xr + br * yi + bi * yr);
    }
}

// Rebuild the m < 0 moments of a full-layout field whose m >= 0 moments are
// in place: f[(l, -m)] = (-1)^m conj(f[(l, m)]) (real radiance).
template <typename R>
__global__ void k_mirror_moments(typename cvec<R>::type *f, size_t V, int N) {
    const int M = (N + 1) * (N + 1);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)M * V;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / V);
        int l = 0;
        while ((l + 1) * (l + 1) <= j) ++l;
        const int m = j - l * l - l;
        if (m >= 0) continue;
        const auto s = f[(size_t)(l * l + l - m) * V + (i % V)];
        const R sg = (-m) % 2 ? R(-1) : R(1);
        f[i].x = sg * s.x;
        f[i].y = -sg * s.y;
    }
}

// The m < 0 moments of a real radiance from its stored m >= 0 moments
// (stored index l (l + 1) / 2 + m): out[j] = (-1)^m conj(psi_{l,m}) with
// j = l (l - 1) / 2 + m - 1 over l >= 1, 1 <= m <= l. Grid: (voxel blocks, j).
template <typename R>
__global__ void k_negative_moments(const typename cvec<R>::type *__restrict__ stored,
                                   typename cvec<R>::type *__restrict__ out, size_t V) {
    const int j = blockIdx.y;
    int l = 1;
    while ((l + 1) * l / 2 <= j) ++l;
    const int m = j - l * (l - 1) / 2 + 1;
    const R sg = m % 2 ? R(-1) : R(1);
    const auto *src = stored + (size_t)(l * (l + 1) / 2 + m) * V;
    auto *dst = out + (size_t)j * V;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (size_t)gridDim.x * blockDim.x) {
        const auto a = src[v];
        dst[v].x = sg * a.x;
        dst[v].y = -sg * a.y;
    }
}

// f[moment][voxel] += val for a short list of points (one thread: points may repeat)
template <typename R>
__global__ void k_scatter_points(typename cvec<R>::type *f, size_t V, int n, const long long *voxel,
                                 const int *moment, const double *val) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        for (int q = 0; q < n; ++q) f[(size_t)moment[q] * V + voxel[q]].x += (R)val[q];
}

}  // namespace rte
