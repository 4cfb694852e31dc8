// rte_expo.cuh -- exponential integrator for a homogeneous periodic medium:
// the arbitrary-step scheme the paper names for homogeneous media (Sec. V).
// With a uniform medium the transport operator is diagonal in k, so per
// wavevector psi^(k, t + dt) = E_k psi^(k, t), E_k = expm(-c dt (S(k) + D)),
// S(k) the streaming matrix of Eq. 10 and D = diag(mu_a + mu_s (1 - g^l)).
// The plan's state (xy-Fourier, z-real) is taken to full k-space by a z-DFT,
// stepped by E_k, and brought back by the inverse z-DFT.
#pragma once
#include "rte_plane.cuh"

namespace rte {

// z-DFT of every moment in place, one CTA per (TX columns, y, moment):
// out = F_z in, or F_z^-1 in (normalised) when inverse != 0. Two-phase DIF;
// phase B writes natural order through the slot map. in and out may alias.
template <typename R, int N1, int N2, int TX, int NT>
__global__ void __launch_bounds__(NT) k_zdft_fixed(const typename cvec<R>::type *in, typename cvec<R>::type *out,
                                                   Geo<R> g, int inverse) {
    using T = typename cvec<R>::type;
    constexpr int NZ = N1 * N2, P = TX + 1;
    __shared__ T s[NZ * P];
    __shared__ T tw[NZ];
    const int x0 = blockIdx.x * TX, y = blockIdx.y, m = blockIdx.z;
    const size_t plane = (size_t)g.ny * g.nx;
    const size_t base = (size_t)m * NZ * plane + (size_t)y * g.nx + x0;
    const int tid = threadIdx.x;
    for (int i = tid; i < NZ; i += NT) tw[i] = g.twz[i];
    __syncthreads();
    for (int w = tid; w < TX * N2; w += NT) {
        const int b = w % TX, t = w / TX;
        const bool ok = x0 + b < g.nx;
        T v[N1];
#pragma unroll
        for (int q = 0; q < N1; ++q) {
            const T u = ok ? in[base + (size_t)(t + N2 * q) * plane + b] : czero<T>();
            v[q] = inverse ? cconj(u) : u;
        }
        dftR<T, N1>(v);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) s[(t + N2 * k1) * P + b] = v[k1];
    }
    __syncthreads();
    const R inv = R(1) / R(NZ);
    for (int w = tid; w < TX * N1; w += NT) {
        const int b = w % TX, k1 = w / TX;
        T v[N2];
#pragma unroll
        for (int t = 0; t < N2; ++t) v[t] = s[(N2 * k1 + t) * P + b];
        dftR<T, N2>(v);
        if (x0 + b >= g.nx) continue;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2)
            out[base + (size_t)(k1 + N1 * k2) * plane + b] = inverse ? cscale(cconj(v[k2]), inv) : v[k2];
    }
}

// Terms of the M x M streaming matrix: entry (o, s) gains coef * f_type(k),
// f_0 = i kz, f_1 = i kx + ky, f_2 = i kx - ky (Eq. 10, d -> +ik).
struct ExpoArgs {
    int M, nterm;
    const int4 *term;          // (o, s, type, unused)
    const double *coef;
    const double *dl;          // D_l per moment (M)
    double cdt;                // c dt
    int nsub;                  // Taylor degree
};

// E is tiled by 32 wavevectors: entry e = c M + r (row r, column c) of
// wavevector k at ((k / 32) M^2 + e) 32 + k % 32, so that a warp's 32 wavevectors read each
// entry as one 256-byte segment and all their entries as one contiguous
// block (V is a multiple of 32: nz is).
__device__ __forceinline__ size_t expm_index(size_t k, int e, int MM) {
    return (((k >> 5) * (size_t)MM + (size_t)e) << 5) + (k & 31);
}

// C = A B for M x M complex matrices in shared memory (row-major), all threads
template <int NT> __device__ void zgemm_smem(const double2 *A, const double2 *B, double2 *C, int M) {
    for (int e = threadIdx.x; e < M * M; e += NT) {
        const int r = e / M, c = e - r * M;
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < M; ++j) {
            const double2 a = A[r * M + j], b = B[j * M + c];
            sr += a.x * b.x - a.y * b.y;
            si += a.x * b.y + a.y * b.x;
        }
        C[e] = make_double2(sr, si);
    }
    __syncthreads();
}

// One CTA per wavevector (kx, ky, kz indices from blockIdx.x): E_k in FP64 by
// scaling and squaring a Taylor series. B = -c dt A / 2^s with |B|_1 <= 1/2,
// E = I + B (I + B/2 (I + ... (I + B/K))) by Horner, then squared s times;
// stored in the plan precision, tiled by 32 wavevectors (expm_index).
// Dynamic shared memory: 3 M^2 double2.
template <typename R, int NT>
__global__ void __launch_bounds__(NT) k_expm_build(Geo<R> g, ExpoArgs ea, typename cvec<R>::type *E) {
    extern __shared__ __align__(16) unsigned char xsm[];
    const int M = ea.M, MM = M * M;
    double2 *A = reinterpret_cast<double2 *>(xsm), *X = A + MM, *Y = X + MM;
    __shared__ double colsum[128];
    __shared__ int s_sh;
    const size_t k = blockIdx.x;
    const int ix = (int)(k % g.nx), iy = (int)((k / g.nx) % g.ny), iz = (int)(k / ((size_t)g.nx * g.ny));
    const double kx = (double)g.kx[ix], ky = (double)g.ky[iy], kz = (double)g.kz[iz];
    for (int e = threadIdx.x; e < MM; e += NT) A[e] = make_double2(0.0, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 0; t < ea.nterm; ++t) {
            const int4 q = ea.term[t];
            const double c = ea.coef[t];
            const double fr = q.z == 0 ? 0.0 : (q.z == 1 ? ky : -ky), fi = q.z == 0 ? kz : kx;
            double2 &a = A[q.x * M + q.y];
            a.x += c * fr;
            a.y += c * fi;
        }
        for (int r = 0; r < M; ++r) A[r * M + r].x += ea.dl[r];
    }
    __syncthreads();
    // |c dt A|_1 and the scaling power s
    for (int c = threadIdx.x; c < M; c += NT) {
        double acc = 0.0;
        for (int r = 0; r < M; ++r) acc += hypot(A[r * M + c].x, A[r * M + c].y);
        colsum[c] = acc * ea.cdt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double nrm = 0.0;
        for (int c = 0; c < M; ++c) nrm = fmax(nrm, colsum[c]);
        int s = 0;
        while (nrm > 0.5 && s < 60) {
            nrm *= 0.5;
            ++s;
        }
        s_sh = s;
    }
    __syncthreads();
    const int s = s_sh;
    const double scale = -ea.cdt * ldexp(1.0, -s);
    for (int e = threadIdx.x; e < MM; e += NT) {
        A[e] = make_double2(A[e].x * scale, A[e].y * scale);      // A <- B
        X[e] = make_double2((e / M) == (e % M) ? 1.0 : 0.0, 0.0);  // X <- I
    }
    __syncthreads();
    for (int j = ea.nsub; j >= 1; --j) {
        zgemm_smem<NT>(A, X, Y, M);                                // Y = B X
        const double inv = 1.0 / j;
        for (int e = threadIdx.x; e < MM; e += NT)
            X[e] = make_double2(((e / M) == (e % M) ? 1.0 : 0.0) + Y[e].x * inv, Y[e].y * inv);
        __syncthreads();
    }
    for (int q = 0; q < s; ++q) {
        zgemm_smem<NT>(X, X, Y, M);
        for (int e = threadIdx.x; e < MM; e += NT) X[e] = Y[e];
        __syncthreads();
    }
    using T = typename cvec<R>::type;
    // column-major within the tile: entry (r, c) at c M + r, so that the
    // apply kernel reads the rows of one column as one contiguous run
    for (int e = threadIdx.x; e < MM; e += NT)
        E[expm_index(k, (e % M) * M + e / M, MM)] = mk<T>((R)X[e].x, (R)X[e].y);
}

// out[r][k] = sum_c E_k[r][c] in[c][k]; one thread per wavevector, rows in
// blocks of RB held in registers. E_k is column-major within each tile of 32
// wavevectors, so a warp reads the RB rows of one column as RB consecutive
// 256-byte segments; eight columns are in flight at a time (with RB = 4 that
// is 36 loads per thread, the most memory-level parallelism at the fewest
// registers among the forms timed: the row-major form with 16 rows reached
// a third of the copy rate, this one 0.9 of it at 128^3 P_3).
template <typename R, int RB>
__global__ void k_expm_apply(const typename cvec<R>::type *__restrict__ E, const typename cvec<R>::type *__restrict__ in,
                             typename cvec<R>::type *__restrict__ out, size_t V, int M) {
    using T = typename cvec<R>::type;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < V; k += (size_t)gridDim.x * blockDim.x) {
        for (int r0 = 0; r0 < M; r0 += RB) {
            R ar[RB], ai[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u) ar[u] = ai[u] = R(0);
#pragma unroll 8
            for (int c = 0; c < M; ++c) {
                const T v = in[(size_t)c * V + k];
                // all RB entries requested before any arithmetic (predicated, no early exit)
                T e[RB];
#pragma unroll
                for (int u = 0; u < RB; ++u)
                    e[u] = r0 + u < M ? E[expm_index(k, c * M + r0 + u, M * M)] : mk<T>(R(0), R(0));
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    ar[u] += e[u].x * v.x - e[u].y * v.y;
                    ai[u] += e[u].x * v.y + e[u].y * v.x;
                }
            }
#pragma unroll
            for (int u = 0; u < RB; ++u)
                if (r0 + u < M) out[(size_t)(r0 + u) * V + k] = mk<T>(ar[u], ai[u]);
        }
    }
}

}  // namespace rte
