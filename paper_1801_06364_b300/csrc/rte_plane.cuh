// rte_plane.cuh -- fixed-size kernels of the step for the common grid axes
// (32, 64, 128 points): a fused per-plane kernel and a z-derivative kernel.
//
// Transforms of length n = N1 N2 are done in two in-place phases, one thread
// per sub-transform, with compile-time indices only:
//   DIF (natural order in, digit-reversed out):
//     A: thread t < N2 takes x[t + N2 q], q < N1: N1-point DFT, twiddle
//        w_n^{t k1}, writes back to the same slots t + N2 k1;
//     B: thread k1 < N1 takes the block N2 k1 + t, t < N2: N2-point DFT,
//        writes back to the same block. Slot N2 k1 + k2 then holds X[k1 + N1 k2].
//   DIT (digit-reversed in, natural out), the transpose of the above:
//     A: thread j1 < N1 takes the block N2 j1 + j2: N2-point DFT, twiddle
//        w_n^{j1 k2}, writes back to the block;
//     B: thread k2 < N2 takes slots N2 j1 + k2, j1 < N1: N1-point DFT, writes
//        X[k2 + N2 k1] to slot N2 k1 + k2 (natural order).
// Every thread writes exactly the slots it read, so no second buffer is
// needed; a barrier separates the phases. The inverse transform inverts the
// conjugate: F^-1 x = conj(F conj(x)) / n. An inverse DIF followed by a
// forward DIT therefore leaves natural order on both ends, and the pointwise
// stage in between maps slots to grid indices.
#pragma once
#include "rte_kernels.cuh"

namespace rte {

// w16^j = exp(-2 pi i j / 16) from cos(pi/8), sin(pi/8) and sqrt(1/2)
template <typename T> __device__ __forceinline__ T w16(int j) {
    using Rr = typename real_of<T>::type;
    const Rr c1 = (Rr)0.92387953251128675613, s1 = (Rr)0.38268343236508977173, r = (Rr)0.70710678118654752440;
    const Rr cs[16] = {1, c1, r, s1, 0, -s1, -r, -c1, -1, -c1, -r, -s1, 0, s1, r, c1};
    const Rr sn[16] = {0, s1, r, c1, 1, c1, r, s1, 0, -s1, -r, -c1, -1, -c1, -r, -s1};
    return mk<T>(cs[j & 15], -sn[j & 15]);
}

template <typename T> __device__ __forceinline__ void dft16(T *v) {
    // 16 = 4 x 4: 4-point DFTs over n2 of x[n1 + 4 n2], twiddle w16^{n1 k1},
    // 4-point DFTs over n1 give X[k1 + 4 k2].
    T a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        T q[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
        dft<T, 4>::run(q);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const int j = n1 * k1;
            if (j == 0) a[n1][k1] = q[k1];
            else if (j == 4) a[n1][k1] = cmuli_neg(q[k1]);
            else a[n1][k1] = cmul(q[k1], w16<T>(j));
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        T q[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        dft<T, 4>::run(q);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = q[k2];
    }
}

// w12^j = exp(-2 pi i j / 12) from sqrt(3)/2 and 1/2
template <typename T> __device__ __forceinline__ T w12(int j) {
    using Rr = typename real_of<T>::type;
    const Rr h = (Rr)0.5, r = (Rr)0.86602540378443864676372317075293618;
    const Rr cs[12] = {1, r, h, 0, -h, -r, -1, -r, -h, 0, h, r};
    const Rr sn[12] = {0, h, r, 1, r, h, 0, -h, -r, -1, -r, -h};
    return mk<T>(cs[j % 12], -sn[j % 12]);
}

// w20^j = exp(-2 pi i j / 20) from the cosines of 18, 36, 54 and 72 degrees
template <typename T> __device__ __forceinline__ T w20(int j) {
    using Rr = typename real_of<T>::type;
    const Rr a = (Rr)0.95105651629515357211643933337938214, b = (Rr)0.80901699437494742410229341718281906,
             c = (Rr)0.58778525229247312916870595463907277, d = (Rr)0.30901699437494742410229341718281906;
    const Rr cs[20] = {1, a, b, c, d, 0, -d, -c, -b, -a, -1, -a, -b, -c, -d, 0, d, c, b, a};
    const Rr sn[20] = {0, d, c, b, a, 1, a, b, c, d, 0, -d, -c, -b, -a, -1, -a, -b, -c, -d};
    return mk<T>(cs[j % 20], -sn[j % 20]);
}

// N = P Q point DFT (N = 12, 20): Q-point DFTs over n2 of x[n1 + P n2],
// twiddle wN^{n1 k1}, P-point DFTs over n1 give X[k1 + Q k2].
template <typename T, int P, int Q> __device__ __forceinline__ void dft_pq(T *v) {
    constexpr int N = P * Q;
    static_assert(N == 12 || N == 20, "twiddle table");
    T a[P][Q];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
        T q[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) q[n2] = v[n1 + P * n2];
        dft<T, Q>::run(q);
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) {
            const int j = n1 * k1;
            if (j == 0) a[n1][k1] = q[k1];
            else a[n1][k1] = cmul(q[k1], N == 12 ? w12<T>(j) : w20<T>(j));
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
        T q[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) q[n1] = a[n1][k1];
        dft<T, P>::run(q);
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) v[k1 + Q * k2] = q[k2];
    }
}

template <typename T, int R> __device__ __forceinline__ void dftR(T *v) {
    if constexpr (R == 16) dft16(v);
    else if constexpr (R == 12) dft_pq<T, 4, 3>(v);
    else if constexpr (R == 20) dft_pq<T, 4, 5>(v);
    else dft<T, R>::run(v);
}

template <typename T, int N1, int N2>
__device__ __forceinline__ void dif_a(T *line, int es, int t, const T *tw) {
    T v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = line[(t + N2 * q) * es];
    dftR<T, N1>(v);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) line[(t + N2 * k1) * es] = v[k1];
}

template <typename T, int N1, int N2> __device__ __forceinline__ void dif_b(T *line, int es, int k1) {
    T v[N2];
#pragma unroll
    for (int t = 0; t < N2; ++t) v[t] = line[(N2 * k1 + t) * es];
    dftR<T, N2>(v);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) line[(N2 * k1 + k2) * es] = v[k2];
}

template <typename T, int N1, int N2>
__device__ __forceinline__ void dit_a(T *line, int es, int j1, const T *tw) {
    T v[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) v[j2] = line[(N2 * j1 + j2) * es];
    dftR<T, N2>(v);
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw[j1 * k2]);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) line[(N2 * j1 + k2) * es] = v[k2];
}

template <typename T, int N1, int N2> __device__ __forceinline__ void dit_b(T *line, int es, int k2) {
    T v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = line[(N2 * j1 + k2) * es];
    dftR<T, N1>(v);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) line[(N2 * k1 + k2) * es] = v[k1];
}

// grid index held by slot p after a DIF, and the slot of grid index k
template <int N1, int N2> __device__ __forceinline__ int slot_index(int p) { return p / N2 + N1 * (p % N2); }
template <int N1, int N2> __device__ __forceinline__ int index_slot(int k) { return N2 * (k % N1) + k / N1; }

// Point injections one (moment, plane) work item can hold.
constexpr int kMaxItemInj = 16;

// Arguments of the fused plane kernel.
template <typename R> struct PlaneArgs {
    using T = typename cvec<R>::type;
    int nz, M;
    R coefD, a, coefS;
    const T *twx, *twy;
    const R *kx, *ky;
    const typename Media4<R>::type *med;
    // damping D_l = mu_a + mu_s (1 - g^l) of each l and z plane in the order
    // X2 reads it: [l][z][x slot][y slot]
    const R *dl_slot;
    const int *lof;
    const CouplingRow *coup;
    const int *step;
    int ndet;
    const int4 *det;
    double *det_out;
    int ninj;
    const int4 *inj;
    const R *inj_amp;
    T *rec_out;
    // adjoint step: gradient terms grad_scale * w_l Re(conj(lambda) psi_n)
    // added to grad_a, and times (1 - g^l) on interior voxels to grad_s
    const T *rec_in;       // psi_n in real space [M][V], or null
    double *grad_a, *grad_s;
    R grad_scale;
    const R *wl;           // w_l per stored moment
    const R *gfac;         // [l-1][z][x slot][y slot]: interior (1 - g^l), l >= 1
};

// Couplings of one output moment grouped by kind (Eq. 10 in mixed space):
// z terms multiply Dz, p terms (i kx + ky) psi~, q terms (i kx - ky) psi~.
// Unused slots have coefficient 0 and point at the moment itself.
template <typename R> struct CouplingKinds {
    int zs[2], ps[2], qs[2];
    int pm[2], qm[2];      // 1: read conj(psi~(-kx, -ky)) (real-radiance layout)
    R zc[2], pc[2], qc[2];
};

template <typename R> __device__ void split_coupling(const CouplingRow &cr, int m, CouplingKinds<R> &k) {
    int nz = 0, np = 0, nq = 0;
    for (int j = 0; j < 2; ++j) {
        k.zs[j] = k.ps[j] = k.qs[j] = m;
        k.pm[j] = k.qm[j] = 0;
        k.zc[j] = k.pc[j] = k.qc[j] = R(0);
    }
    for (int t = 0; t < cr.n; ++t) {
        const int ty = cr.type[t];
        if (ty == 0) { k.zs[nz] = cr.src[t]; k.zc[nz++] = (R)cr.coef[t]; }
        else if (ty == 1 || ty == 3) { k.ps[np] = cr.src[t]; k.pm[np] = ty == 3; k.pc[np++] = (R)cr.coef[t]; }
        else { k.qs[nq] = cr.src[t]; k.qm[nq] = ty == 4; k.qc[nq++] = (R)cr.coef[t]; }
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Persistent CTAs, one per SM (the plane needs most of the shared memory).
// Work item b = z M + m (moment fastest, so that the neighbouring moments
// read by the coupling are in L2 together); CTA i takes b = i, i + G, ...
// and, while it works on b, asks L2 for the psi~ and Dz planes item b + G
// will read. Per item, with the plane in shared memory between phases:
//   Y1  inverse y, DIF phase A, read straight from global memory
//   Y2  inverse y, DIF phase B
//   X1  inverse x, DIF phase A
//   X2  inverse x DIF phase B -> real psi of 8 (or 4) voxels in registers ->
//       readouts, inc = coefD D_l psi + injections -> forward x DIT phase A
//       on the same slots
//   X3  forward x, DIT phase B
//   Y3  forward y, DIT phase A
//   Y4  forward y, DIT phase B -> F_xy[inc] in registers ->
//       out = a psi~ + F_xy[inc] + coefS S~(psi~, Dz), written to global memory.
template <typename R, int NX1, int NX2, int NY1, int NY2, int NT>
__global__ void __launch_bounds__(NT, 1)
    k_plane(const typename cvec<R>::type *__restrict__ psi_in, const typename cvec<R>::type *__restrict__ dz,
            typename cvec<R>::type *__restrict__ out, PlaneArgs<R> pa) {
    using T = typename cvec<R>::type;
    constexpr int NX = NX1 * NX2, NY = NY1 * NY2, P = NX + 1;
    constexpr int NE = NX * NY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    T *twx = s + NY * P;
    T *twy = twx + NX;
    __shared__ CouplingKinds<R> ck;
    __shared__ int step_s, ninj_item;
    __shared__ int inj_x[kMaxItemInj], inj_y[kMaxItemInj];
    __shared__ R inj_a[kMaxItemInj];
    const int tid = threadIdx.x;
    const int M = pa.M;
    const int nitems = M * pa.nz;
    const size_t V = (size_t)pa.nz * NE;
    for (int i = tid; i < NX; i += NT) twx[i] = pa.twx[i];
    for (int i = tid; i < NY; i += NT) twy[i] = pa.twy[i];
    if (tid == 0) step_s = pa.step ? *pa.step : 0;
    __syncthreads();   // twiddle tables are read by every phase, the first one included
    const R inv = R(1) / R(NE);
    constexpr int NY1T = (NX * NY2 + NT - 1) / NT;   // Y1 tasks per thread
    // The first Y1 task's operands of the next item are loaded into registers
    // while the current item finishes (software pipelining across items);
    // further tasks (planes of more than NT x NY1 elements) load at Y1. Holding
    // all of them would need 2 NY1T NY1 registers and spill at 128 x 128.
    T y1[NY1];
    auto load_y1 = [&](int item) {
        const int mi = item % M;
        const T *sp = psi_in + (size_t)mi * V + (size_t)(item / M) * NE;
        const int w = tid;
        if (w < NX * NY2) {
            const int x = w % NX, t = w / NX;
#pragma unroll
            for (int q = 0; q < NY1; ++q) y1[q] = sp[(t + NY2 * q) * NX + x];
        }
    };
    if ((int)blockIdx.x < nitems) load_y1(blockIdx.x);
    for (int b = blockIdx.x; b < nitems; b += gridDim.x) {
        const int m = b % M, z = b / M;
        const size_t zoff = (size_t)z * NE;
        if (tid == 0) {
            split_coupling<R>(pa.coup[m], m, ck);
            int n = 0;
            for (int q = 0; q < pa.ninj && n < kMaxItemInj; ++q) {
                const int4 pt = pa.inj[q];
                if (pt.w == m && pt.z == z) {
                    inj_x[n] = pt.x;
                    inj_y[n] = pt.y;
                    inj_a[n] = pa.inj_amp[(size_t)step_s * pa.ninj + q];
                    ++n;
                }
            }
            ninj_item = n;
            // the coupling of this item reads up to two Dz planes: ask L2 for them now
            const CouplingRow &cr = pa.coup[m];
            for (int t = 0; t < cr.n; ++t)
                if (cr.type[t] == 0) prefetch_l2(dz + (size_t)cr.src[t] * V + zoff, NE * sizeof(T));
            const int nb = b + gridDim.x;
            if (nb < nitems) {
                const int m2 = nb % M;
                const size_t z2 = (size_t)(nb / M) * NE;
                prefetch_l2(psi_in + (size_t)m2 * V + z2, NE * sizeof(T));
            }
        }
        // Y1: column x, rows t + NY2 q, conjugated (F^-1 = conj F conj / n)
#pragma unroll
        for (int h = 0; h < NY1T; ++h) {
            const int w = tid + h * NT;
            if (w < NX * NY2) {
                const int x = w % NX, t = w / NX;
                T v[NY1];
                if (h == 0) {
#pragma unroll
                    for (int q = 0; q < NY1; ++q) v[q] = cconj(y1[q]);
                } else {
                    const T *sp = psi_in + (size_t)m * V + zoff;
#pragma unroll
                    for (int q = 0; q < NY1; ++q) v[q] = cconj(sp[(t + NY2 * q) * NX + x]);
                }
                dftR<T, NY1>(v);
#pragma unroll
                for (int k1 = 1; k1 < NY1; ++k1) v[k1] = cmul(v[k1], twy[t * k1]);
#pragma unroll
                for (int k1 = 0; k1 < NY1; ++k1) s[(t + NY2 * k1) * P + x] = v[k1];
            }
        }
        __syncthreads();
        for (int w = tid; w < NX * NY1; w += NT) dif_b<T, NY1, NY2>(s + (w % NX), P, w / NX);
        __syncthreads();
        for (int w = tid; w < NY * NX2; w += NT) dif_a<T, NX1, NX2>(s + (w % NY) * P, 1, w / NY, twx);
        __syncthreads();
        // X2: row slot py (real y), block k1 of NX2 slots (real x = k1 + NX1 k2)
        const int l = pa.lof[m];
        for (int w = tid; w < NY * NX1; w += NT) {
            const int py = w % NY, k1 = w / NY;
            const int y = slot_index<NY1, NY2>(py);
            T *line = s + py * P + NX2 * k1;
            T v[NX2];
            R dl[NX2];
            const size_t rowv = zoff + (size_t)y * NX;
            const R *dsrc = pa.dl_slot + (size_t)l * V + zoff + py;
#pragma unroll
            for (int k2 = 0; k2 < NX2; ++k2) dl[k2] = dsrc[(size_t)(NX2 * k1 + k2) * NY];
#pragma unroll
            for (int t = 0; t < NX2; ++t) v[t] = line[t];
            dftR<T, NX2>(v);
#pragma unroll
            for (int k2 = 0; k2 < NX2; ++k2) {
                const int x = k1 + NX1 * k2;
                const T p = mk<T>(v[k2].x * inv, -v[k2].y * inv);
                if (pa.rec_out) pa.rec_out[(size_t)m * V + rowv + x] = p;
                if (pa.rec_in) {
                    const T ps = pa.rec_in[(size_t)m * V + rowv + x];
                    const double pr = (double)pa.grad_scale * (double)pa.wl[m] * ((double)p.x * ps.x + (double)p.y * ps.y);
                    atomicAdd(pa.grad_a + rowv + x, pr);
                    if (l > 0)
                        atomicAdd(pa.grad_s + rowv + x,
                                  pr * (double)pa.gfac[(size_t)(l - 1) * V + zoff + py + (size_t)(NX2 * k1 + k2) * NY]);
                }
                v[k2] = cscale(p, pa.coefD * dl[k2]);
            }
            dftR<T, NX2>(v);
#pragma unroll
            for (int k2 = 1; k2 < NX2; ++k2) v[k2] = cmul(v[k2], twx[k1 * k2]);
#pragma unroll
            for (int k2 = 0; k2 < NX2; ++k2) line[k2] = v[k2];
        }
        __syncthreads();
        for (int w = tid; w < NY * NX2; w += NT) dit_b<T, NX1, NX2>(s + (w % NY) * P, 1, w / NY);
        __syncthreads();
        for (int w = tid; w < NX * NY1; w += NT) dit_a<T, NY1, NY2>(s + (w % NX), P, w / NX, twy);
        __syncthreads();
        // Y4: column kx, outputs ky = k2 + NY2 k1; coupling and update. The
        // operands of output pair c0 + 2 are loaded while pair c0 is computed.
        T *dst = out + (size_t)m * V + zoff;
        const CouplingKinds<R> k = ck;
        const T zero = czero<T>();
        const T *bz0 = dz + (size_t)k.zs[0] * V + zoff, *bz1 = dz + (size_t)k.zs[1] * V + zoff;
        const T *bp0 = psi_in + (size_t)k.ps[0] * V + zoff, *bp1 = psi_in + (size_t)k.ps[1] * V + zoff;
        const T *bq0 = psi_in + (size_t)k.qs[0] * V + zoff, *bq1 = psi_in + (size_t)k.qs[1] * V + zoff;
        const T *bs = psi_in + (size_t)m * V + zoff;
        for (int w = tid; w < NX * NY2; w += NT) {
            const int kx = w % NX, k2 = w / NX;
            constexpr int U = NY1 > 16 ? 1 : 2;   // operand double buffer within 128 registers
            T op[2][7][U];
            auto load_ops = [&](int slot, int c0) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ky = k2 + NY2 * (c0 + u);
                    const int e = ky * NX + kx;
                    const int em = ((NY - ky) % NY) * NX + (NX - kx) % NX;   // (-kx, -ky)
                    op[slot][0][u] = bs[e];
                    op[slot][1][u] = k.zc[0] != R(0) ? bz0[e] : zero;
                    op[slot][2][u] = k.zc[1] != R(0) ? bz1[e] : zero;
                    op[slot][3][u] = k.pc[0] != R(0) ? bp0[k.pm[0] ? em : e] : zero;
                    op[slot][4][u] = k.pc[1] != R(0) ? bp1[k.pm[1] ? em : e] : zero;
                    op[slot][5][u] = k.qc[0] != R(0) ? bq0[k.qm[0] ? em : e] : zero;
                    op[slot][6][u] = k.qc[1] != R(0) ? bq1[k.qm[1] ? em : e] : zero;
                }
            };
            load_ops(0, 0);
            T v[NY1];
#pragma unroll
            for (int j1 = 0; j1 < NY1; ++j1) v[j1] = s[(NY2 * j1 + k2) * P + kx];
            dftR<T, NY1>(v);
            // point injections enter as the DFT of a delta: a w_NX^{kx x} w_NY^{ky y}
            for (int q = 0; q < ninj_item; ++q) {
                const T ex = twx[(kx * inj_x[q]) % NX];
                const R a = inj_a[q];
#pragma unroll
                for (int k1 = 0; k1 < NY1; ++k1) {
                    const T ph = cmul(ex, twy[((k2 + NY2 * k1) * inj_y[q]) % NY]);
                    v[k1].x += a * ph.x;
                    v[k1].y += a * ph.y;
                }
            }
            const R kxv = pa.kx[kx];
            // conj of a mirrored operand flips its imaginary part: fold into the coefficient
            const R pcy0 = k.pm[0] ? -k.pc[0] : k.pc[0], pcy1 = k.pm[1] ? -k.pc[1] : k.pc[1];
            const R qcy0 = k.qm[0] ? -k.qc[0] : k.qc[0], qcy1 = k.qm[1] ? -k.qc[1] : k.qc[1];
#pragma unroll
            for (int c0 = 0; c0 < NY1; c0 += U) {
                const int cur = (c0 / U) & 1;
                if (c0 + U < NY1) load_ops(cur ^ 1, c0 + U);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ky = k2 + NY2 * (c0 + u);
                    const R kyv = pa.ky[ky];
                    const T p0 = op[cur][3][u], p1 = op[cur][4][u], q0 = op[cur][5][u], q1 = op[cur][6][u];
                    const T z0 = op[cur][1][u], z1 = op[cur][2][u], self = op[cur][0][u];
                    const R zr = k.zc[0] * z0.x + k.zc[1] * z1.x, zi = k.zc[0] * z0.y + k.zc[1] * z1.y;
                    const R pr = k.pc[0] * p0.x + k.pc[1] * p1.x, pi = pcy0 * p0.y + pcy1 * p1.y;
                    const R qr = k.qc[0] * q0.x + k.qc[1] * q1.x, qi = qcy0 * q0.y + qcy1 * q1.y;
                    // S = Z + (i kx + ky) P + (i kx - ky) Q
                    const R sr = zr + kyv * (pr - qr) - kxv * (pi + qi);
                    const R si = zi + kxv * (pr + qr) + kyv * (pi - qi);
                    const T f = v[c0 + u];
                    dst[(size_t)ky * NX + kx] =
                        mk<T>(pa.a * self.x + f.x + pa.coefS * sr, pa.a * self.y + f.y + pa.coefS * si);
                }
            }
        }
        if (b + (int)gridDim.x < nitems) load_y1(b + gridDim.x);
        __syncthreads();   // the next item reuses the shared plane and ck
    }
}

// Readouts Re psi_00 at detector voxels of the state psi~ (before a step):
// psi(x, y, z) = (1/(nx ny)) sum_{kx, ky} psi~(kx, ky, z) w^{-(kx x + ky y)}.
// Grid (ndet, kTapChunks): CTA (d, c) sums rows ky = c, c + kTapChunks, ...
// in FP64 and writes one partial sum; k_taps_finish adds the partials of each
// detector in a fixed order.
constexpr int kTapChunks = 16;

template <typename R>
__global__ void k_taps(const typename cvec<R>::type *__restrict__ psi_t, int nx, int ny,
                       const typename cvec<R>::type *__restrict__ twx, const typename cvec<R>::type *__restrict__ twy,
                       const int4 *__restrict__ det, double *__restrict__ part) {
    using T = typename cvec<R>::type;
    const int d = blockIdx.x, c = blockIdx.y;
    const int4 q = det[d];
    const T *plane = psi_t + (size_t)q.z * ny * nx;
    double acc = 0.0;
    for (int ky = c; ky < ny; ky += kTapChunks) {
        const T b = twy[(int)(((long)ky * q.y) % ny)];
        for (int kx = threadIdx.x; kx < nx; kx += blockDim.x) {
            const T a = twx[(int)(((long)kx * q.x) % nx)];
            // w^{-j} = conj(w^j)
            const double cr = (double)a.x * b.x - (double)a.y * b.y, ci = -((double)a.x * b.y + (double)a.y * b.x);
            const T v = plane[(size_t)ky * nx + kx];
            acc += (double)v.x * cr - (double)v.y * ci;
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        part[(size_t)d * kTapChunks + c] = sum;
    }
}

static __global__ void k_taps_finish(const double *__restrict__ part, int ndet, double scale, const int *__restrict__ step,
                              double *det_out) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndet) return;
    double s = 0.0;
    for (int c = 0; c < kTapChunks; ++c) s += part[(size_t)d * kTapChunks + c];
    det_out[(size_t)(*step) * ndet + d] = s * scale;
}

// Z pass for a fixed nz = N1 N2: Dz = F_z^-1[i kz F_z psi~] for a tile of TX
// consecutive kx columns of one (moment, ky), with two shared-memory round
// trips:
//   A  DIF phase A read straight from global memory (rows t + N2 q)
//   B  DIF phase B, times conj(i kz / nz), DIT phase A, all on the same
//      N2-slot block of one thread (slot N2 k1 + k2 holds kz index k1 + N1 k2)
//   C  DIT phase B, written straight to global memory in natural order
// The inverse is taken as conj(F conj(.)): B conjugates, C conjugates back.
template <typename R, int N1, int N2, int TX, int NT>
__global__ void __launch_bounds__(NT)
    k_zderiv_fixed(const typename cvec<R>::type *__restrict__ in, typename cvec<R>::type *__restrict__ out,
                   Geo<R> g) {
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
    // A: column b, rows t + N2 q
    for (int w = tid; w < TX * N2; w += NT) {
        const int b = w % TX, t = w / TX;
        const bool ok = x0 + b < g.nx;
        T v[N1];
#pragma unroll
        for (int q = 0; q < N1; ++q) v[q] = ok ? in[base + (size_t)(t + N2 * q) * plane + b] : czero<T>();
        dftR<T, N1>(v);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) s[(t + N2 * k1) * P + b] = v[k1];
    }
    __syncthreads();
    // B: block N2 k1 of column b
    const R inv = R(1) / R(NZ);
    for (int w = tid; w < TX * N1; w += NT) {
        const int b = w % TX, k1 = w / TX;
        T v[N2];
#pragma unroll
        for (int t = 0; t < N2; ++t) v[t] = s[(N2 * k1 + t) * P + b];
        dftR<T, N2>(v);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const R k = g.kz[k1 + N1 * k2] * inv;
            v[k2] = mk<T>(-k * v[k2].y, -k * v[k2].x);   // conj(i k v)
        }
        dftR<T, N2>(v);
#pragma unroll
        for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw[k1 * k2]);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) s[(N2 * k1 + k2) * P + b] = v[k2];
    }
    __syncthreads();
    // C: slots N2 j1 + k2 of column b -> z index k2 + N2 k1
    for (int w = tid; w < TX * N2; w += NT) {
        const int b = w % TX, k2 = w / TX;
        if (x0 + b >= g.nx) continue;
        T v[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) v[j1] = s[(N2 * j1 + k2) * P + b];
        dftR<T, N1>(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) out[base + (size_t)(k2 + N2 * k1) * plane + b] = cconj(v[k1]);
    }
}


// ---------------------------------------------------------------- fixed-size line passes
// The split schedule's Y and X passes for a fixed axis n = N1 N2, used where
// the fused plane kernel does not fit (planes of 256 points, FP64 planes
// over 200 KB). In-place two-phase transforms as above; a transform whose
// output is written straight from the DIF phase B lands in natural order by
// the slot map (slot N2 k1 + k2 holds index k1 + N1 k2).

// Y pass: one CTA per (moment, TX columns, z), the moment fastest so that
// the CTAs reading each other's tiles as coupling operands run together.
// COUPLE = 0: out = F_y^-1 in (inverse) or F_y in; COUPLE = 1: out =
// a psi_in + F_y in + coefS * S~(psi_in, dz) (Eq. 10 in mixed space, as
// k_ypass). in and out may alias (the tile is read before any write).
template <typename R, int N1, int N2, int TX, int NT, int COUPLE>
__global__ void __launch_bounds__(NT, 2048 / NT / 2)
    k_ypass_fixed(const typename cvec<R>::type *in, typename cvec<R>::type *out, Geo<R> g, int inverse,
                  const typename cvec<R>::type *__restrict__ psi_in, const typename cvec<R>::type *__restrict__ dz,
                  R a, R coefS, const CouplingRow *__restrict__ coup) {
    using T = typename cvec<R>::type;
    constexpr int NY = N1 * N2, P = TX + 1;
    __shared__ T s[NY * P];
    __shared__ T tw[NY];
    const int m = blockIdx.x, x0 = blockIdx.y * TX, z = blockIdx.z;
    const size_t V = (size_t)g.nz * g.ny * g.nx;
    const size_t zoff = (size_t)z * g.ny * g.nx;
    const size_t base = (size_t)m * V + zoff + x0;
    const int tid = threadIdx.x;
    for (int i = tid; i < NY; i += NT) tw[i] = g.twy[i];
    __syncthreads();
    // A: column b, rows t + N2 q (conjugated for the inverse)
    for (int w = tid; w < TX * N2; w += NT) {
        const int b = w % TX, t = w / TX;
        const bool ok = x0 + b < g.nx;
        T v[N1];
#pragma unroll
        for (int q = 0; q < N1; ++q) {
            const T u = ok ? in[base + (size_t)(t + N2 * q) * g.nx + b] : czero<T>();
            v[q] = inverse ? cconj(u) : u;
        }
        dftR<T, N1>(v);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) s[(t + N2 * k1) * P + b] = v[k1];
    }
    __syncthreads();
    // B: block N2 k1 of column b -> ky = k1 + N1 k2
    const R inv = R(1) / R(NY);
    if constexpr (!COUPLE) {
        for (int w = tid; w < TX * N1; w += NT) {
            const int b = w % TX, k1 = w / TX;
            T v[N2];
#pragma unroll
            for (int t = 0; t < N2; ++t) v[t] = s[(N2 * k1 + t) * P + b];
            dftR<T, N2>(v);
            if (x0 + b >= g.nx) continue;
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const size_t o = base + (size_t)(k1 + N1 * k2) * g.nx + b;
                out[o] = inverse ? cscale(cconj(v[k2]), inv) : v[k2];
            }
        }
        return;
    } else {
        // forward + coupling, grouped as in the plane kernel: z terms (Dz), p terms
        // (i kx + ky) psi~, q terms (i kx - ky) psi~; mirrored operands (real
        // layout) read conj(psi~(-kx, -ky)), folded into signed coefficients.
        // Phase B writes its outputs back to their slots; the epilogue then takes
        // one output per thread, so that few registers leave room for many warps
        // to cover the operand loads.
        __shared__ CouplingKinds<R> ck;
        if (tid == 0) split_coupling<R>(coup[m], m, ck);
        for (int w = tid; w < TX * N1; w += NT) {
            const int b = w % TX, k1 = w / TX;
            T v[N2];
#pragma unroll
            for (int t = 0; t < N2; ++t) v[t] = s[(N2 * k1 + t) * P + b];
            dftR<T, N2>(v);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) s[(N2 * k1 + k2) * P + b] = v[k2];
        }
        __syncthreads();
        const CouplingKinds<R> &k = ck;   // read from shared memory (uniform across the CTA)
        const R pcy0 = k.pm[0] ? -k.pc[0] : k.pc[0], pcy1 = k.pm[1] ? -k.pc[1] : k.pc[1];
        const R qcy0 = k.qm[0] ? -k.qc[0] : k.qc[0], qcy1 = k.qm[1] ? -k.qc[1] : k.qc[1];
        const T zero = czero<T>();
        const T *bz0 = dz + (size_t)k.zs[0] * V + zoff, *bz1 = dz + (size_t)k.zs[1] * V + zoff;
        const T *bp0 = psi_in + (size_t)k.ps[0] * V + zoff, *bp1 = psi_in + (size_t)k.ps[1] * V + zoff;
        const T *bq0 = psi_in + (size_t)k.qs[0] * V + zoff, *bq1 = psi_in + (size_t)k.qs[1] * V + zoff;
        const T *bs = psi_in + (size_t)m * V + zoff;
        for (int w = tid; w < TX * NY; w += NT) {
            const int b = w % TX, e = w / TX, x = x0 + b;
            if (x >= g.nx) continue;
            const T f = s[index_slot<N1, N2>(e) * P + b];
            const size_t ep = (size_t)e * g.nx + x;
            const size_t em = (size_t)((g.ny - e) % g.ny) * g.nx + (g.nx - x) % g.nx;   // (-kx, -ky)
            const T self = bs[ep];
            const T z0 = k.zc[0] != R(0) ? bz0[ep] : zero, z1 = k.zc[1] != R(0) ? bz1[ep] : zero;
            const T p0 = k.pc[0] != R(0) ? bp0[k.pm[0] ? em : ep] : zero;
            const T p1 = k.pc[1] != R(0) ? bp1[k.pm[1] ? em : ep] : zero;
            const T q0 = k.qc[0] != R(0) ? bq0[k.qm[0] ? em : ep] : zero;
            const T q1 = k.qc[1] != R(0) ? bq1[k.qm[1] ? em : ep] : zero;
            const R kxv = g.kx[x], kyv = g.ky[e];
            const R zr = k.zc[0] * z0.x + k.zc[1] * z1.x, zi = k.zc[0] * z0.y + k.zc[1] * z1.y;
            const R pr = k.pc[0] * p0.x + k.pc[1] * p1.x, pi = pcy0 * p0.y + pcy1 * p1.y;
            const R qr = k.qc[0] * q0.x + k.qc[1] * q1.x, qi = qcy0 * q0.y + qcy1 * q1.y;
            // S = Z + (i kx + ky) P + (i kx - ky) Q
            const R sr = zr + kyv * (pr - qr) - kxv * (pi + qi);
            const R si = zi + kxv * (pr + qr) + kyv * (pi - qi);
            out[base + ep - x0] = mk<T>(a * self.x + f.x + coefS * sr, a * self.y + f.y + coefS * si);
        }
    }
}

// X pass of a step or an operator application (inverse x-DFT, pointwise
// stage, forward x-DFT), one CTA per (row y, z, mcs <= MC moments):
//   A  inverse DIF phase A read straight from global memory
//   B  DIF phase B -> real psi of N2 voxels in registers -> readouts (moment
//      0), record (rec_out), inc = coefD D_l psi + injections -> forward DIT
//      phase A on the same slots
//   C  DIT phase B written straight to global memory
// Adjoint gradient terms are not handled here (k_xpass does them). in and
// out may alias.
template <typename R, int N1, int N2, int MC, int NT>
__global__ void __launch_bounds__(NT, 4)
    k_xpass_fixed(const typename cvec<R>::type *in, typename cvec<R>::type *out, Geo<R> g, int mcs, XArgs<R> xa) {
    using T = typename cvec<R>::type;
    constexpr int NX = N1 * N2;
    // a row keeps one pad slot after every N2 elements (slot i at i + i / N2),
    // so that the lanes of phase B (stride N2 in the row) hit distinct banks
    constexpr int P = NX + NX / N2 + 1;
    extern __shared__ __align__(16) unsigned char xs_raw[];
    T *s = reinterpret_cast<T *>(xs_raw);   // mcs rows of P
    // twiddles laid out for the lanes that read them: twA[k1 N2 + t] =
    // w^{t k1} (phase A, lanes over t), twB[k2 N1 + k1] = w^{k1 k2} (phase B,
    // lanes over k1)
    __shared__ T twA[NX], twB[NX];
    __shared__ int step_s;
    const size_t V = (size_t)g.nz * g.ny * NX;
    const int tid = threadIdx.x, nthr = blockDim.x;   // nthr <= NT: as many threads as tasks
    const int nch = (g.M + mcs - 1) / mcs, nitems = g.ny * g.nz * nch;
    for (int i = tid; i < NX; i += nthr) {
        twA[i] = g.twx[((i / N2) * (i % N2)) % NX];
        twB[i] = g.twx[((i / N1) * (i % N1)) % NX];
    }
    if (tid == 0) step_s = xa.step ? *xa.step : 0;
    __syncthreads();
    const R inv = R(1) / R(NX);
    const int step = step_s;
    auto pad = [](int i) { return i + i / N2; };
    // persistent: items (row y, z, chunk of mcs moments), row fastest
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int y = it % g.ny, z = (it / g.ny) % g.nz, m0 = (it / (g.ny * g.nz)) * mcs;
        const int mc = min(mcs, g.M - m0);
        const size_t row = ((size_t)z * g.ny + y) * NX;
        // A: moment b, x = t + N2 q, conjugated (F^-1 = conj F conj / n)
        for (int w = tid; w < mc * N2; w += nthr) {
            const int b = w / N2, t = w % N2;
            const T *src = in + (size_t)(m0 + b) * V + row;
            T v[N1];
#pragma unroll
            for (int q = 0; q < N1; ++q) v[q] = cconj(src[t + N2 * q]);
            dftR<T, N1>(v);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], twA[k1 * N2 + t]);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) s[b * P + pad(t + N2 * k1)] = v[k1];
        }
        __syncthreads();
        for (int w = tid; w < mc * N1; w += nthr) {
            const int b = w / N1, k1 = w % N1, m = m0 + b;
            const int l = xa.lof[m];
            T v[N2];
#pragma unroll
            for (int t = 0; t < N2; ++t) v[t] = s[b * P + pad(N2 * k1 + t)];
            dftR<T, N2>(v);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int x = k1 + N1 * k2;
                const size_t vx = row + x;
                const T p = mk<T>(v[k2].x * inv, -v[k2].y * inv);
                if (m == 0)
                    for (int d = 0; d < xa.ndet; ++d) {
                        const int4 q = xa.det[d];
                        if (q.x == x && q.y == y && q.z == z) xa.det_out[(size_t)step * xa.ndet + d] = (double)p.x;
                    }
                if (xa.rec_out) xa.rec_out[(size_t)m * V + vx] = p;
                const typename Media4<R>::type md = xa.med[vx];
                R gl = 1;
                for (int q = 0; q < l; ++q) gl *= md.z;
                T inc = cscale(p, xa.coefD * (md.x + md.y * (R(1) - gl)));
                for (int q = 0; q < xa.ninj; ++q) {
                    const int4 pt = xa.inj[q];
                    if (pt.w == m && pt.x == x && pt.y == y && pt.z == z)
                        inc.x += xa.inj_amp[(size_t)step * xa.ninj + q];
                }
                v[k2] = inc;
            }
            dftR<T, N2>(v);
#pragma unroll
            for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], twB[k2 * N1 + k1]);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) s[b * P + pad(N2 * k1 + k2)] = v[k2];
        }
        __syncthreads();
        // C: slots N2 j1 + k2 of moment b -> kx = k2 + N2 k1
        for (int w = tid; w < mc * N2; w += nthr) {
            const int b = w / N2, k2 = w % N2;
            T v[N1];
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) v[j1] = s[b * P + pad(N2 * j1 + k2)];
            dftR<T, N1>(v);
            T *dst = out + (size_t)(m0 + b) * V + row;
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) dst[k2 + N2 * k1] = v[k1];
        }
        __syncthreads();   // the next item reuses s
    }
}

}  // namespace rte
