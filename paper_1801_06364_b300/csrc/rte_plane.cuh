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
#include <cuda.h>
#include "rte_kernels.cuh"

namespace rte {

// cos(2 pi j / 480), j = 0..120: a quarter wave on a grid that every
// in-register DFT length below (12, 16, 20, 24, 32, 40) divides. Values
// computed to 21 digits in multiple precision.
__device__ __forceinline__ double cos480(int j) {
    const double t[121] = {
        1.0, 0.999914327574007032249, 0.999657324975557280037, 0.999229036240722934737, 0.998629534754573873784,
        0.997858923238603506738, 0.996917333733127976198, 0.995804927574661729379, 0.994521895368273336923, 0.993068456954926295637,
        0.991444861373810411145, 0.989651386819670214764, 0.98768834059513772619, 0.985556059058077729491, 0.983254907563954584555,
        0.980785280403230449126, 0.978147600733805637929, 0.975342320508512694867, 0.972369920397676601834, 0.969230909706754393016,
        0.96592582628906828675, 0.96245523645364728763, 0.958819734868193049761, 0.955019944457186627432, 0.951056516295153572116,
        0.946930129495105664256, 0.942641491092178394777, 0.938191335922484134452, 0.93358042649720174899, 0.928809552871924233956,
        0.923879532511286756128, 0.918791210148898296585, 0.913545457642600895502, 0.908143173825081299258, 0.902585284349860606763,
        0.896872741532688303894, 0.89100652418836786236, 0.884987637463041862073, 0.87881711266196537413, 0.872496007072797114525,
        0.866025403784438646764, 0.859406411501452674335, 0.852640164354092221519, 0.845727821703973253052, 0.838670567945424029638,
        0.831469612302545237079, 0.82412618862201566173, 0.816641555161678913944, 0.809016994374947424102, 0.801253812691060652479,
        0.79335334029123516458, 0.78531693088074492747, 0.77714596145697087998, 0.768841832073459520277, 0.760405965600030938175,
        0.751839807478977396408, 0.743144825477394235015, 0.734322509435685535636, 0.725374371012287637993, 0.716301943424654248861,
        0.707106781186547524401, 0.697790459841680139672, 0.688354575693753984389, 0.678800745532941741394, 0.669130606358858213826,
        0.659345815100068868425, 0.649448048330183655726, 0.639439001980584753023, 0.629320391049837452706, 0.619093949309833986942,
        0.608761429008720639416, 0.59832460057065904607, 0.587785252292473129169, 0.577145190037233642703, 0.566406236924832831822,
        0.555570233019602224743, 0.544639035015027082224, 0.533614515915611527147, 0.522498564715948864988, 0.511293086077052084829,
        0.5, 0.48862124149695494742, 0.477158760259608415049, 0.46561452032511140759, 0.45399049973954679156,
        0.442288690219001281995, 0.430511096808295144376, 0.418659737537428086676, 0.406736643075800207754, 0.394743856384267249568,
        0.382683432365089771728, 0.370557437509836227823, 0.358367949545300273484, 0.346117057077492976468, 0.333806859233770928828,
        0.321439465303161580701, 0.309016994374947424102, 0.296541574975570953473, 0.284015344703922617444, 0.271440449865074253344,
        0.258819045102520762349, 0.246153293028993038769, 0.233445363855905411768, 0.220697435021501091796, 0.207911690817759337102,
        0.195090322016128267848, 0.182235525492147456603, 0.169349503849024614175, 0.15643446504023086901, 0.143492621991179306485,
        0.130526192220051591548, 0.117537397457837644106, 0.1045284632676534714, 0.091501618663402385314, 0.078459095727844945033,
        0.0654031292301430668153, 0.0523359562429438327221, 0.0392598157590686090208, 0.0261769483078731526106, 0.0130895955713444401903,
        0.0};
    return t[j];
}

// v * w_N^j, w_N = exp(-2 pi i / N), for a j known at compile time (every
// caller's loops are unrolled). Multiples of an eighth turn use exact forms;
// the rest take cos and sin from the quarter-wave table. N is a multiple of 4.
template <typename T, int N> __device__ __forceinline__ T twmul(T v, int j) {
    using Rr = typename real_of<T>::type;
    j = ((j % N) + N) % N;
    if (j == 0) return v;
    if ((8 * j) % N == 0) {
        const Rr h = (Rr)0.70710678118654752440084436210484904;   // 1/sqrt(2)
        switch (8 * j / N) {
            case 1: return mk<T>((v.x + v.y) * h, (v.y - v.x) * h);
            case 2: return mk<T>(v.y, -v.x);
            case 3: return mk<T>((v.y - v.x) * h, -(v.x + v.y) * h);
            case 4: return mk<T>(-v.x, -v.y);
            case 5: return mk<T>(-(v.x + v.y) * h, (v.x - v.y) * h);
            case 6: return mk<T>(-v.y, v.x);
            default: return mk<T>((v.x - v.y) * h, (v.x + v.y) * h);
        }
    }
    constexpr int Q = N / 4;
    const int q = j / Q, r = j % Q;
    const double c0 = cos480(r * (480 / N)), s0 = cos480((Q - r) * (480 / N));
    const double c = q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;   // cos(2 pi j / N)
    const double s = q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;   // sin(2 pi j / N)
    const Rr cr = (Rr)c, sr = (Rr)s;
    return mk<T>(v.x * cr + v.y * sr, v.y * cr - v.x * sr);   // v (c - i s)
}

template <typename T, int R> __device__ __forceinline__ void dftR(T *v);

// N = P Q point DFT in registers: Q-point DFTs over n2 of x[n1 + P n2],
// twiddle w_N^{n1 k1}, then P-point DFTs over n1 give X[k1 + Q k2]
// (n k = n1 k1 + Q n1 k2 + P n2 k1 mod N).
template <typename T, int P, int Q> __device__ __forceinline__ void dft_comp(T *v) {
    constexpr int N = P * Q;
    T a[P][Q];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
        T q[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) q[n2] = v[n1 + P * n2];
        dftR<T, Q>(q);
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) a[n1][k1] = twmul<T, N>(q[k1], n1 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
        T q[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) q[n1] = a[n1][k1];
        dftR<T, P>(q);
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) v[k1 + Q * k2] = q[k2];
    }
}

// forward R-point DFT in place, R in {2, 3, 4, 5, 8, 12, 16, 20, 24, 32, 40}
template <typename T, int R> __device__ __forceinline__ void dftR(T *v) {
    if constexpr (R == 12) dft_comp<T, 4, 3>(v);
    else if constexpr (R == 16) dft_comp<T, 4, 4>(v);
    else if constexpr (R == 20) dft_comp<T, 4, 5>(v);
    else if constexpr (R == 24) dft_comp<T, 3, 8>(v);
    else if constexpr (R == 32) dft_comp<T, 4, 8>(v);
    else if constexpr (R == 40) dft_comp<T, 5, 8>(v);
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

// Plans one launch of the step kernels advances together (same grid, order,
// precision and layout; their own media, sources, states and dt).
constexpr int kMaxGroup = 8;

// What the plane kernel needs of one plan of the group.
template <typename R> struct PlanePlan {
    using T = typename cvec<R>::type;
    // psi_in as a 2-D array of rows ([M][nz][ny] rows of nx elements, in
    // 8-byte units), read by TMA in boxes of 8 rows that are as wide as the
    // shared-memory row pitch (the columns past a row's end lie outside the
    // array and arrive as zeros); filled in at launch
    CUtensorMap rows_map;
    const T *psi_in;       // psi~ the step starts from
    const T *win;          // w = a psi~ + coefS S~ from k_zstream
    T *out;                // psi~ after the step
    // damping D_l = mu_a + mu_s (1 - g^l) of each l and z plane in the order
    // the X2 phase reads it: [l][z][x slot][y slot]
    const R *dl_slot;
    R coefD;
    int ninj;              // point injections amp[step * ninj + i] into moment inj.w at (x, y, z)
    const int4 *inj;
    const R *inj_amp;
    const int *step;       // device step counter (injections)
    int *nonfinite;        // see Geo::nonfinite (null: not checked)
    int *status;           // set to 1 when a bulk copy did not complete in time
};

// Arguments of the fused plane kernel.
template <typename R> struct PlaneArgs {
    using T = typename cvec<R>::type;
    int nz, M, nplans;
    const T *twx, *twy;
    const int *lof;
    PlanePlan<R> pl[kMaxGroup];
    // adjoint (single plan): record of the real-space psi, or gradient terms
    // grad_scale * w_l Re(conj(lambda) psi_n) added to grad_a, and times
    // (1 - g^l) on interior voxels to grad_s
    T *rec_out;
    const T *rec_in;       // psi_n in real space [M][V], or null
    double *grad_a, *grad_s;
    R grad_scale;
    const R *wl;           // w_l per stored moment
    const R *gfac;         // [l-1][z][x slot][y slot]: interior (1 - g^l), l >= 1
    // host side: coefficients of the z-streaming pass and the readouts
    R a, coefS;
    int ndet;
    const int4 *det;
    double *det_out;
};

// Arguments of the z-streaming kernel for a group of plans.
template <typename R> struct ZArgs {
    using T = typename cvec<R>::type;
    int nplans, nxt;       // plans, x tiles per plan
    const T *in[kMaxGroup];
    T *out[kMaxGroup];
    R a[kMaxGroup], coefS[kMaxGroup];
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

// ---------------------------------------------------------------- bulk copies and mbarriers
// Global -> shared copies by the bulk-copy (TMA) engine complete on an
// mbarrier in shared memory: one thread arrives on the barrier announcing the
// bytes to expect, the copies count them down, and the phase completes when
// both are done. Waits are bounded (kWaitTests tests of the phase); a wait
// that runs out reports false and the caller records the failure and returns.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the bulk-copy engine
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival on the current phase, which then also waits for `bytes` of copies
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

constexpr unsigned kWaitTests = 1u << 24;

// wait until the phase with the given parity has completed; false if it did
// not within kWaitTests tests
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    for (unsigned i = 0; i < kWaitTests; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, counted on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 2-D tensor copy (TMA) of one box at coordinates (x, y) of the tensor map
// `map` (a kernel parameter) into this CTA's shared memory (128-byte aligned),
// counted on `bar`
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// rows of the plane kernel's psi~ plane per tensor copy
constexpr int kRowsPerCopy = 8;

// order this thread's shared-memory accesses before later bulk-copy accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Row pitch of the plane tile in shared memory: with 8-byte elements an even
// pitch keeps rows 16-byte aligned for the vector accesses of the X2 phase
// (rows 8 lanes apart then fall 16 bytes apart in the banks); with 16-byte
// elements an odd pitch does the same.
template <typename R, int NX> __host__ __device__ constexpr int plane_pitch() { return sizeof(R) == 4 ? NX + 2 : NX + 1; }

// y split of the plane kernel: n = (n / SY) * SY
__host__ __device__ constexpr int plane_sy(int ny) { return ny >= 64 ? 8 : 4; }

// Shared memory of the plane kernel: the plane, six twiddle tables, three
// mbarriers and, where it fits in 220 KB, a staging buffer that holds the
// item's D_l plane up to the X2 phase and the first rows of its w plane after.
template <typename R> __host__ __device__ constexpr size_t plane_smem_core(int nx, int ny) {
    return ((size_t)ny * (sizeof(R) == 4 ? nx + 2 : nx + 1) + 3 * (size_t)nx + 3 * (size_t)ny) * 2 * sizeof(R) + 32;
}
template <typename R> __host__ __device__ constexpr bool plane_dl_staged(int nx, int ny) {
    return plane_smem_core<R>(nx, ny) + (size_t)nx * ny * sizeof(R) <= 220 * 1024;
}
template <typename R> __host__ __device__ constexpr size_t plane_smem_bytes(int nx, int ny) {
    return plane_smem_core<R>(nx, ny) + (plane_dl_staged<R>(nx, ny) ? (size_t)nx * ny * sizeof(R) : 0);
}
// Rows of w the staging buffer takes (a multiple of the y split, at most ny):
// as many as fit beside the plane, the twiddles and the barriers in the CTA's
// share of 220 KB (minb CTAs per SM); none where D_l is not staged.
template <typename R> __host__ __device__ constexpr int plane_w_rows(int nx, int ny, int minb) {
    if (!plane_dl_staged<R>(nx, ny)) return 0;
    const size_t budget = (size_t)220 * 1024 / minb, core = plane_smem_core<R>(nx, ny);
    if (budget <= core) return 0;
    const int sy = plane_sy(ny);
    const int rows = (int)((budget - core) / ((size_t)nx * 2 * sizeof(R))) / sy * sy;
    return rows < ny ? rows : ny;
}
// bytes of the staging buffer, and the kernel's shared memory in all
template <typename R> __host__ __device__ constexpr size_t plane_stage_bytes(int nx, int ny, int minb) {
    const size_t dl = plane_dl_staged<R>(nx, ny) ? (size_t)nx * ny * sizeof(R) : 0;
    const size_t wb = (size_t)plane_w_rows<R>(nx, ny, minb) * nx * 2 * sizeof(R);
    return dl > wb ? dl : wb;
}
template <typename R> __host__ __device__ constexpr size_t plane_smem_launch(int nx, int ny, int minb) {
    return plane_smem_core<R>(nx, ny) + plane_stage_bytes<R>(nx, ny, minb);
}

// L consecutive complex values of a shared-memory row, 16 bytes per access
template <typename T, int L> __device__ __forceinline__ void row_load(const T *src, T *v) {
    if constexpr (sizeof(T) == 8 && L % 2 == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int i = 0; i < L / 2; ++i) {
            const float4 q = s4[i];
            v[2 * i] = mk<T>(q.x, q.y);
            v[2 * i + 1] = mk<T>(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < L; ++i) v[i] = src[i];
    }
}
template <typename T, int L> __device__ __forceinline__ void row_store(T *dst, const T *v) {
    if constexpr (sizeof(T) == 8 && L % 2 == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int i = 0; i < L / 2; ++i) d4[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
    } else {
#pragma unroll
        for (int i = 0; i < L; ++i) dst[i] = v[i];
    }
}

// Fused per-plane pass of the step (paper stages 1-3 for one moment and one
// z plane): out = w + F_xy[coefD D_l F_xy^-1 psi~ + injections], where w
// (from k_zstream) already holds a psi~ + coefS S~.
//
// Persistent CTAs; work item b = z M + m (moment fastest), CTA i takes
// b = i, i + G, ... Both axes are split so that the middle phases of the two
// transforms meet in one shared-memory round trip:
//   y: n = BY * SY (DIF: BY-point DFTs, then SY-point; DIT the reverse)
//   x: n = 4 * BX  (DIF: 4-point DFTs, then BX-point; DIT the reverse)
// The psi~ plane of an item arrives in shared memory by 2-D tensor copies (TMA;
// NY / 8 boxes of 8 rows, already in the padded row pitch) and its D_l plane
// by one bulk copy, both issued an item ahead:
//   YA  inverse y, DIF phase A (BY points), in place on the loaded rows
//   F1  inverse y DIF phase B (SY points) and inverse x DIF phase A
//       (4 points) on an SY x 4 block per thread
//   X2  inverse x DIF phase B (BX points) -> real psi of BX voxels ->
//       inc = coefD D_l psi (+ record / gradient terms) -> forward x DIT
//       phase A (BX points) on the same slots; then the next item's D_l copy
//       is issued into the freed buffer
//   F2  forward x DIT phase B and forward y DIT phase A (4 x SY block)
//   YB  forward y DIT phase B (BY points): with at most two tasks per thread
//       the columns are read into registers first, after which the plane is
//       free and the next item's psi~ rows are issued into it; the outputs get
//       the injections and w (read from global memory, asked of L2 at the
//       start of the item) and go to global memory while those copies are in
//       flight.
// MODE 0: plain step or operator application; 1: also record the real-space
// psi of the item (rec_out, forward segments of the adjoint); 2: adjoint step
// with the gradient terms (rec_in, grad_a, grad_s).
template <typename R, int NX, int NY, int NT, int MINB, int MODE>
__global__ void __launch_bounds__(NT, MINB) k_plane(const __grid_constant__ PlaneArgs<R> pa) {
    using T = typename cvec<R>::type;
    constexpr int SY = plane_sy(NY), BY = NY / SY, BX = NX / 4, PX = plane_pitch<R, NX>();
    constexpr int NE = NX * NY;
    constexpr unsigned kDlBytes = NE * sizeof(R);
    constexpr bool DLS = plane_dl_staged<R>(NX, NY);   // D_l staged in shared memory
    constexpr int NYB = (NX * SY + NT - 1) / NT;       // YA / YB tasks per thread
    constexpr bool EARLY = NYB <= 2;                    // YB columns held in registers
    // rows 0 .. WS-1 of the item's w plane are staged in shared memory after X2
    constexpr int WS = plane_w_rows<R>(NX, NY, MINB);
    constexpr unsigned kWBytes = WS * NX * sizeof(T);
    static_assert(WS % SY == 0, "staged w rows are whole k1 levels of the YB outputs");
    // a name of its own: declarations of one extern shared array share one alignment
    extern __shared__ __align__(128) unsigned char plane_smem_raw[];
    T *s = reinterpret_cast<T *>(plane_smem_raw);
    unsigned char *stg = reinterpret_cast<unsigned char *>(s + NY * PX);   // staging buffer
    R *dls = reinterpret_cast<R *>(stg);   // D_l of the item, slot order [x slot][y slot], up to X2
    const T *wst = reinterpret_cast<const T *>(stg);   // w rows 0 .. WS-1 of the item, after X2
    T *twx = reinterpret_cast<T *>(stg + plane_stage_bytes<R>(NX, NY, MINB));   // w_NX^j
    T *twy = twx + NX;                                      // w_NY^j
    T *twxa = twy + NY;   // [k1][t]: w_NX^{t k1}, k1 < 4, t < BX (lanes over t)
    T *twxb = twxa + NX;  // [j1][k2]: w_NX^{j1 k2}, j1 < 4, k2 < BX (one row per warp)
    T *twya = twxb + NX;  // [t][k1]: w_NY^{t k1}, t < SY, k1 < BY
    T *twyb = twya + NY;  // [j1][k2]: w_NY^{j1 k2}, j1 < BY, k2 < SY
    static_assert(NY % kRowsPerCopy == 0 && NY / kRowsPerCopy <= 32, "one tensor copy per lane of warp 0");
    static_assert(PX * sizeof(T) % 16 == 0 && kRowsPerCopy * PX * sizeof(T) % 128 == 0,
                  "box rows a multiple of 16 bytes, boxes 128-byte aligned in shared memory");
    constexpr unsigned kPlaneBytes = NY * PX * sizeof(T);   // bytes the tensor copies write
    // the barriers live in dynamic shared memory too (no static shared
    // memory), so that the plane starts at the 128-byte aligned base
    unsigned long long &bar_rows = reinterpret_cast<unsigned long long *>(twyb + SY * BY)[0];
    unsigned long long &bar_dl = reinterpret_cast<unsigned long long *>(twyb + SY * BY)[1];
    unsigned long long &bar_w = reinterpret_cast<unsigned long long *>(twyb + SY * BY)[2];
    const int tid = threadIdx.x;
    const int M = pa.M;
    const int per = M * pa.nz;               // items of one plan
    const int nitems = per * pa.nplans;
    const size_t V = (size_t)pa.nz * NE;
    // warp 0: the psi~ plane of `item` by NY / 8 tensor copies of 8 rows, one
    // per lane; row (m nz + z) ny + y of the plan's rows_map is row y of the
    // plane (moment m, plane z)
    auto issue_rows = [&](int item) {
        const int ip = item % per;
        const int row0 = ((ip % M) * pa.nz + ip / M) * NY;
        if (tid == 0) mbar_arrive_expect(&bar_rows, kPlaneBytes);
        __syncwarp();
        if (tid < NY / kRowsPerCopy)
            tma_load_2d(s + tid * kRowsPerCopy * PX, &pa.pl[item / per].rows_map, 0, row0 + tid * kRowsPerCopy,
                        &bar_rows);
    };
    auto issue_dl = [&](int item) {     // thread 0: D_l of `item`
        const int ip = item % per;
        mbar_arrive_expect(&bar_dl, kDlBytes);
        bulk_g2s(dls, pa.pl[item / per].dl_slot + (size_t)pa.lof[ip % M] * V + (size_t)(ip / M) * NE, kDlBytes,
                 &bar_dl);
    };
    auto issue_w = [&](int item) {      // thread 0: rows 0 .. WS-1 of the w plane of `item` (contiguous)
        const int ip = item % per;
        mbar_arrive_expect(&bar_w, kWBytes);
        bulk_g2s(stg, pa.pl[item / per].win + (size_t)(ip % M) * V + (size_t)(ip / M) * NE, kWBytes, &bar_w);
    };
    auto fail_all = [&]() {             // thread 0: record an abandoned step in every plan of the group
        for (int q = 0; q < pa.nplans; ++q) atomicOr(pa.pl[q].status, 1);
    };
    for (int i = tid; i < NX; i += NT) {
        twx[i] = pa.twx[i];
        twxa[i] = pa.twx[(i % BX) * (i / BX)];
        twxb[i] = pa.twx[(i / BX) * (i % BX)];
    }
    for (int i = tid; i < NY; i += NT) {
        twy[i] = pa.twy[i];
        twya[i] = pa.twy[(i / BY) * (i % BY)];
        twyb[i] = pa.twy[(i / SY) * (i % SY)];
    }
    // tensor copies need a 128-byte aligned destination: refuse to run
    // (and report) rather than copy to a misaligned plane
    if (smem_u32(plane_smem_raw) & 127u) {
        if (tid == 0) fail_all();
        return;
    }
    if (tid == 0) {
        mbar_init(&bar_rows, 1);
        mbar_init(&bar_dl, 1);
        mbar_init(&bar_w, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if ((int)blockIdx.x < nitems) {
        if (tid < 32) issue_rows(blockIdx.x);
        if (DLS && tid == 0) issue_dl(blockIdx.x);
    }
    const R inv = R(1) / R(NE);
    unsigned parity = 0;
    bool w_late = false;   // a staged w copy did not arrive in time (agreed on at the next barrier)
    for (int b = blockIdx.x; b < nitems; b += gridDim.x, parity ^= 1u) {
        const int pp = b / per, bi = b % per;
        const int m = bi % M, z = bi / M;
        const PlanePlan<R> &P = pa.pl[pp];
        const size_t zoff = (size_t)z * NE;
        const int l = pa.lof[m];
        const int nb = b + gridDim.x;
        if (tid == 0) {
            prefetch_l2(P.win + (size_t)m * V + zoff, NE * sizeof(T));
            if (nb < nitems) {
                const int ni = nb % per;
                prefetch_l2(pa.pl[nb / per].psi_in + (size_t)(ni % M) * V + (size_t)(ni / M) * NE, NE * sizeof(T));
            }
            if (!DLS || WS > 0) prefetch_l2(P.dl_slot + (size_t)l * V + zoff, NE * sizeof(R));
        }
        // YA: column x, rows t + SY q, conjugated (F^-1 = conj F conj / n); in
        // place, once the plane has arrived. A wait that runs out is agreed on
        // by the whole CTA at the barrier below.
        const bool arrived = mbar_wait(&bar_rows, parity);
        for (int w = tid; arrived && w < NX * SY; w += NT) {
            const int x = w % NX, t = w / NX;
            T v[BY], tw[BY];
#pragma unroll
            for (int q = 0; q < BY; ++q) v[q] = cconj(s[(t + SY * q) * PX + x]);
            row_load<T, BY>(twya + t * BY, tw);
            dftR<T, BY>(v);
#pragma unroll
            for (int k1 = 1; k1 < BY; ++k1) v[k1] = cmul(v[k1], tw[k1]);
#pragma unroll
            for (int k1 = 0; k1 < BY; ++k1) s[(t + SY * k1) * PX + x] = v[k1];
        }
        if (__syncthreads_or(!arrived || w_late)) {
            if (tid == 0) {
                fail_all();
                mbar_wait(&bar_rows, parity);   // bounded: copies in flight
                if (DLS && (WS == 0 || b == (int)blockIdx.x)) mbar_wait(&bar_dl, parity);
                if (w_late) mbar_wait(&bar_w, parity ^ 1u);   // the previous item's w rows
            }
            return;
        }
        // with w staged, the buffer is free from here (every thread has read
        // the previous item's w rows) until this item's X2: D_l goes in now
        if (WS > 0 && tid == 0 && b != (int)blockIdx.x) issue_dl(b);
        // F1: y slots SY k1y + j, x = tx + BX q
        for (int w = tid; w < BY * BX; w += NT) {
            const int tx = w % BX, k1y = w / BX;
            T *blk = s + SY * k1y * PX + tx;
            T v[4][SY];   // [q][j]
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < SY; ++j) v[q][j] = blk[j * PX + BX * q];
#pragma unroll
            for (int q = 0; q < 4; ++q) dftR<T, SY>(v[q]);
            const T ta1 = twxa[BX + tx], ta2 = twxa[2 * BX + tx], ta3 = twxa[3 * BX + tx];
#pragma unroll
            for (int j = 0; j < SY; ++j) {
                T u[4] = {v[0][j], v[1][j], v[2][j], v[3][j]};
                dft<T, 4>::run(u);
                blk[j * PX] = u[0];
                blk[j * PX + BX] = cmul(u[1], ta1);
                blk[j * PX + 2 * BX] = cmul(u[2], ta2);
                blk[j * PX + 3 * BX] = cmul(u[3], ta3);
            }
        }
        if (__syncthreads_or(DLS && !mbar_wait(&bar_dl, parity))) {
            if (tid == 0) fail_all();
            return;
        }
        // X2: row slot py (real y), block k1x of BX slots (real x = k1x + 4 k2)
        for (int w = tid; w < NY * 4; w += NT) {
            const int py = w % NY, k1x = w / NY;
            const int y = py / SY + BY * (py % SY);
            T *row = s + py * PX + BX * k1x;
            T v[BX];
            row_load<T, BX>(row, v);
            dftR<T, BX>(v);
            const size_t rowv = zoff + (size_t)y * NX;
            const R *dsrc = DLS ? dls + (BX * k1x) * NY + py
                                : P.dl_slot + (size_t)l * V + zoff + (size_t)(BX * k1x) * NY + py;
#pragma unroll
            for (int k2 = 0; k2 < BX; ++k2) {
                const int x = k1x + 4 * k2;
                const T p = mk<T>(v[k2].x * inv, -v[k2].y * inv);
                if constexpr (MODE == 1) pa.rec_out[(size_t)m * V + rowv + x] = p;
                if constexpr (MODE == 2) {
                    const T ps = pa.rec_in[(size_t)m * V + rowv + x];
                    const double pr = (double)pa.grad_scale * (double)pa.wl[m] * ((double)p.x * ps.x + (double)p.y * ps.y);
                    atomicAdd(pa.grad_a + rowv + x, pr);
                    if (l > 0)
                        atomicAdd(pa.grad_s + rowv + x,
                                  pr * (double)pa.gfac[(size_t)(l - 1) * V + zoff + (size_t)(BX * k1x + k2) * NY + py]);
                }
                v[k2] = cscale(p, P.coefD * dsrc[k2 * NY]);
            }
            dftR<T, BX>(v);
            {
                T tw[BX];
                row_load<T, BX>(twxb + k1x * BX, tw);
#pragma unroll
                for (int k2 = 1; k2 < BX; ++k2) v[k2] = cmul(v[k2], tw[k2]);
            }
            row_store<T, BX>(row, v);
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            if (WS > 0) issue_w(b);                          // the buffer is free until YB
            else if (DLS && nb < nitems) issue_dl(nb);       // the D_l buffer is free until the next X2
        }
        // F2: x slots BX j1x + k2x, y slots SY j1y + j2
        for (int w = tid; w < BY * BX; w += NT) {
            const int k2x = w % BX, j1y = w / BX;
            T *blk = s + SY * j1y * PX + k2x;
            T v[SY][4];   // [j2][j1x]
#pragma unroll
            for (int j2 = 0; j2 < SY; ++j2)
#pragma unroll
                for (int j1 = 0; j1 < 4; ++j1) v[j2][j1] = blk[j2 * PX + BX * j1];
#pragma unroll
            for (int j2 = 0; j2 < SY; ++j2) dft<T, 4>::run(v[j2]);   // x = k2x + BX k1
            T tw[SY];
            row_load<T, SY>(twyb + j1y * SY, tw);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) {
                T u[SY];
#pragma unroll
                for (int j2 = 0; j2 < SY; ++j2) u[j2] = v[j2][k1];
                dftR<T, SY>(u);
#pragma unroll
                for (int k2 = 0; k2 < SY; ++k2) blk[k2 * PX + BX * k1] = k2 ? cmul(u[k2], tw[k2]) : u[k2];
            }
        }
        __syncthreads();
        // YB: column kx, outputs ky = k2 + SY k1
        T v[EARLY ? NYB : 1][BY];
        if constexpr (EARLY) {
#pragma unroll
            for (int h = 0; h < NYB; ++h) {
                const int w = tid + h * NT;
                if (w < NX * SY) {
                    const int kx = w % NX, k2 = w / NX;
#pragma unroll
                    for (int j1 = 0; j1 < BY; ++j1) v[h][j1] = s[(SY * j1 + k2) * PX + kx];
                }
            }
            fence_proxy_async();
            __syncthreads();
            if (tid < 32 && nb < nitems) issue_rows(nb);   // the plane is free: next item's rows
        }
        {
            const T *wp = P.win + (size_t)m * V + zoff;
            T *dst = P.out + (size_t)m * V + zoff;
            const int step = P.ninj ? *P.step : 0;
            // rows below WS of w come from the staging buffer
            if (WS > 0 && !mbar_wait(&bar_w, parity)) w_late = true;
#pragma unroll
            for (int h = 0; h < NYB; ++h) {
                const int w = tid + h * NT;
                if (w >= NX * SY) continue;
                const int kx = w % NX, k2 = w / NX;
                T *vv = v[EARLY ? h : 0];
                if constexpr (!EARLY) {
#pragma unroll
                    for (int j1 = 0; j1 < BY; ++j1) vv[j1] = s[(SY * j1 + k2) * PX + kx];
                }
                T wv[BY];
#pragma unroll
                for (int k1 = WS / SY; k1 < BY; ++k1) wv[k1] = wp[(k2 + SY * k1) * NX + kx];
#pragma unroll
                for (int k1 = 0; k1 < WS / SY; ++k1) wv[k1] = wst[(k2 + SY * k1) * NX + kx];
                dftR<T, BY>(vv);
                // point injections enter as the DFT of a delta: a w_NX^{kx x} w_NY^{ky y}
                for (int q = 0; q < P.ninj; ++q) {
                    const int4 pt = P.inj[q];
                    if (pt.w != m || pt.z != z) continue;
                    const T ex = twx[(kx * pt.x) % NX];
                    const R a = P.inj_amp[(size_t)step * P.ninj + q];
#pragma unroll
                    for (int k1 = 0; k1 < BY; ++k1) {
                        const T ph = cmul(ex, twy[((k2 + SY * k1) * pt.y) % NY]);
                        vv[k1].x += a * ph.x;
                        vv[k1].y += a * ph.y;
                    }
                }
#pragma unroll
                for (int k1 = 0; k1 < BY; ++k1) {
                    const T o = cadd(wv[k1], vv[k1]);
                    if (kx == 0) flag_nonfinite(P.nonfinite, o);
                    dst[(k2 + SY * k1) * NX + kx] = o;
                }
            }
        }
        if constexpr (!EARLY) {
            fence_proxy_async();
            __syncthreads();
            if (tid < 32 && nb < nitems) issue_rows(nb);
        }
        if constexpr (WS > 0) fence_proxy_async();   // w reads before the next D_l copy
    }
    // the last item's staged w: a late copy is reported like the others
    if (WS > 0 && __syncthreads_or(w_late) && tid == 0) {
        fail_all();
        mbar_wait(&bar_w, parity ^ 1u);   // bounded: the copy in flight
    }
}

// Z pass with the streaming term, for a fixed nz = N1 N2:
//   w = a psi~ + coefS S~(psi~),
//   S~ = Z + (i kx + ky) P + (i kx - ky) Q                  (Eq. 10, mixed space)
//   Z  = F_z^-1[i kz F_z (zc0 psi~_{zs0} + zc1 psi~_{zs1})]
//   P  = pc0 psi~_{ps0} + pc1 psi~_{ps1},  Q = qc0 psi~_{qs0} + qc1 psi~_{qs1},
// mirrored operands (real-radiance layout) read conj(psi~(-kx, -ky)). The
// z derivative is linear, so the two z couplings are combined before one
// transform. One CTA per (output moment m, TX columns of one plan of the
// group, row ky); the moment runs fastest over the grid and the rows go 0,
// n-1, 1, n-2, ... so that the
// CTAs reading each other's tiles (neighbouring moments, mirrored rows) run
// together. Transform phases as in k_zderiv_fixed. NT = TX N2 threads: the
// last transform phase leaves each thread one column and the N1 rows
// k2 + N2 k1, and the epilogue takes the same column and rows from those
// registers. GNX, GNY > 0 fix the plane's extents at compile time (all
// operand offsets become constants; GNX a multiple of TX), 0 reads them from g.
template <typename R, int N1, int N2, int TX, int NT, int GNX = 0, int GNY = 0>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 ? 1024 : 384) / NT)
    k_zstream(const __grid_constant__ ZArgs<R> za, Geo<R> g, const CouplingRow *__restrict__ coup) {
    using T = typename cvec<R>::type;
    constexpr int NZ = N1 * N2, P = TX + 1;
    static_assert(NT == TX * N2, "one (column, row class) per thread");
    static_assert(GNX % TX == 0, "compile-time planes hold whole x tiles");
    constexpr bool kWhole = GNX > 0;    // every tile lies inside the plane
    __shared__ T s[NZ * P];
    __shared__ T tw[NZ];
    __shared__ R kzs[NZ];    // coefS kz / NZ
    __shared__ CouplingKinds<R> ck;
    const int pl = blockIdx.y / za.nxt;
    const int m = blockIdx.x, x0 = (blockIdx.y % za.nxt) * TX, yi = blockIdx.z;
    const T *__restrict__ in = za.in[pl];
    T *__restrict__ out = za.out[pl];
    const R a = za.a[pl], coefS = za.coefS[pl];
    const int gnx = GNX ? GNX : g.nx, gny = GNY ? GNY : g.ny;
    const int y = (yi & 1) ? gny - 1 - (yi >> 1) : (yi >> 1);
    const int ym = (gny - y) % gny;
    const size_t plane = (size_t)gny * gnx, V = (size_t)NZ * plane;
    const int tid = threadIdx.x;
    for (int i = tid; i < NZ; i += NT) {
        tw[i] = g.twz[i];
        kzs[i] = g.kz[i] * (coefS / R(NZ));
    }
    if (tid == 0) split_coupling<R>(coup[m], m, ck);
    __syncthreads();
    const CouplingKinds<R> k = ck;
    const bool zterm = k.zc[0] != R(0);
    T vc[N1];    // Z at this thread's column and rows k2 + N2 k1 (phase C)
    if (zterm) {
        const T *b0 = in + (size_t)k.zs[0] * V + (size_t)y * gnx + x0;
        const T *b1 = in + (size_t)k.zs[1] * V + (size_t)y * gnx + x0;
        const bool two = k.zc[1] != R(0);
        // A: column b, rows t + N2 q of zc0 psi~_{zs0} + zc1 psi~_{zs1}
        for (int w = tid; w < TX * N2; w += NT) {
            const int b = w % TX, t = w / TX;
            const bool ok = kWhole || x0 + b < gnx;
            T v[N1];
#pragma unroll
            for (int q = 0; q < N1; ++q) {
                const size_t o = (size_t)(t + N2 * q) * plane + b;
                const T u0 = ok ? b0[o] : czero<T>();
                const T u1 = ok && two ? b1[o] : czero<T>();
                v[q] = mk<T>(k.zc[0] * u0.x + k.zc[1] * u1.x, k.zc[0] * u0.y + k.zc[1] * u1.y);
            }
            dftR<T, N1>(v);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) s[(t + N2 * k1) * P + b] = v[k1];
        }
        __syncthreads();
        // B: block N2 k1 of column b: DIF phase B, times conj(i coefS kz / nz), DIT phase A
        for (int w = tid; w < TX * N1; w += NT) {
            const int b = w % TX, k1 = w / TX;
            T v[N2];
#pragma unroll
            for (int t = 0; t < N2; ++t) v[t] = s[(N2 * k1 + t) * P + b];
            dftR<T, N2>(v);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const R kk = kzs[k1 + N1 * k2];
                v[k2] = mk<T>(-kk * v[k2].y, -kk * v[k2].x);   // conj(i coefS k v / nz)
            }
            dftR<T, N2>(v);
#pragma unroll
            for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw[k1 * k2]);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) s[(N2 * k1 + k2) * P + b] = v[k2];
        }
        __syncthreads();
        // C: DIT phase B in registers: vc[k1] is (the conjugate of) Z at
        // z index k2 + N2 k1 of column b, with (b, k2) = (tid % TX, tid / TX)
        {
            const int b = tid % TX, k2 = tid / TX;
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) vc[j1] = s[(N2 * j1 + k2) * P + b];
            dftR<T, N1>(vc);
        }
    }
    // epilogue: thread (column b, first row zr) takes rows zr + N2 j; the
    // operand addresses are fixed per thread up to the row offset. Z already
    // carries coefS (folded into the i kz scale of phase B).
    const int b = tid % TX, zr = tid / TX, x = x0 + b;
    if (kWhole || x < gnx) {
        const R pcy0 = k.pm[0] ? -k.pc[0] : k.pc[0], pcy1 = k.pm[1] ? -k.pc[1] : k.pc[1];
        const R qcy0 = k.qm[0] ? -k.qc[0] : k.qc[0], qcy1 = k.qm[1] ? -k.qc[1] : k.qc[1];
        const size_t oe = (size_t)y * gnx + x;
        const size_t om = (size_t)ym * gnx + (x ? gnx - x : 0);   // (-kx, -ky)
        const T *ps = in + (size_t)m * V + oe;
        const T *pp0 = in + (size_t)k.ps[0] * V + (k.pm[0] ? om : oe);
        const T *pp1 = in + (size_t)k.ps[1] * V + (k.pm[1] ? om : oe);
        const T *pq0 = in + (size_t)k.qs[0] * V + (k.qm[0] ? om : oe);
        const T *pq1 = in + (size_t)k.qs[1] * V + (k.qm[1] ? om : oe);
        // an absent operand points at the moment itself (split_coupling) with
        // a zero coefficient, so every load is unconditional
        if (!zterm) {
#pragma unroll
            for (int j = 0; j < N1; ++j) vc[j] = czero<T>();
        }
        T *pd = out + (size_t)m * V + oe;
        const R ckx = coefS * g.kx[x], cky = coefS * g.ky[y];
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const int zz = zr + N2 * j;
            const size_t o = (size_t)zz * plane;
            const T self = ps[o];
            const T p0 = pp0[o], p1 = pp1[o];
            const T q0 = pq0[o], q1 = pq1[o];
            const T zv = cconj(vc[j]);
            const R pr = k.pc[0] * p0.x + k.pc[1] * p1.x, pi = pcy0 * p0.y + pcy1 * p1.y;
            const R qr = k.qc[0] * q0.x + k.qc[1] * q1.x, qi = qcy0 * q0.y + qcy1 * q1.y;
            // coefS (i kx + ky) P + coefS (i kx - ky) Q
            const R sr = cky * (pr - qr) - ckx * (pi + qi);
            const R si = ckx * (pr + qr) + cky * (pi - qi);
            pd[o] = mk<T>(a * self.x + zv.x + sr, a * self.y + zv.y + si);
        }
    }
}

// Readouts Re psi_00 at detector voxels of the state psi~ (before a step):
// psi(x, y, z) = (1/(nx ny)) sum_{kx, ky} psi~(kx, ky, z) w^{-(kx x + ky y)}.
// Grid (ndet, kTapChunks): CTA (d, c) sums rows ky = c, c + kTapChunks, ...
// in FP64 and writes one partial sum; k_taps_finish adds the partials of each
// detector in a fixed order.
constexpr int kTapChunks = 16;

// The twiddles are FP64 for both plan precisions: a detector where the field
// is far below its peak reads a sum with much cancellation, which FP32
// twiddles would turn into a relative error of order 6e-8 times the ratio.
template <typename R>
__global__ void k_taps(const typename cvec<R>::type *__restrict__ psi_t, int nx, int ny,
                       const double2 *__restrict__ twx, const double2 *__restrict__ twy,
                       const int4 *__restrict__ det, double *__restrict__ part) {
    using T = typename cvec<R>::type;
    const int d = blockIdx.x, c = blockIdx.y;
    const int4 q = det[d];
    const T *plane = psi_t + (size_t)q.z * ny * nx;
    double acc = 0.0;
    for (int ky = c; ky < ny; ky += kTapChunks) {
        const double2 b = twy[(int)(((long)ky * q.y) % ny)];
        for (int kx = threadIdx.x; kx < nx; kx += blockDim.x) {
            const double2 a = twx[(int)(((long)kx * q.x) % nx)];
            // w^{-j} = conj(w^j)
            const double cr = a.x * b.x - a.y * b.y, ci = -(a.x * b.y + a.y * b.x);
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
// FP64 instances take half the CTAs per SM of the FP32 ones: their
// register DFTs of 16 to 20 complex doubles spill at 64 registers.
template <typename R, int N1, int N2, int TX, int NT, int COUPLE>
__global__ void __launch_bounds__(NT, 2048 / NT / (sizeof(R) == 4 ? 2 : 4))
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
            const T o = mk<T>(a * self.x + f.x + coefS * sr, a * self.y + f.y + coefS * si);
            if (x == 0) flag_nonfinite(g.nonfinite, o);
            out[base + ep - x0] = o;
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
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2)
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
