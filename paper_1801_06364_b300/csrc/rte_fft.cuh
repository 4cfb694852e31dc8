// rte_fft.cuh -- complex arithmetic and shared-memory Stockham FFT passes.
//
// A batch of B lines of length n sits in shared memory; element e of line b
// lives at s[b * ls + e * es]. Each pass of radix R (R in {2, 3, 4, 5, 8})
// reads R inputs per butterfly into registers, applies the twiddles and an
// R-point DFT, and writes the outputs in self-sorting (Stockham) order to a
// second buffer of the same layout, so no bit-reversal is needed and a
// thread holds only one butterfly at a time. Lanes of a warp run over lines
// (b fastest): with an odd line pitch every shared-memory access is free of
// bank conflicts.
//
// Twiddles come from a table tw[j] = exp(-2 pi i j / n) computed in FP64 on
// the host (rounded once to FP32 for the FP32 path). The inverse transform is
// conj(FFT(conj(x))) / n.
#pragma once
#include <cuda_runtime.h>
#include "rte_types.h"

namespace rte {

template <typename R> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };

template <typename T> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename T>
__host__ __device__ __forceinline__ T mk(typename real_of<T>::type x, typename real_of<T>::type y) {
    T r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ T cconj(T a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ T cscale(T a, typename real_of<T>::type s) {
    return mk<T>(a.x * s, a.y * s);
}
// multiply by -i
template <typename T> __device__ __forceinline__ T cmuli_neg(T a) { return mk<T>(a.y, -a.x); }

// Forward R-point DFTs, X[k] = sum_n v[n] exp(-2 pi i n k / R), in place.
template <typename T, int R> struct dft;

template <typename T> struct dft<T, 2> {
    __device__ __forceinline__ static void run(T *v) {
        T a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <typename T> struct dft<T, 4> {
    __device__ __forceinline__ static void run(T *v) {
        T a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        T a2 = cadd(v[1], v[3]), a3 = cmuli_neg(csub(v[1], v[3]));
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    }
};

template <typename T> struct dft<T, 8> {
    __device__ __forceinline__ static void run(T *v) {
        using Rr = typename real_of<T>::type;
        const Rr h = (Rr)0.70710678118654752440084436210484904;   // 1/sqrt(2)
        T e[4] = {v[0], v[2], v[4], v[6]};
        T o[4] = {v[1], v[3], v[5], v[7]};
        dft<T, 4>::run(e);
        dft<T, 4>::run(o);
        // o[k] *= exp(-i pi k / 4)
        T o1 = mk<T>((o[1].x + o[1].y) * h, (o[1].y - o[1].x) * h);
        T o2 = cmuli_neg(o[2]);
        T o3 = mk<T>((o[3].y - o[3].x) * h, -(o[3].x + o[3].y) * h);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <typename T> struct dft<T, 3> {
    __device__ __forceinline__ static void run(T *v) {
        using Rr = typename real_of<T>::type;
        const Rr s3 = (Rr)0.86602540378443864676372317075293618;  // sin(2 pi / 3)
        T s = cadd(v[1], v[2]);
        T d = csub(v[1], v[2]);
        T t = mk<T>(v[0].x - (Rr)0.5 * s.x, v[0].y - (Rr)0.5 * s.y);
        T u = cmuli_neg(cscale(d, s3));
        v[0] = cadd(v[0], s);
        v[1] = cadd(t, u);
        v[2] = csub(t, u);
    }
};

template <typename T> struct dft<T, 5> {
    __device__ __forceinline__ static void run(T *v) {
        using Rr = typename real_of<T>::type;
        // cos/sin of 2 pi/5 and 4 pi/5: (sqrt5 - 1)/4, -(sqrt5 + 1)/4,
        // sqrt((5 + sqrt5)/8), sqrt((5 - sqrt5)/8)
        const Rr c1 = (Rr)0.30901699437494742410229341718281906;
        const Rr c2 = (Rr)-0.80901699437494742410229341718281906;
        const Rr s1 = (Rr)0.95105651629515357211643933337938214;
        const Rr s2 = (Rr)0.58778525229247312916870595463907277;
        T a0 = v[0];
        T p1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
        T p2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
        T r1 = mk<T>(a0.x + c1 * p1.x + c2 * p2.x, a0.y + c1 * p1.y + c2 * p2.y);
        T r2 = mk<T>(a0.x + c2 * p1.x + c1 * p2.x, a0.y + c2 * p1.y + c1 * p2.y);
        T i1 = cmuli_neg(mk<T>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
        T i2 = cmuli_neg(mk<T>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
        v[0] = cadd(a0, cadd(p1, p2));
        v[1] = cadd(r1, i1);
        v[4] = csub(r1, i1);
        v[2] = cadd(r2, i2);
        v[3] = csub(r2, i2);
    }
};

// One Stockham pass from src to dst (Ns = product of the radices already
// applied): butterfly j of line b reads src[j + r n/R], applies the twiddles
// w_{Ns R}^{r (j mod Ns)} and an R-point DFT, and writes
// dst[(j / Ns) Ns R + (j mod Ns) + r Ns].
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const T *src, T *dst, int n, int Ns, int B, int es, int ls,
                                              const T *__restrict__ tw, int tid, int nthr) {
    const int nb = n / R;
    const int total = B * nb;
    const int twmul = n / (Ns * R);
    for (int w = tid; w < total; w += nthr) {
        const int b = w % B, j = w / B;
        const int k = j % Ns;
        const T *in = src + b * ls + j * es;
        T v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T x = in[r * nb * es];
            if (r > 0 && k > 0) x = cmul(x, tw[r * k * twmul]);
            v[r] = x;
        }
        dft<T, R>::run(v);
        T *out = dst + b * ls + ((j / Ns) * Ns * R + k) * es;
#pragma unroll
        for (int r = 0; r < R; ++r) out[r * Ns * es] = v[r];
    }
    __syncthreads();
}

// Forward transform of B lines held in s0, ping-ponging with s1 (same
// layout). Returns the buffer that holds the result. The caller synchronises
// before the call; the call ends with a barrier.
template <typename T>
__device__ __forceinline__ T *fft_lines(T *s0, T *s1, const FftPlan &p, int B, int es, int ls,
                                        const T *__restrict__ tw, int tid, int nthr) {
    T *src = s0, *dst = s1;
    int Ns = 1;
    for (int q = 0; q < p.npass; ++q) {
        const int R = p.radix[q];
        switch (R) {
            case 8: stockham_pass<T, 8>(src, dst, p.n, Ns, B, es, ls, tw, tid, nthr); break;
            case 4: stockham_pass<T, 4>(src, dst, p.n, Ns, B, es, ls, tw, tid, nthr); break;
            case 2: stockham_pass<T, 2>(src, dst, p.n, Ns, B, es, ls, tw, tid, nthr); break;
            case 3: stockham_pass<T, 3>(src, dst, p.n, Ns, B, es, ls, tw, tid, nthr); break;
            default: stockham_pass<T, 5>(src, dst, p.n, Ns, B, es, ls, tw, tid, nthr); break;
        }
        T *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

}  // namespace rte
