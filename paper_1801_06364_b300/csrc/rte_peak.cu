// rte_peak.cu -- rte_fma_peak: the FMA throughput of the current device in
// FP32 or FP64, measured with this library's own kernel. The FP64 leg of the
// explicit step is bound by the FP64 pipe on B300 (its FP64 rate is a small
// fraction of FP32), so its roofline needs this peak; FP32 is given for the
// ridge point of the FP32 step.
#include <cuda_runtime.h>

#include <string>

#include "rte.h"

namespace rte {
void set_last_error(const std::string &msg);
}

namespace {

// 8 independent FMA chains per thread, 16 steps per iteration: the pipe sees
// one FMA per chain and cycle of its latency
template <typename R> __global__ void k_fma_chains(R *out, int iters, R b, R c) {
    R a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (R)(threadIdx.x + j) * (R)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = a[j] * b + c;
    }
    R sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) sum += a[j];
    if (sum == (R)1234.5) out[0] = sum;   // never true; keeps the chains live
}

template <typename R> rte_status measure(double *flops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    R *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(R));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8;
    // about 20 ms on a B300 in either precision
    const int iters = sizeof(R) == 4 ? 4096 : 256;
    float ms = 0.0f;
    if (e == cudaSuccess) {
        k_fma_chains<R><<<blocks, threads>>>(out, 8, (R)0.999999, (R)1e-7);   // warm-up
        cudaEventRecord(e0);
        k_fma_chains<R><<<blocks, threads>>>(out, iters, (R)0.999999, (R)1e-7);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        rte::set_last_error(std::string("rte_fma_peak: ") + cudaGetErrorString(e));
        return RTE_ERR_CUDA;
    }
    *flops = 2.0 * 8.0 * 16.0 * (double)iters * threads * blocks / (ms * 1e-3);
    return RTE_OK;
}

}  // namespace

extern "C" rte_status rte_fma_peak(int precision, double *flop_per_s) {
    if (!flop_per_s || (precision != RTE_FP32 && precision != RTE_FP64)) {
        rte::set_last_error("rte_fma_peak: bad argument");
        return RTE_ERR_INVALID_ARG;
    }
    return precision == RTE_FP64 ? measure<double>(flop_per_s) : measure<float>(flop_per_s);
}
