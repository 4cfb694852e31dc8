// rte_noalloc.cu -- rte_apply_transport_noalloc: the transport operator
// T psi = F^-1[psidot] + D_l psi for callers that must not allocate device
// memory (code running where cudaMalloc is forbidden or unavailable: inside
// another framework's memory pool, under a fixed device-memory budget, or in
// a plugin that may not call the CUDA allocator). It runs the same kernels as
// rte_apply_transport, with every table and work buffer placed in one
// file-scope device array instead of memory owned by a plan.
//
// The scratch array (kScratchBytes, 32 MiB) is part of the library image:
// every GPU that loads librte holds it until the process exits. Its device
// address is looked up with cudaGetSymbolAddress on every call, so a call made
// after a device reset or in a re-created context gets the address valid in
// that context rather than a stale one. All calls share the array: two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and corrupt each other's results. Each call overwrites every byte it
// later reads, so nothing has to start at zero and the contents left by the
// previous call do not matter.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rte.h"
#include "rte_host.h"
#include "rte_kernels.cuh"

using namespace rte;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];


rte_status na_fail(rte_status s, const std::string &msg) {
    rte::set_last_error(msg);   // readable through rte_last_error_string()
    return s;
}

#define NA_CK(x)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) return na_fail(RTE_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define NA_RT(x)                      \
    do {                              \
        rte_status s_ = (x);          \
        if (s_ != RTE_OK) return s_;  \
    } while (0)

// Device address of the scratch array in the current context, looked up on
// every call (the lookup costs microseconds; the transport it serves costs
// milliseconds), so that no address outlives the context it belongs to.
rte_status scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
        return na_fail(RTE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return RTE_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename R> using CTn = typename cvec<R>::type;

// Carving of the scratch array for one problem.
struct Layout {
    size_t tw[3], kt[3], lof, coup, med, psit, dz, t1, total;
};

template <typename R> Layout layout_for(const rte_grid_desc *d) {
    const size_t V = (size_t)d->nx * d->ny * d->nz;
    const int M = (d->N + 1) * (d->N + 1);
    const int dims[3] = {d->nx, d->ny, d->nz};
    Layout L;
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
        L.tw[a] = off;
        off += align256(dims[a] * sizeof(CTn<R>));
        L.kt[a] = off;
        off += align256(dims[a] * sizeof(R));
    }
    L.lof = off;
    off += align256(M * sizeof(int));
    L.coup = off;
    off += align256(M * sizeof(CouplingRow));
    L.med = off;
    off += align256(V * sizeof(typename Media4<R>::type));
    const size_t fb = align256(V * M * sizeof(CTn<R>));
    L.psit = off;
    off += fb;
    L.dz = off;
    off += fb;
    L.t1 = off;
    off += fb;
    L.total = off;
    return L;
}

// The dynamic shared memory limit belongs to the kernel function, not to the
// launch: every caller sets the most the device allows next to the kernel's
// static shared memory, so that concurrent callers on other host threads
// cannot lower it under a pending launch.
template <typename K> cudaError_t na_allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const size_t most = (size_t)optin - fa.sharedSizeBytes;   // static + dynamic <= opt-in
    if (bytes > most) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
}

int na_threads(long elems) {
    long t = (elems + 7) / 8;
    t = ((t + 31) / 32) * 32;
    return (int)std::min<long>(std::max<long>(t, 64), kMaxThreads);
}

template <typename R> int na_tile_cols(int n) {
    int TX = sizeof(R) == 4 ? 16 : 8;
    while (TX > 1 && 2 * (size_t)n * (TX + 1) * sizeof(CTn<R>) > 200 * 1024) TX /= 2;
    return TX;
}

// Launch context: geometry plus the scratch carving.
template <typename R> struct Ctx {
    const rte_grid_desc *d;
    int M;
    cudaStream_t st;
    Geo<R> g;
    const CouplingRow *coup;
    const typename Media4<R>::type *med;
    const int *lof;
};

template <typename R> rte_status na_zderiv(const Ctx<R> &c, const void *in, void *out) {
    const int TX = na_tile_cols<R>(c.d->nz);
    const size_t smem = 2 * (size_t)c.d->nz * (TX + 1) * sizeof(CTn<R>);
    dim3 grid((c.d->nx + TX - 1) / TX, c.d->ny, c.M);
    NA_CK(na_allow_smem(k_zderiv<R>, smem));
    k_zderiv<R><<<grid, na_threads((long)c.d->nz * TX), smem, c.st>>>((const CTn<R> *)in, (CTn<R> *)out, c.g, TX);
    NA_CK(cudaGetLastError());
    return RTE_OK;
}

template <typename R>
rte_status na_ypass(const Ctx<R> &c, const void *in, void *out, int inverse, const void *psi_in, const void *dz,
                    double a, double coefS) {
    const int TX = na_tile_cols<R>(c.d->ny);
    const size_t smem = 2 * (size_t)c.d->ny * (TX + 1) * sizeof(CTn<R>);
    dim3 grid((c.d->nx + TX - 1) / TX, c.d->nz, c.M);
    NA_CK(na_allow_smem(k_ypass<R>, smem));
    k_ypass<R><<<grid, na_threads((long)c.d->ny * TX), smem, c.st>>>((const CTn<R> *)in, (CTn<R> *)out, c.g, TX,
                                                                   inverse, (const CTn<R> *)psi_in,
                                                                   (const CTn<R> *)dz, (R)a, (R)coefS, c.coup);
    NA_CK(cudaGetLastError());
    return RTE_OK;
}

template <typename R> rte_status na_xpass(const Ctx<R> &c, const void *in, void *out, const XArgs<R> &xa) {
    const size_t line = 2 * (size_t)(c.d->nx + 1) * sizeof(CTn<R>);
    int maxmc = (int)std::max<size_t>(1, (96 * 1024) / line);
    maxmc = std::min(maxmc, c.M);
    const int nch = (c.M + maxmc - 1) / maxmc;
    const int MC = (c.M + nch - 1) / nch;
    const size_t smem = 2 * (size_t)MC * (c.d->nx + 1) * sizeof(CTn<R>);
    dim3 grid(c.d->ny, c.d->nz, nch);
    NA_CK(na_allow_smem(k_xpass<R>, smem));
    k_xpass<R><<<grid, na_threads((long)MC * c.d->nx), smem, c.st>>>((const CTn<R> *)in, (CTn<R> *)out, c.g, MC, xa);
    NA_CK(cudaGetLastError());
    return RTE_OK;
}

template <typename R>
rte_status apply_noalloc(const rte_grid_desc *d, const double *mua, const double *mus, const double *gg,
                         const void *psi_in, void *psi_out, cudaStream_t st) {
    const Layout L = layout_for<R>(d);
    if (L.total > kScratchBytes) {
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "problem needs %zu bytes of scratch; rte_apply_transport_noalloc holds at most %zu bytes "
                      "(use rte_apply_transport with a plan instead)",
                      L.total, kScratchBytes);
        return na_fail(RTE_ERR_INVALID_ARG, buf);
    }
    void *base_v = nullptr;
    NA_RT(scratch_address(&base_v));
    char *base = (char *)base_v;
    const size_t V = (size_t)d->nx * d->ny * d->nz;
    const int M = (d->N + 1) * (d->N + 1);
    const int dims[3] = {d->nx, d->ny, d->nz};

    // host-built tables, copied into the scratch array (no device allocation)
    Ctx<R> c;
    c.d = d;
    c.M = M;
    c.st = st;
    c.g.nx = d->nx;
    c.g.ny = d->ny;
    c.g.nz = d->nz;
    c.g.M = M;
    c.g.nonfinite = nullptr;
    FftPlan *fp[3] = {&c.g.px, &c.g.py, &c.g.pz};
    const CTn<R> **tws[3] = {&c.g.twx, &c.g.twy, &c.g.twz};
    const R **kts[3] = {&c.g.kx, &c.g.ky, &c.g.kz};
    for (int a = 0; a < 3; ++a) {
        radix_plan(dims[a], fp[a]);
        auto tw = twiddles(dims[a]);
        std::vector<CTn<R>> twr(dims[a]);
        std::vector<R> kr(dims[a]);
        for (int j = 0; j < dims[a]; ++j) {
            twr[j].x = (R)tw[j].real();
            twr[j].y = (R)tw[j].imag();
            kr[j] = (R)wavenumber(j, dims[a], d->dx_mm);
        }
        NA_CK(cudaMemcpyAsync(base + L.tw[a], twr.data(), dims[a] * sizeof(CTn<R>), cudaMemcpyHostToDevice, st));
        NA_CK(cudaMemcpyAsync(base + L.kt[a], kr.data(), dims[a] * sizeof(R), cudaMemcpyHostToDevice, st));
        *tws[a] = (const CTn<R> *)(base + L.tw[a]);
        *kts[a] = (const R *)(base + L.kt[a]);
    }
    std::vector<int> lof(M);
    for (int l = 0; l <= d->N; ++l)
        for (int m = -l; m <= l; ++m) lof[l * l + l + m] = l;
    auto rows = coupling_rows(d->N);
    std::vector<double> mub;
    std::vector<uint8_t> mask;
    layer_profile(d->nx, d->ny, d->nz, d->pml_cells, d->pml_mu0, d->pml_mu1, mub, mask);
    std::vector<typename Media4<R>::type> med(V);
    for (size_t v = 0; v < V; ++v) {
        med[v].x = (R)(mask[v] ? mub[v] : mua[v]);
        med[v].y = (R)(mask[v] ? 0.0 : mus[v]);
        med[v].z = (R)gg[v];
        med[v].w = mask[v] ? (R)0 : (R)1;
    }
    NA_CK(cudaMemcpyAsync(base + L.lof, lof.data(), M * sizeof(int), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(base + L.coup, rows.data(), M * sizeof(CouplingRow), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(base + L.med, med.data(), V * sizeof(med[0]), cudaMemcpyHostToDevice, st));
    c.lof = (const int *)(base + L.lof);
    c.coup = (const CouplingRow *)(base + L.coup);
    c.med = (const typename Media4<R>::type *)(base + L.med);
    void *psit = base + L.psit, *dz = base + L.dz, *t1 = base + L.t1;

    XArgs<R> plain;
    std::memset(&plain, 0, sizeof(plain));
    plain.med = c.med;
    plain.lof = c.lof;
    // psi (real space) -> psi~ = F_xy psi
    NA_CK(cudaMemcpyAsync(t1, psi_in, V * M * sizeof(CTn<R>), cudaMemcpyDeviceToDevice, st));
    XArgs<R> xf = plain;
    xf.fwd_out = 1;
    NA_RT(na_xpass<R>(c, t1, t1, xf));
    NA_RT(na_ypass<R>(c, t1, psit, 0, nullptr, nullptr, 0.0, 0.0));
    // T psi~ = S~ psi~ + F_xy[D psi]
    NA_RT(na_zderiv<R>(c, psit, dz));
    NA_RT(na_ypass<R>(c, psit, t1, 1, nullptr, nullptr, 0.0, 0.0));
    XArgs<R> xp = plain;
    xp.inv_in = 1;
    xp.pointwise = 1;
    xp.fwd_out = 1;
    xp.coefD = (R)1;
    NA_RT(na_xpass<R>(c, t1, t1, xp));
    NA_RT(na_ypass<R>(c, t1, t1, 0, psit, dz, 0.0, 1.0));
    // back to real space, into the caller's output
    NA_RT(na_ypass<R>(c, t1, t1, 1, nullptr, nullptr, 0.0, 0.0));
    XArgs<R> xi = plain;
    xi.inv_in = 1;
    NA_RT(na_xpass<R>(c, t1, psi_out, xi));
    NA_CK(cudaStreamSynchronize(st));
    return RTE_OK;
}

bool na_axis_ok(int n) {
    FftPlan p;
    return n >= 4 && n <= 1024 && radix_plan(n, &p);
}

}  // namespace

extern "C" {

rte_status rte_apply_transport_noalloc(const rte_grid_desc *d, const double *mua, const double *mus,
                                       const double *g, const void *psi_in, void *psi_out, void *cuda_stream) {
    if (!d || !mua || !mus || !g || !psi_in || !psi_out || psi_in == psi_out)
        return na_fail(RTE_ERR_INVALID_ARG, "null or aliased argument");
    if (!na_axis_ok(d->nx) || !na_axis_ok(d->ny) || !na_axis_ok(d->nz) || d->N < 0 || d->N > 21 ||
        !(d->dx_mm > 0.0) || !(d->c_mm_per_ps > 0.0) || (d->precision != RTE_FP32 && d->precision != RTE_FP64) ||
        d->pml_cells < 0 || 2 * d->pml_cells >= std::min(d->nx, std::min(d->ny, d->nz)) ||
        (d->real_radiance != 0 && d->real_radiance != 1))
        return na_fail(RTE_ERR_INVALID_ARG, "bad grid descriptor");
    const size_t V = (size_t)d->nx * d->ny * d->nz;
    for (size_t v = 0; v < V; ++v)
        if (!std::isfinite(mua[v]) || !std::isfinite(mus[v]) || !std::isfinite(g[v]) || mua[v] < 0 || mus[v] < 0 ||
            g[v] < -1.0 || g[v] > 1.0)
            return na_fail(RTE_ERR_INVALID_ARG, "optical map has a negative, non-finite or out-of-range value");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return d->precision == RTE_FP64 ? apply_noalloc<double>(d, mua, mus, g, psi_in, psi_out, st)
                                    : apply_noalloc<float>(d, mua, mus, g, psi_in, psi_out, st);
}

}  // extern "C"
