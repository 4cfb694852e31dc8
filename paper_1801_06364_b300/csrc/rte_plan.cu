// rte_plan.cu -- the C ABI of librte (include/rte.h): plans, the explicit
// step, the transport operator, the steady-state GMRES solve and the
// checkpointed adjoint of the pseudospectral P_N method (Powell, Cox &
// Arridge, arXiv:1801.06364).
#include <algorithm>
#include <type_traits>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "rte.h"
#include "rte_host.h"
#include "rte_kernels.cuh"
#include "rte_plane.cuh"
#include "rte_expo.cuh"

using namespace rte;

namespace {

thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
const double kPi = 3.14159265358979323846264338327950288;

rte_status fail(rte_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

rte_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RTE_ERR_OOM : RTE_ERR_CUDA;
}

#define CK(x)                                                 \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x);      \
    } while (0)

#define RT(x)                                                 \
    do {                                                      \
        rte_status s_ = (x);                                  \
        if (s_ != RTE_OK) return s_;                          \
    } while (0)


// Threads of an FFT tile kernel: one per 8 elements (one radix-8 butterfly),
// a multiple of 32, at most kMaxThreads.
int threads_for(long elems) {
    long t = (elems + 7) / 8;
    t = ((t + 31) / 32) * 32;
    return (int)std::min<long>(std::max<long>(t, 64), kMaxThreads);
}

// Opt-in shared memory per block of the current device.
int smem_optin() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            v = 227 * 1024;
        return v;
    }();
    return n;
}

// The dynamic shared memory limit is an attribute of the kernel function,
// shared by every plan in the process, not of one launch. Plans driven from
// other host threads launch the same kernel with other sizes, so every caller
// raises it to the same value, the most the device allows next to the
// kernel's static shared memory; a per-launch value could be lowered by
// another thread between the set and the launch.
template <typename K> cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const size_t most = (size_t)smem_optin() - fa.sharedSizeBytes;
    if (bytes > most) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
}

bool axis_ok(int n) {
    FftPlan p;
    return n >= 4 && n <= 1024 && radix_plan(n, &p);
}

}  // namespace

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Where a plan's device memory comes from: cudaMallocAsync / cudaFreeAsync on
// the plan's stream (both null), or the caller's rte_set_allocator pair.
struct Allocator {
    rte_alloc_fn alloc = nullptr;
    rte_free_fn release = nullptr;
    void *ctx = nullptr;
};

namespace {
std::mutex g_alloc_mu;
Allocator g_alloc;   // taken by plans created from now on

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}
}  // namespace

struct rte_plan {
    rte_grid_desc d{};
    Allocator al;                   // source of every device buffer of the plan
    int M = 0;                      // stored moments: (N+1)^2, or (N+1)(N+2)/2 for real radiance
    int Mfull = 0;                  // (N+1)^2, the moments of the ABI layout
    int real = 0;                   // real-radiance layout (m >= 0 stored)
    double *mw = nullptr;           // dot-product weight of each stored moment
    size_t V = 0, n = 0, esz = 0;   // n = M V complex elements, esz = bytes per element
    cudaStream_t st = nullptr;
    double time = 0.0;
    // device state and workspace
    void *psi[2] = {nullptr, nullptr};
    int cur = 0;
    void *dz = nullptr, *t1 = nullptr;
    void *med = nullptr;
    void *dl_slot = nullptr;       // D_l per l, in the plane kernel's slot order
    void *tw[3] = {nullptr, nullptr, nullptr};
    void *tw64[2] = {nullptr, nullptr};   // FP64 x and y twiddles for the readouts
    void *kt[3] = {nullptr, nullptr, nullptr};
    int *lof = nullptr;
    void *wl = nullptr;
    CouplingRow *coup = nullptr;
    int *step = nullptr;            // step counter of the current rte_step call
    // device flags: [0] set by the step kernels on a non-finite state value,
    // [1] set by the plane kernel when a bulk copy did not complete in time
    int *flags = nullptr;
    bool nf_on = true;              // kernels check for non-finite values (off for operator applications)
    int sched = RTE_SCHED_AUTO;     // step schedule (rte_set_schedule)
    int gsteps = 2;                 // steps per captured step graph; 0 = no graphs
    // two explicit steps (psi[cur] -> psi[1-cur] -> psi[cur]) captured as one
    // CUDA graph, replayed for runs of steps; valid while gkey matches
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_st = nullptr;  // private stream the graph is recorded on
    int gkern = 0;                  // kernels in the graph
    std::vector<unsigned char> gkey;
    FftPlan fp[3];
    // host copies of the optical maps (used for the FP64 refinement operator)
    std::vector<double> mua, mus, g;
    std::vector<std::array<double, 3>> classes;
    double kmax = 0.0, dtstar = -1.0;
    // sources and detectors
    std::vector<long long> src_vox;
    std::vector<int> src_mom;
    std::vector<double> src_amp, src_t0, src_fwhm;
    std::vector<long long> det_vox;
    DevBuf inj, inj_amp, det, det_out, integ, tap_part;
    // steady-state solver
    DevBuf kry, kw, parts, dres, dcoef, rhs, kpz;
    int prec = RTE_PREC_LOW_ORDER;  // GMRES right preconditioner
    PrecLow plow{};                 // its l <= 1 block (mean medium)
    void *prec_scale = nullptr;     // its 1 / Dbar_l per stored moment (l >= 2)
    void *gfac = nullptr;           // adjoint on the plane path: interior (1 - g^l), l >= 1, slot order
    // exponential step (homogeneous media): E_k for exp_dt, [c][r][k] in tiles of 32 k
    DevBuf expE, exp_term, exp_coef, exp_dl;
    double exp_dt = -1.0;
    int exp_nterm = 0;
    rte_plan *sub = nullptr;       // FP64 twin of an FP32 plan (refinement residuals)
    DevBuf x64, r64;
    // adjoint
    int fw_nsteps = 0, fw_K = 0;
    double fw_dt = 0.0, fw_t0 = 0.0;
    std::vector<double> fw_w;      // [nsteps][ndet] gate weights
    DevBuf ckpt, rec, lam[2], fwd[2], grad_inj;
    bool fw_valid = false;
    // per-kernel event timing
    struct Pending {
        const char *name;
        cudaEvent_t a, b;
    };
    bool prof = false;
    cudaEvent_t ev_open = nullptr;
    std::vector<Pending> ev_pend;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::string> prof_names;
    std::vector<int> prof_count;
    std::vector<double> prof_ms;
};

namespace {

// All device memory of a plan is stream-ordered on the plan's stream, so that
// creating, growing and destroying one plan never waits for the work of plans
// running on other streams (cudaMalloc / cudaFree may synchronise the device).
rte_status ensure(rte_plan *p, DevBuf &b, size_t bytes);
void release(rte_plan *p, DevBuf &b);

// device memory of the plan, stream-ordered on its stream, from its allocator
cudaError_t plan_malloc(rte_plan *p, void **q, size_t bytes) {
    if (!p->al.alloc) return cudaMallocAsync(q, bytes, p->st);
    *q = p->al.alloc((uint64_t)bytes, (void *)p->st, p->al.ctx);
    return *q ? cudaSuccess : cudaErrorMemoryAllocation;
}

void plan_free(rte_plan *p, void *q) {
    if (!q) return;
    if (p->al.alloc)
        p->al.release(q, (void *)p->st, p->al.ctx);
    else
        cudaFreeAsync(q, p->st);
}

rte_status ensure(rte_plan *p, DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return RTE_OK;
    plan_free(p, b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (bytes == 0) return RTE_OK;
    CK(plan_malloc(p, &b.p, bytes));
    b.bytes = bytes;
    return RTE_OK;
}

void release(rte_plan *p, DevBuf &b) {
    plan_free(p, b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// allocate on the plan's stream and copy host data in stream order (a pageable
// source is staged before the call returns, so it may go out of scope)
rte_status upload(rte_plan *p, void **dst, const void *src, size_t bytes) {
    CK(plan_malloc(p, dst, bytes));
    CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, p->st));
    return RTE_OK;
}

template <typename R> using CT = typename cvec<R>::type;

// Per-kernel timing: when enabled, every launch is bracketed by two CUDA
// events on the plan's stream; rte_profile_read sums the intervals by name.
void prof_begin(rte_plan *p) {
    if (!p->prof) return;
    cudaEvent_t e;
    if (!p->ev_pool.empty()) {
        e = p->ev_pool.back();
        p->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, p->st);
    p->ev_open = e;
}

rte_status after_launch(rte_plan *p, const char *name) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, name);
    if (p && p->prof && p->ev_open) {
        cudaEvent_t e2;
        if (!p->ev_pool.empty()) {
            e2 = p->ev_pool.back();
            p->ev_pool.pop_back();
        } else if (cudaEventCreate(&e2) != cudaSuccess) {
            return RTE_OK;
        }
        cudaEventRecord(e2, p->st);
        p->ev_pend.push_back({name, p->ev_open, e2});
        p->ev_open = nullptr;
    }
    return RTE_OK;
}


template <typename R> int tx_of() { return sizeof(R) == 4 ? 16 : 8; }

template <typename R> Geo<R> geo(const rte_plan *p) {
    Geo<R> g;
    g.nx = p->d.nx;
    g.ny = p->d.ny;
    g.nz = p->d.nz;
    g.M = p->M;
    g.px = p->fp[0];
    g.py = p->fp[1];
    g.pz = p->fp[2];
    g.twx = (const CT<R> *)p->tw[0];
    g.twy = (const CT<R> *)p->tw[1];
    g.twz = (const CT<R> *)p->tw[2];
    g.kx = (const R *)p->kt[0];
    g.ky = (const R *)p->kt[1];
    g.kz = (const R *)p->kt[2];
    g.nonfinite = p->nf_on ? p->flags : nullptr;
    return g;
}

template <typename R> XArgs<R> xargs_plain(const rte_plan *p) {
    XArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.med = (const typename Media4<R>::type *)p->med;
    a.lof = p->lof;
    a.wl = (const R *)p->wl;
    return a;
}

// ---------------------------------------------------------------- launchers

// Columns per z/y tile: 16 (FP32) or 8 (FP64) consecutive x, halved until
// the two ping-pong tiles fit in 200 KB of shared memory.
template <typename R> int tile_cols(int n) {
    int TX = sizeof(R) == 4 ? 16 : 8;
    while (TX > 1 && 2 * (size_t)n * (TX + 1) * sizeof(CT<R>) > 200 * 1024) TX /= 2;
    return TX;
}

// Fixed-size kernels exist for axes of 32, 64, 96, 128 and 160 points
// (two-phase transforms 4x8, 8x8, 12x8, 16x8, 20x8) and, for the z pass
// only, 256 points (16x16); other lengths use the runtime Stockham passes.
template <typename R, int N1, int N2> rte_status launch_zderiv_fixed(rte_plan *p, const void *in, void *out) {
    constexpr int TX = sizeof(R) == 4 ? 16 : 8, NT = 128;
    dim3 grid((p->d.nx + TX - 1) / TX, p->d.ny, p->M);
    prof_begin(p);
    k_zderiv_fixed<R, N1, N2, TX, NT><<<grid, NT, 0, p->st>>>((const CT<R> *)in, (CT<R> *)out, geo<R>(p));
    return after_launch(p, "k_zderiv(fixed)");
}

template <typename R> rte_status launch_zderiv(rte_plan *p, const void *in, void *out) {
    switch (p->d.nz) {
        case 32: return launch_zderiv_fixed<R, 4, 8>(p, in, out);
        case 64: return launch_zderiv_fixed<R, 8, 8>(p, in, out);
        case 96: return launch_zderiv_fixed<R, 12, 8>(p, in, out);
        case 128: return launch_zderiv_fixed<R, 16, 8>(p, in, out);
        case 160: return launch_zderiv_fixed<R, 20, 8>(p, in, out);
        case 256: return launch_zderiv_fixed<R, 16, 16>(p, in, out);
        default: break;
    }
    const int TX = tile_cols<R>(p->d.nz);
    const long elems = (long)p->d.nz * TX;
    const int nthr = threads_for(elems);
    const size_t smem = 2 * (size_t)p->d.nz * (TX + 1) * sizeof(CT<R>);
    dim3 grid((p->d.nx + TX - 1) / TX, p->d.ny, p->M);
    CK(allow_smem(k_zderiv<R>, smem));
    prof_begin(p);
    k_zderiv<R><<<grid, nthr, smem, p->st>>>((const CT<R> *)in, (CT<R> *)out, geo<R>(p), TX);
    return after_launch(p, "k_zderiv");
}

// fixed-size line passes (split schedule) for these axis lengths
template <typename F> rte_status with_line_split(int n, F f) {
    switch (n) {
        case 32: return f(std::integral_constant<int, 4>{}, std::integral_constant<int, 8>{});
        case 64: return f(std::integral_constant<int, 8>{}, std::integral_constant<int, 8>{});
        case 96: return f(std::integral_constant<int, 12>{}, std::integral_constant<int, 8>{});
        case 128: return f(std::integral_constant<int, 16>{}, std::integral_constant<int, 8>{});
        case 160: return f(std::integral_constant<int, 20>{}, std::integral_constant<int, 8>{});
        default: return f(std::integral_constant<int, 16>{}, std::integral_constant<int, 16>{});
    }
}
bool line_fixed(int n) { return n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 256; }

template <typename R>
rte_status launch_ypass(rte_plan *p, const void *in, void *out, int inverse, const void *psi_in, const void *dz,
                        double a, double coefS) {
    if (line_fixed(p->d.ny)) {
        return with_line_split(p->d.ny, [&](auto n1, auto n2) -> rte_status {
            constexpr int N1 = decltype(n1)::value, N2 = decltype(n2)::value;
            constexpr int TX = sizeof(R) == 4 ? 16 : 8, NT = TX * N2;
            dim3 grid(p->M, (p->d.nx + TX - 1) / TX, p->d.nz);
            prof_begin(p);
            if (psi_in && !inverse)
                k_ypass_fixed<R, N1, N2, TX, NT, 1><<<grid, NT, 0, p->st>>>(
                    (const CT<R> *)in, (CT<R> *)out, geo<R>(p), 0, (const CT<R> *)psi_in, (const CT<R> *)dz, (R)a,
                    (R)coefS, p->coup);
            else
                k_ypass_fixed<R, N1, N2, TX, NT, 0><<<grid, NT, 0, p->st>>>(
                    (const CT<R> *)in, (CT<R> *)out, geo<R>(p), inverse, nullptr, nullptr, (R)0, (R)0, p->coup);
            return after_launch(p, inverse ? "k_ypass_fixed(inverse)"
                                           : (psi_in ? "k_ypass_fixed(forward+coupling)" : "k_ypass_fixed(forward)"));
        });
    }
    const int TX = tile_cols<R>(p->d.ny);
    const long elems = (long)p->d.ny * TX;
    const int nthr = threads_for(elems);
    const size_t smem = 2 * (size_t)p->d.ny * (TX + 1) * sizeof(CT<R>);
    dim3 grid((p->d.nx + TX - 1) / TX, p->d.nz, p->M);
    CK(allow_smem(k_ypass<R>, smem));
    prof_begin(p);
    k_ypass<R><<<grid, nthr, smem, p->st>>>((const CT<R> *)in, (CT<R> *)out, geo<R>(p), TX, inverse,
                                            (const CT<R> *)psi_in, (const CT<R> *)dz, (R)a, (R)coefS, p->coup);
    return after_launch(p, inverse ? "k_ypass(inverse)" : (psi_in ? "k_ypass(forward+coupling)" : "k_ypass(forward)"));
}

// Moments per X-pass CTA: as many as fit two ping-pong tiles in 96 KB,
// spread evenly over the chunks.
template <typename R> int xpass_moments(const rte_plan *p, int *nchunks) {
    const size_t line = 2 * (size_t)(p->d.nx + 1) * sizeof(CT<R>);
    int maxmc = (int)std::max<size_t>(1, (96 * 1024) / line);
    maxmc = std::min(maxmc, p->M);
    const int nch = (p->M + maxmc - 1) / maxmc;
    *nchunks = nch;
    return (p->M + nch - 1) / nch;
}

int num_sms();

template <typename R> rte_status launch_xpass(rte_plan *p, const void *in, void *out, const XArgs<R> &xa) {
    if (line_fixed(p->d.nx) && xa.inv_in && xa.pointwise && xa.fwd_out && !xa.grad_a && !xa.rec_in) {
        return with_line_split(p->d.nx, [&](auto n1, auto n2) -> rte_status {
            constexpr int N1 = decltype(n1)::value, N2 = decltype(n2)::value, NX = N1 * N2;
            // moments per CTA: rows of all of them within 40 KB of static shared memory
            constexpr int MCmax = (int)(40960 / ((NX + NX / N2 + 1) * sizeof(CT<R>)));
            constexpr int MC = MCmax < 32 ? MCmax : 32, NT = 256;
            const int nch = (p->M + MC - 1) / MC, mcs = (p->M + nch - 1) / nch;   // even chunks
            const int items = p->d.ny * p->d.nz * nch;
            const int tasks = mcs * std::max(N1, N2);
            const int nthr = std::min(NT, (tasks + 31) / 32 * 32);                 // one task per thread
            const size_t smem = (size_t)mcs * (NX + NX / N2 + 1) * sizeof(CT<R>);
            CK(allow_smem(k_xpass_fixed<R, N1, N2, MC, NT>, smem));
            // persistent: exactly the CTAs that are resident at once
            int per_sm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xpass_fixed<R, N1, N2, MC, NT>, nthr, smem));
            const int grid = std::min(items, num_sms() * std::max(1, per_sm));
            prof_begin(p);
            k_xpass_fixed<R, N1, N2, MC, NT><<<grid, nthr, smem, p->st>>>((const CT<R> *)in, (CT<R> *)out, geo<R>(p), mcs,
                                                                     xa);
            return after_launch(p, "k_xpass_fixed(pointwise)");
        });
    }
    int nch;
    const int MC = xpass_moments<R>(p, &nch);
    const long elems = (long)MC * p->d.nx;
    const int nthr = threads_for(elems);
    const size_t smem = 2 * (size_t)MC * (p->d.nx + 1) * sizeof(CT<R>);
    dim3 grid(p->d.ny, p->d.nz, nch);
    CK(allow_smem(k_xpass<R>, smem));
    prof_begin(p);
    k_xpass<R><<<grid, nthr, smem, p->st>>>((const CT<R> *)in, (CT<R> *)out, geo<R>(p), MC, xa);
    return after_launch(p, xa.pointwise ? "k_xpass(pointwise)" : "k_xpass(transform)");
}

template <typename R> rte_status launch_advance(rte_plan *p, const void *psi_t, double *integral, int delta) {
    const double vol = p->d.dx_mm * p->d.dx_mm * p->d.dx_mm;
    prof_begin(p);
    k_advance<R><<<1, 32, 0, p->st>>>((const CT<R> *)psi_t, p->d.nx, p->d.ny, p->d.nz, p->step, integral, vol, delta);
    return after_launch(p, "k_advance");
}

// ---------------------------------------------------------------- fused plane kernel

// nz for which the z-streaming pass k_zstream is instantiated
bool zstream_ok(int nz) { return nz == 32 || nz == 64 || nz == 96 || nz == 128 || nz == 160 || nz == 256; }

template <typename R> size_t plane_smem(int nx, int ny) { return plane_smem_bytes<R>(nx, ny); }

// xy planes the fused plane kernel is instantiated for: any pair of 32, 64,
// 128, and the square 96 x 96 and 160 x 160 planes
bool plane_shape_ok(int nx, int ny) {
    auto pow2 = [](int n) { return n == 32 || n == 64 || n == 128; };
    return (pow2(nx) && pow2(ny)) || (nx == ny && (nx == 96 || nx == 160));
}

int num_sms() {
    // initialised once, thread-safely: plans may be driven from several host threads
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        return v;
    }();
    return n;
}

// the plane and its twiddles must fit one CTA's shared memory; in FP64 the
// BX- and BY-point register DFTs are kept to 16 points (64 registers)
template <typename R> bool plane_fits(int nx, int ny) {
    if (sizeof(R) == 8 && (nx > 64 || ny > 64)) return false;
    return plane_shape_ok(nx, ny) && plane_smem<R>(nx, ny) <= 220 * 1024;
}

template <typename R> bool plane_ok(const rte_plan *p) {
    return p->dl_slot && plane_fits<R>(p->d.nx, p->d.ny) && zstream_ok(p->d.nz);
}

// the fused plane path runs where it fits unless the split schedule is chosen
template <typename R> bool use_plane(const rte_plan *p) { return p->sched != RTE_SCHED_SPLIT && plane_ok<R>(p); }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// Tensor map of a state buffer for the plane kernel's row copies: rows x
// units 8-byte elements (a complex64 is one unit, a complex128 two) with
// rows of `units` elements, read in boxes of `box_units` x kRowsPerCopy; box
// columns past a row's end lie outside the array and are filled with zeros.
rte_status encode_rows_map(CUtensorMap *map, const void *base, int units, long long rows, int box_units) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(RTE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {(cuuint64_t)units, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)units * 8};
    const cuuint32_t box[2] = {(cuuint32_t)box_units, (cuuint32_t)kRowsPerCopy};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(RTE_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    return RTE_OK;
}

template <typename R, int NX, int NY, int MODE>
rte_status launch_plane_m(rte_plan *p, const PlaneArgs<R> &pa_in) {
    // the row copies of every plan's psi_in
    PlaneArgs<R> pa = pa_in;
    constexpr int units = (int)(sizeof(CT<R>) / 8);
    for (int i = 0; i < pa.nplans; ++i)
        RT(encode_rows_map(&pa.pl[i].rows_map, pa.pl[i].psi_in, NX * units, (long long)pa.M * pa.nz * NY,
                           plane_pitch<R, NX>() * units));
    // threads: the larger of the y-column tasks (NX * SY) and the x-row tasks
    // (4 NY), at most 512; 64 x 64 planes take 256 (two CTAs per SM), 160 x 160
    // planes 320 (their 40-point register DFTs need more registers per thread)
    constexpr int ta = NX * plane_sy(NY), tb = 4 * NY, tmax = ta > tb ? ta : tb;
    constexpr int NT = (NX == 160) ? 320 : (NX == 64 && NY == 64) ? 256 : (tmax < 512 ? tmax : 512);
    constexpr int MINB = sizeof(R) == 8 ? (NT <= 128 ? 2 : 1) : (NT <= 128 ? 4 : NT <= 256 ? 2 : 1);
    const size_t smem = plane_smem_launch<R>(NX, NY, MINB);
    auto kern = k_plane<R, NX, NY, NT, MINB, MODE>;
    CK(allow_smem(kern, smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const int items = p->M * p->d.nz * pa.nplans;
    const int grid = std::min(items, num_sms() * std::max(1, per_sm));
    prof_begin(p);
    kern<<<grid, NT, smem, p->st>>>(pa);
    return after_launch(p, "k_plane");
}

// plain step / operator (MODE 0), forward segment with the real-space record
// (1), adjoint step with the gradient terms (2)
template <typename R, int NX, int NY>
rte_status launch_plane_t(rte_plan *p, const PlaneArgs<R> &pa) {
    if (pa.rec_in) return launch_plane_m<R, NX, NY, 2>(p, pa);
    if (pa.rec_out) return launch_plane_m<R, NX, NY, 1>(p, pa);
    return launch_plane_m<R, NX, NY, 0>(p, pa);
}

template <typename R, int NX>
rte_status launch_plane_y(rte_plan *p, const PlaneArgs<R> &pa) {
    switch (p->d.ny) {
        case 32: return launch_plane_t<R, NX, 32>(p, pa);
        case 64: return launch_plane_t<R, NX, 64>(p, pa);
        default: return launch_plane_t<R, NX, 128>(p, pa);
    }
}

// the plane pass for the plans in pa (their buffers already set)
template <typename R> rte_status launch_plane_args(rte_plan *p, const PlaneArgs<R> &pa) {
    if constexpr (sizeof(R) == 8) {
        // FP64 planes: 32 and 64 points per axis (plane_fits)
        switch (p->d.nx) {
            case 32: return p->d.ny == 32 ? launch_plane_t<R, 32, 32>(p, pa) : launch_plane_t<R, 32, 64>(p, pa);
            default: return p->d.ny == 32 ? launch_plane_t<R, 64, 32>(p, pa) : launch_plane_t<R, 64, 64>(p, pa);
        }
    } else {
        switch (p->d.nx) {
            case 32: return launch_plane_y<R, 32>(p, pa);
            case 64: return launch_plane_y<R, 64>(p, pa);
            case 96: return launch_plane_t<R, 96, 96>(p, pa);
            case 160: return launch_plane_t<R, 160, 160>(p, pa);
            default: return launch_plane_y<R, 128>(p, pa);
        }
    }
}

// the plane pass of one plan: psi~ in `in`, w in `w`, result in `out`
template <typename R>
rte_status launch_plane(rte_plan *p, const void *in, const void *w, void *out, const PlaneArgs<R> &pa) {
    PlaneArgs<R> q = pa;
    q.nplans = 1;
    q.pl[0].psi_in = (const CT<R> *)in;
    q.pl[0].win = (const CT<R> *)w;
    q.pl[0].out = (CT<R> *)out;
    return launch_plane_args<R>(p, q);
}

// w = a psi~ + coefS S~(psi~) for the plane kernel (fixed nz only: zstream_ok).
// x tiles of 32 columns in FP32 (4 CTAs of 256 threads per SM at 64
// registers), 8 in FP64.
template <typename R, int N1, int N2, int G = 0>
rte_status launch_zstream_t(rte_plan *p, ZArgs<R> za) {
    constexpr int TX = sizeof(R) == 4 ? 32 : 8, NT = TX * N2;
    za.nxt = (p->d.nx + TX - 1) / TX;
    dim3 grid(p->M, za.nxt * za.nplans, p->d.ny);
    prof_begin(p);
    k_zstream<R, N1, N2, TX, NT, G, G><<<grid, NT, 0, p->st>>>(za, geo<R>(p), p->coup);
    return after_launch(p, "k_zstream");
}

// w = a psi~ + coefS S~(psi~) for the plans in za (fixed nz only: zstream_ok).
// Cubic grids of the common sizes take the instance with compile-time plane
// extents (constant operand offsets: fewer instructions per element).
template <typename R> rte_status launch_zstream_args(rte_plan *p, const ZArgs<R> &za) {
    const bool cube = p->d.nx == p->d.nz && p->d.ny == p->d.nz;
    switch (p->d.nz) {
        case 32: return cube ? launch_zstream_t<R, 4, 8, 32>(p, za) : launch_zstream_t<R, 4, 8>(p, za);
        case 64: return cube ? launch_zstream_t<R, 8, 8, 64>(p, za) : launch_zstream_t<R, 8, 8>(p, za);
        case 96:
            if constexpr (sizeof(R) == 4)
                if (cube) return launch_zstream_t<R, 12, 8, 96>(p, za);
            return launch_zstream_t<R, 12, 8>(p, za);
        case 128:
            if constexpr (sizeof(R) == 4)
                if (cube) return launch_zstream_t<R, 16, 8, 128>(p, za);
            return launch_zstream_t<R, 16, 8>(p, za);
        case 160:
            if constexpr (sizeof(R) == 4)
                if (cube) return launch_zstream_t<R, 20, 8, 160>(p, za);
            return launch_zstream_t<R, 20, 8>(p, za);
        case 256: return launch_zstream_t<R, 16, 16>(p, za);
        default: return fail(RTE_ERR_UNSUPPORTED, "k_zstream: nz has no fixed-size transform");
    }
}

template <typename R> rte_status launch_zstream(rte_plan *p, const void *in, void *out, double a, double coefS) {
    ZArgs<R> za;
    std::memset(&za, 0, sizeof(za));
    za.nplans = 1;
    za.in[0] = (const CT<R> *)in;
    za.out[0] = (CT<R> *)out;
    za.a[0] = (R)a;
    za.coefS[0] = (R)coefS;
    return launch_zstream_args<R>(p, za);
}

template <typename R> PlaneArgs<R> plane_args(const rte_plan *p, double coefD, double a, double coefS) {
    PlaneArgs<R> pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.nz = p->d.nz;
    pa.M = p->M;
    pa.nplans = 1;
    pa.a = (R)a;
    pa.coefS = (R)coefS;
    pa.twx = (const CT<R> *)p->tw[0];
    pa.twy = (const CT<R> *)p->tw[1];
    pa.lof = p->lof;
    PlanePlan<R> &q = pa.pl[0];
    q.win = (const CT<R> *)p->dz;
    q.dl_slot = (const R *)p->dl_slot;
    q.coefD = (R)coefD;
    q.nonfinite = p->nf_on ? p->flags : nullptr;
    q.status = p->flags + 1;
    return pa;
}

// real-space field (ABI layout) in `buf` -> psi~ in `out` (buf is overwritten)
template <typename R> rte_status to_tilde(rte_plan *p, void *buf, void *out) {
    XArgs<R> xa = xargs_plain<R>(p);
    xa.fwd_out = 1;
    RT(launch_xpass<R>(p, buf, buf, xa));
    return launch_ypass<R>(p, buf, out, 0, nullptr, nullptr, 0.0, 0.0);
}

// psi~ in `in` -> real-space field in `out` via `buf` (buf may equal out)
template <typename R> rte_status from_tilde(rte_plan *p, const void *in, void *buf, void *out) {
    RT(launch_ypass<R>(p, in, buf, 1, nullptr, nullptr, 0.0, 0.0));
    XArgs<R> xa = xargs_plain<R>(p);
    xa.inv_in = 1;
    return launch_xpass<R>(p, buf, out, xa);
}

// Operator applications leave the non-finite flag alone: it reports the
// state of the time-stepping calls only.
struct FlagOff {
    rte_plan *p;
    bool f;
    explicit FlagOff(rte_plan *q) : p(q), f(q->nf_on) { q->nf_on = false; }
    ~FlagOff() { p->nf_on = f; }
};

// out~ = T in~ (sgn = +1) or (-S + D) in~ (sgn = -1); uses dz and t1; out may be t1.
template <typename R> rte_status apply_T_tilde(rte_plan *p, const void *in, void *out, double sgn) {
    FlagOff off(p);
    if (use_plane<R>(p)) {
        RT(launch_zstream<R>(p, in, p->dz, 0.0, sgn));
        return launch_plane<R>(p, in, p->dz, out, plane_args<R>(p, 1.0, 0.0, sgn));
    }
    RT(launch_zderiv<R>(p, in, p->dz));
    RT(launch_ypass<R>(p, in, p->t1, 1, nullptr, nullptr, 0.0, 0.0));
    XArgs<R> xa = xargs_plain<R>(p);
    xa.inv_in = 1;
    xa.pointwise = 1;
    xa.fwd_out = 1;
    xa.coefD = (R)1;
    RT(launch_xpass<R>(p, p->t1, p->t1, xa));
    return launch_ypass<R>(p, p->t1, out, 0, in, p->dz, 0.0, sgn);
}

// out = P^-1 in, the GMRES right preconditioner (in, out: psi~ vectors of the
// plan's layout; they may not alias)
template <typename R> rte_status apply_prec(rte_plan *p, const void *in, void *out) {
    const int per = (int)std::max<size_t>(1, std::min<size_t>((p->V + 255) / 256, std::max(1, num_sms() * 8 / p->M)));
    prof_begin(p);
    k_scale_moments<R><<<dim3(per, p->M), 256, 0, p->st>>>((const CT<R> *)in, (CT<R> *)out, p->V,
                                                          (const R *)p->prec_scale);
    RT(after_launch(p, "k_scale_moments"));
    if (p->d.N < 1) return RTE_OK;
    int TX = sizeof(R) == 4 ? 8 : 4;
    while (TX > 1 && 2 * (size_t)p->d.nz * (4 * TX + 1) * sizeof(CT<R>) > 200 * 1024) TX /= 2;
    const size_t smem = 2 * (size_t)p->d.nz * (4 * TX + 1) * sizeof(CT<R>);
    const int nthr = threads_for((long)p->d.nz * 4 * TX);
    CK(allow_smem(k_prec_low<R>, smem));
    prof_begin(p);
    k_prec_low<R><<<dim3((p->d.nx + TX - 1) / TX, p->d.ny), nthr, smem, p->st>>>(
        (const CT<R> *)in, (CT<R> *)out, geo<R>(p), TX, p->real, p->plow);
    return after_launch(p, "k_prec_low");
}

// weighted dot products res[i] = <B_i, w> (FP64, to host)
template <typename R>
rte_status wdots(rte_plan *p, const void *basis, int ncolb, const void *w, double *out /* 2*(ncolb+self) */,
                 int self = 0) {
    const int ncol = ncolb + self;   // with self, the last result is |w|^2
    const int nthr = 256;
    const size_t smem = (size_t)ncol * 32 * sizeof(double2);
    CK(allow_smem(k_wdot_multi<R>, smem));
    // one wave: as many CTAs as are resident at once (4 per SM in FP32),
    // shared out over the moments
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_wdot_multi<R>, nthr, smem));
    const int per_m = (int)std::max<size_t>(1, std::min<size_t>((p->V + nthr - 1) / nthr,
                                                                std::max(1, num_sms() * std::max(occ, 1) / p->M)));
    const int nblk = per_m * p->M;
    RT(ensure(p, p->parts, (size_t)nblk * ncol * sizeof(double2)));
    RT(ensure(p, p->dres, (size_t)std::max(ncol, 64) * sizeof(double2)));
    prof_begin(p);
    k_wdot_multi<R><<<dim3(per_m, p->M), nthr, smem, p->st>>>((const CT<R> *)basis, p->n, ncolb, ncol,
                                                              (const CT<R> *)w, p->V, p->mw, (double2 *)p->parts.p);
    RT(after_launch(p, "k_wdot_multi"));
    prof_begin(p);
    k_sum_parts<<<ncol, 256, 0, p->st>>>((const double2 *)p->parts.p, nblk, ncol, (double2 *)p->dres.p);
    RT(after_launch(p, "k_sum_parts"));
    CK(cudaMemcpyAsync(out, p->dres.p, (size_t)ncol * sizeof(double2), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    // real radiance: the full inner product of two real-radiance fields is real
    if (p->real)
        for (int c = 0; c < ncol; ++c) out[2 * c + 1] = 0.0;
    return RTE_OK;
}

template <typename R> rte_status wnorm(rte_plan *p, const void *v, double *nrm) {
    double d[2];
    RT(wdots<R>(p, v, 1, v, d));
    *nrm = std::sqrt(std::max(d[0], 0.0));
    return RTE_OK;
}

int vec_grid(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 148 * 8); }

template <typename R, typename Q>
rte_status axpby(rte_plan *p, const void *x, void *y, double ar, double ai, double br, double bi) {
    prof_begin(p);
    k_axpby<R, Q><<<vec_grid(p->n), 256, 0, p->st>>>((const CT<Q> *)x, (CT<R> *)y, p->n, ar, ai, br, bi);
    return after_launch(p, "k_axpby");
}

// out = scale (w - sum_i h_i B_i); out may be w
template <typename R>
rte_status sub_multi(rte_plan *p, const void *basis, int ncol, const double *h, void *w, void *out = nullptr,
                     double scale = 1.0) {
    RT(ensure(p, p->dcoef, (size_t)std::max(ncol, 64) * sizeof(double2)));
    CK(cudaMemcpyAsync(p->dcoef.p, h, (size_t)ncol * sizeof(double2), cudaMemcpyHostToDevice, p->st));
    prof_begin(p);
    k_sub_multi<R><<<vec_grid(p->n), 256, 0, p->st>>>((const CT<R> *)basis, p->n, ncol,
                                                      (const double2 *)p->dcoef.p, (const CT<R> *)w,
                                                      (CT<R> *)(out ? out : w), (R)scale);
    RT(after_launch(p, "k_sub_multi"));
    CK(cudaStreamSynchronize(p->st));   // h lives on the host stack of the caller
    return RTE_OK;
}

template <typename R> rte_status add_multi(rte_plan *p, const void *basis, int ncol, const double *c, void *y) {
    RT(ensure(p, p->dcoef, (size_t)std::max(ncol, 64) * sizeof(double2)));
    CK(cudaMemcpyAsync(p->dcoef.p, c, (size_t)ncol * sizeof(double2), cudaMemcpyHostToDevice, p->st));
    prof_begin(p);
    k_add_multi<R, R><<<vec_grid(p->n), 256, 0, p->st>>>((const CT<R> *)basis, p->n, ncol,
                                                         (const double2 *)p->dcoef.p, (CT<R> *)y);
    RT(after_launch(p, "k_add_multi"));
    CK(cudaStreamSynchronize(p->st));
    return RTE_OK;
}

// ---------------------------------------------------------------- sources

// int4 (x, y, z, moment) of a flat voxel index
int4 voxel4(const rte_plan *p, long long v, int w) {
    const int nx = p->d.nx, ny = p->d.ny;
    int4 r;
    r.x = (int)(v % nx);
    r.y = (int)((v / nx) % ny);
    r.z = (int)(v / ((long long)nx * ny));
    r.w = w;
    return r;
}

double source_density(double t, double amp, double t0, double fwhm, double dx) {
    const double vol = dx * dx * dx;
    if (fwhm <= 0.0) return amp / vol;
    const double u = (t - t0) / fwhm;
    return amp * std::exp(-4.0 * std::log(2.0) * u * u) / vol;
}

// Upload injections: amp[s][q] for s < nsteps, points (voxel, moment).
template <typename R>
rte_status upload_injections(rte_plan *p, const std::vector<int4> &pts, const std::vector<double> &amp, int nsteps) {
    const int ninj = (int)pts.size();
    if (ninj == 0) return RTE_OK;
    RT(ensure(p, p->inj, (size_t)ninj * sizeof(int4)));
    RT(ensure(p, p->inj_amp, (size_t)nsteps * ninj * sizeof(R)));
    std::vector<R> a(amp.size());
    for (size_t i = 0; i < amp.size(); ++i) a[i] = (R)amp[i];
    CK(cudaMemcpyAsync(p->inj.p, pts.data(), (size_t)ninj * sizeof(int4), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemcpyAsync(p->inj_amp.p, a.data(), a.size() * sizeof(R), cudaMemcpyHostToDevice, p->st));
    CK(cudaStreamSynchronize(p->st));
    return RTE_OK;
}

template <typename R> rte_status upload_sources(rte_plan *p, double dt, int nsteps, double t0) {
    const int ns = (int)p->src_vox.size();
    std::vector<int4> pts(ns);
    std::vector<double> amp((size_t)nsteps * ns);
    const double cdt = p->d.c_mm_per_ps * dt;
    for (int q = 0; q < ns; ++q) pts[q] = voxel4(p, p->src_vox[q], p->src_mom[q]);
    for (int s = 0; s < nsteps; ++s)
        for (int q = 0; q < ns; ++q)
            amp[(size_t)s * ns + q] =
                cdt * source_density(t0 + s * dt, p->src_amp[q], p->src_t0[q], p->src_fwhm[q], p->d.dx_mm);
    return upload_injections<R>(p, pts, amp, nsteps);
}

template <typename R> rte_status upload_detectors(rte_plan *p) {
    const int nd = (int)p->det_vox.size();
    if (nd == 0) return RTE_OK;
    std::vector<int4> pts(nd);
    for (int d = 0; d < nd; ++d) pts[d] = voxel4(p, p->det_vox[d], 0);
    RT(ensure(p, p->det, (size_t)nd * sizeof(int4)));
    CK(cudaMemcpyAsync(p->det.p, pts.data(), (size_t)nd * sizeof(int4), cudaMemcpyHostToDevice, p->st));
    CK(cudaStreamSynchronize(p->st));
    return RTE_OK;
}

// One explicit step of Eq. 11 on psi[cur] -> psi[1-cur] (or, for the adjoint
// sweep, of the reversed-streaming step): Z, Y^-1, X (pointwise), Y+ and the
// step-end kernel.
template <typename R>
rte_status one_step(rte_plan *p, void *A, void *B, double cdt, double sgn, const XArgs<R> &xa, double *integral,
                    int delta) {
    RT(launch_zderiv<R>(p, A, p->dz));
    RT(launch_ypass<R>(p, A, p->t1, 1, nullptr, nullptr, 0.0, 0.0));
    RT(launch_xpass<R>(p, p->t1, p->t1, xa));
    RT(launch_ypass<R>(p, p->t1, B, 0, A, p->dz, 1.0, -cdt * sgn));
    return launch_advance<R>(p, A, integral, delta);
}

// ---------------------------------------------------------------- step graphs

// Step graphs are used unless per-kernel profiling is on (its events would
// be captured too) or RTE_NO_GRAPHS is set in the environment.
bool graphs_enabled(const rte_plan *p) {
    static const bool off = [] {
        const char *e = std::getenv("RTE_NO_GRAPHS");
        return e && *e && *e != '0';
    }();
    return !off && !p->prof;
}

template <typename T> void key_append(std::vector<unsigned char> &k, const T &v) {
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&v);
    k.insert(k.end(), b, b + sizeof(T));
}

// (Re)capture p->gexec from `record` (which launches on p->st) unless the
// cached graph was captured with the same key. The launches are recorded on
// a private stream (the plan's own may be the legacy default stream, which
// cannot be captured); the graph is then launched on the plan's stream.
// Capture is thread-local, so plans on other host threads keep running and
// allocating meanwhile.
template <typename F> rte_status ensure_step_graph(rte_plan *p, const std::vector<unsigned char> &key, F record) {
    if (p->gexec && p->gkey == key) return RTE_OK;
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    if (!p->cap_st) CK(cudaStreamCreateWithFlags(&p->cap_st, cudaStreamNonBlocking));
    cudaStream_t own = p->st;
    p->st = p->cap_st;
    cudaError_t e = cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        p->st = own;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    const int cur0 = p->cur;
    const rte_status rs = record();
    p->cur = cur0;    // capturing ran no step
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->st, &g);
    p->st = own;
    if (rs != RTE_OK) {
        if (g) cudaGraphDestroy(g);
        return rs;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    // every launch recorded went through after_launch, which counted it as
    // executed: take the graph's kernel nodes back off the counter
    size_t nn = 0;
    cudaError_t ei = cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (ei == cudaSuccess && nn) ei = cudaGraphGetNodes(g, nodes.data(), &nn);
    int nk = 0;
    for (size_t i = 0; ei == cudaSuccess && i < nn; ++i) {
        cudaGraphNodeType t;
        ei = cudaGraphNodeGetType(nodes[i], &t);
        if (ei == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    if (ei == cudaSuccess) ei = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        p->gexec = nullptr;
        return cuda_fail(ei, "step graph");
    }
    g_launches.fetch_sub((uint64_t)nk, std::memory_order_relaxed);
    p->gkern = nk;
    p->gkey = key;
    return RTE_OK;
}

// One explicit step with the fused plane kernel: z streaming (w = a psi~ +
// coefS S~ into the dz buffer), plane, readouts, step end.
template <typename R> PlaneArgs<R> plane_args_step(rte_plan *p, double cdt, int with_det) {
    PlaneArgs<R> pa = plane_args<R>(p, -cdt, 1.0, -cdt);
    pa.pl[0].step = p->step;
    if (with_det && !p->det_vox.empty()) {
        pa.ndet = (int)p->det_vox.size();
        pa.det = (const int4 *)p->det.p;
        pa.det_out = (double *)p->det_out.p;
    }
    if (!p->src_vox.empty()) {
        pa.pl[0].ninj = (int)p->src_vox.size();
        pa.pl[0].inj = (const int4 *)p->inj.p;
        pa.pl[0].inj_amp = (const R *)p->inj_amp.p;
    }
    return pa;
}

template <typename R>
rte_status plane_step(rte_plan *p, void *A, void *B, const PlaneArgs<R> &pa, double *integral, int delta = 1) {
    RT(launch_zstream<R>(p, A, p->dz, (double)pa.a, (double)pa.coefS));
    RT(launch_plane<R>(p, A, p->dz, B, pa));
    if (pa.ndet > 0) {
        RT(ensure(p, p->tap_part, (size_t)pa.ndet * kTapChunks * sizeof(double)));   // sized before any capture
        prof_begin(p);
        k_taps<R><<<dim3(pa.ndet, kTapChunks), 128, 0, p->st>>>((const CT<R> *)A, p->d.nx, p->d.ny,
                                                               (const double2 *)p->tw64[0], (const double2 *)p->tw64[1],
                                                               pa.det, (double *)p->tap_part.p);
        RT(after_launch(p, "k_taps"));
        prof_begin(p);
        k_taps_finish<<<(pa.ndet + 127) / 128, 128, 0, p->st>>>((const double *)p->tap_part.p, pa.ndet,
                                                               1.0 / ((double)p->d.nx * p->d.ny), p->step,
                                                               pa.det_out);
        RT(after_launch(p, "k_taps_finish"));
    }
    return launch_advance<R>(p, A, integral, delta);
}

// The plane kernel keeps at most kMaxItemInj injections per (moment, plane).
bool injections_fit_plane(const rte_plan *p, const std::vector<long long> &vox, const std::vector<int> &mom) {
    const long long plane = (long long)p->d.nx * p->d.ny;
    for (size_t i = 0; i < vox.size(); ++i) {
        int same = 0;
        for (size_t j = 0; j < vox.size(); ++j)
            if (mom[j] == mom[i] && vox[j] / plane == vox[i] / plane) ++same;
        if (same > kMaxItemInj) return false;
    }
    return true;
}

template <typename R> XArgs<R> xargs_step(rte_plan *p, double cdt, int with_det) {
    XArgs<R> xa = xargs_plain<R>(p);
    xa.inv_in = 1;
    xa.pointwise = 1;
    xa.fwd_out = 1;
    xa.coefD = (R)(-cdt);
    xa.step = p->step;
    if (with_det && !p->det_vox.empty()) {
        xa.ndet = (int)p->det_vox.size();
        xa.det = (const int4 *)p->det.p;
        xa.det_out = (double *)p->det_out.p;
    }
    if (!p->src_vox.empty()) {
        xa.ninj = (int)p->src_vox.size();
        xa.inj = (const int4 *)p->inj.p;
        xa.inj_amp = (const R *)p->inj_amp.p;
    }
    return xa;
}

rte_status check_dt(rte_plan *p, double dt, int allow_unstable);

// Steps between checks of the non-finite flag inside one rte_step call.
constexpr int kFiniteCheckSteps = 1024;

// Report (and clear) a non-finite state value flagged by the step kernels.
// Synchronises the plan's stream; not called under stream capture.
rte_status check_finite(rte_plan *p) {
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, p->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    if (!h[0] && !h[1]) return RTE_OK;
    CK(cudaMemsetAsync(p->flags, 0, 2 * sizeof(int), p->st));
    if (h[1]) return fail(RTE_ERR_TIMEOUT, "a bulk copy into shared memory did not complete in time; the step was "
                                           "abandoned and the state is not valid");
    return fail(RTE_ERR_NONFINITE,
                "the state holds a non-finite value (a step beyond the stability limit, or a NaN or Inf in the "
                "state or the sources)");
}

template <typename R>
rte_status step_impl(rte_plan *p, double dt, int nsteps, int allow_unstable, double *det_series, double *integral) {
    RT(check_dt(p, dt, allow_unstable));
    if (nsteps == 0) return RTE_OK;
    const double cdt = p->d.c_mm_per_ps * dt;
    RT(upload_sources<R>(p, dt, nsteps, p->time));
    const int nd = (int)p->det_vox.size();
    const bool want_det = det_series && nd > 0;
    if (want_det) {
        RT(upload_detectors<R>(p));
        RT(ensure(p, p->det_out, (size_t)nsteps * nd * sizeof(double)));
    }
    if (integral) RT(ensure(p, p->integ, (size_t)nsteps * 2 * sizeof(double)));
    CK(cudaMemsetAsync(p->step, 0, sizeof(int), p->st));
    XArgs<R> xa = xargs_step<R>(p, cdt, want_det);
    const bool fast = use_plane<R>(p) && injections_fit_plane(p, p->src_vox, p->src_mom);
    const PlaneArgs<R> pa = plane_args_step<R>(p, cdt, want_det);
    double *integ = integral ? (double *)p->integ.p : nullptr;
    if (fast && pa.ndet > 0) RT(ensure(p, p->tap_part, (size_t)pa.ndet * kTapChunks * sizeof(double)));
    auto one = [&]() -> rte_status {
        void *A = p->psi[p->cur], *B = p->psi[1 - p->cur];
        const rte_status s = fast ? plane_step<R>(p, A, B, pa, integ) : one_step<R>(p, A, B, cdt, 1.0, xa, integ, 1);
        p->cur = 1 - p->cur;
        return s;
    };
    int s = 0;
    const int G = p->gsteps;
    if (graphs_enabled(p) && G > 0 && nsteps >= G + 2) {
        // the kernels' arguments are the same every step but for the ping-pong
        // buffers, so a graph of G (even) steps replays any run of G steps
        std::vector<unsigned char> key;
        key_append(key, G);
        key_append(key, fast);
        key_append(key, p->cur);
        key_append(key, integ);
        key_append(key, p->psi[0]);
        key_append(key, p->psi[1]);
        key_append(key, p->tap_part.p);
        if (fast) key_append(key, pa);
        else key_append(key, xa);
        key_append(key, cdt);
        if (!(p->gexec && p->gkey == key)) {
            // the first launches of each kernel (module loading) run outside any capture
            RT(one());
            RT(one());
            s = 2;
        }
        RT(ensure_step_graph(p, key, [&]() -> rte_status {
            for (int i = 0; i < G; ++i) RT(one());
            return RTE_OK;
        }));
        int since = 0;
        for (; s + G <= nsteps; s += G) {
            CK(cudaGraphLaunch(p->gexec, p->st));
            g_launches.fetch_add((uint64_t)p->gkern, std::memory_order_relaxed);
            since += G;
            if (since >= kFiniteCheckSteps && s + G < nsteps) {
                since = 0;
                const rte_status fs = check_finite(p);
                if (fs != RTE_OK) {
                    p->time += (s + G) * dt;
                    return fs;
                }
            }
        }
    }
    for (; s < nsteps; ++s) RT(one());
    if (want_det)
        CK(cudaMemcpyAsync(det_series, p->det_out.p, (size_t)nsteps * nd * sizeof(double), cudaMemcpyDeviceToHost,
                           p->st));
    if (integral)
        CK(cudaMemcpyAsync(integral, p->integ.p, (size_t)nsteps * 2 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    p->time += nsteps * dt;
    // calls that synchronise anyway, and long runs, report a non-finite state;
    // otherwise the flag stays set for the next synchronising call
    if (want_det || integral || nsteps >= kFiniteCheckSteps) return check_finite(p);
    return RTE_OK;
}

// ---------------------------------------------------------------- plan groups

// readouts and step end of one plan of a group (on the group's stream)
template <typename R> rte_status group_tail(rte_plan *p, const void *A, const PlaneArgs<R> &pa, double *integral) {
    if (pa.ndet > 0) {
        prof_begin(p);
        k_taps<R><<<dim3(pa.ndet, kTapChunks), 128, 0, p->st>>>((const CT<R> *)A, p->d.nx, p->d.ny,
                                                               (const double2 *)p->tw64[0], (const double2 *)p->tw64[1],
                                                               pa.det, (double *)p->tap_part.p);
        RT(after_launch(p, "k_taps"));
        prof_begin(p);
        k_taps_finish<<<(pa.ndet + 127) / 128, 128, 0, p->st>>>((const double *)p->tap_part.p, pa.ndet,
                                                               1.0 / ((double)p->d.nx * p->d.ny), p->step,
                                                               pa.det_out);
        RT(after_launch(p, "k_taps_finish"));
    }
    return launch_advance<R>(p, A, integral, 1);
}

template <typename R>
rte_status step_group_impl(rte_plan *const *pl, int n, const double *dt, int nsteps, double *const *det_series) {
    rte_plan *p0 = pl[0];
    for (int i = 0; i < n; ++i) {
        rte_plan *p = pl[i];
        if (p->d.nx != p0->d.nx || p->d.ny != p0->d.ny || p->d.nz != p0->d.nz || p->d.N != p0->d.N ||
            p->d.precision != p0->d.precision || p->real != p0->real || p->st != p0->st)
            return fail(RTE_ERR_INVALID_ARG, "group plans must share grid, order, precision, layout and stream");
        for (int j = 0; j < i; ++j)
            if (pl[j] == p) return fail(RTE_ERR_INVALID_ARG, "a plan appears twice in the group");
        if (!use_plane<R>(p) || !injections_fit_plane(p, p->src_vox, p->src_mom))
            return fail(RTE_ERR_UNSUPPORTED, "group steps need the fused plane path");
        RT(check_dt(p, dt[i], 0));
    }
    if (nsteps == 0) return RTE_OK;
    PlaneArgs<R> pa;
    ZArgs<R> za;
    std::memset(&za, 0, sizeof(za));
    std::vector<PlaneArgs<R>> own(n);   // each plan's readout arguments
    for (int i = 0; i < n; ++i) {
        rte_plan *p = pl[i];
        const double cdt = p->d.c_mm_per_ps * dt[i];
        const bool want_det = det_series && det_series[i] && !p->det_vox.empty();
        RT(upload_sources<R>(p, dt[i], nsteps, p->time));
        if (want_det) {
            RT(upload_detectors<R>(p));
            RT(ensure(p, p->det_out, (size_t)nsteps * p->det_vox.size() * sizeof(double)));
        }
        own[i] = plane_args_step<R>(p, cdt, want_det);
        if (own[i].ndet > 0) RT(ensure(p, p->tap_part, (size_t)own[i].ndet * kTapChunks * sizeof(double)));
        CK(cudaMemsetAsync(p->step, 0, sizeof(int), p0->st));
        if (i == 0) pa = own[0];
        pa.pl[i] = own[i].pl[0];
        za.a[i] = (R)1;
        za.coefS[i] = (R)(-cdt);
    }
    pa.nplans = za.nplans = n;
    auto one = [&]() -> rte_status {
        for (int i = 0; i < n; ++i) {
            rte_plan *p = pl[i];
            za.in[i] = (const CT<R> *)p->psi[p->cur];
            za.out[i] = (CT<R> *)p->dz;
            pa.pl[i].psi_in = (const CT<R> *)p->psi[p->cur];
            pa.pl[i].win = (const CT<R> *)p->dz;
            pa.pl[i].out = (CT<R> *)p->psi[1 - p->cur];
        }
        RT(launch_zstream_args<R>(p0, za));
        RT(launch_plane_args<R>(p0, pa));
        for (int i = 0; i < n; ++i) {
            rte_plan *p = pl[i];
            cudaStream_t own_st = p->st;
            p->st = p0->st;   // the same stream, or p0's capture stream while a graph is recorded
            const rte_status st = group_tail<R>(p, p->psi[p->cur], own[i], nullptr);
            p->st = own_st;
            RT(st);
            p->cur = 1 - p->cur;
        }
        return RTE_OK;
    };
    int s = 0;
    const int G = p0->gsteps;
    if (graphs_enabled(p0) && G > 0 && nsteps >= G + 2) {
        std::vector<unsigned char> key;
        key_append(key, -n);   // a group graph never matches a single plan's key
        key_append(key, G);
        for (int i = 0; i < n; ++i) {
            key_append(key, (const void *)pl[i]);
            key_append(key, pl[i]->cur);
            key_append(key, pl[i]->psi[0]);
            key_append(key, pl[i]->psi[1]);
            key_append(key, pl[i]->tap_part.p);
            key_append(key, own[i]);
            key_append(key, dt[i]);
        }
        if (!(p0->gexec && p0->gkey == key)) {
            RT(one());
            RT(one());
            s = 2;
        }
        std::vector<int> cur0(n);
        for (int i = 0; i < n; ++i) cur0[i] = pl[i]->cur;
        RT(ensure_step_graph(p0, key, [&]() -> rte_status {
            for (int k = 0; k < G; ++k) RT(one());
            return RTE_OK;
        }));
        for (int i = 0; i < n; ++i) pl[i]->cur = cur0[i];   // capturing ran no step
        for (; s + G <= nsteps; s += G) {
            CK(cudaGraphLaunch(p0->gexec, p0->st));
            g_launches.fetch_add((uint64_t)p0->gkern, std::memory_order_relaxed);
        }
    }
    for (; s < nsteps; ++s) RT(one());
    bool sync = nsteps >= kFiniteCheckSteps;
    for (int i = 0; i < n; ++i) {
        rte_plan *p = pl[i];
        if (own[i].ndet > 0) {
            CK(cudaMemcpyAsync(det_series[i], p->det_out.p, (size_t)nsteps * own[i].ndet * sizeof(double),
                               cudaMemcpyDeviceToHost, p0->st));
            sync = true;
        }
        p->time += nsteps * dt[i];
    }
    if (sync)
        for (int i = 0; i < n; ++i) RT(check_finite(pl[i]));
    return RTE_OK;
}

// ---------------------------------------------------------------- plans

template <typename R> rte_status upload_tables(rte_plan *p) {
    const int dims[3] = {p->d.nx, p->d.ny, p->d.nz};
    for (int a = 0; a < 3; ++a) {
        const int nn = dims[a];
        auto tw = twiddles(nn);
        std::vector<CT<R>> twr(nn);
        std::vector<R> kr(nn);
        for (int j = 0; j < nn; ++j) {
            twr[j].x = (R)tw[j].real();
            twr[j].y = (R)tw[j].imag();
            kr[j] = (R)wavenumber(j, nn, p->d.dx_mm);
        }
        RT(upload(p, (void **)&p->tw[a], twr.data(), nn * sizeof(CT<R>)));
        if (a < 2) {
            std::vector<double2> tw64(nn);
            for (int j = 0; j < nn; ++j) tw64[j] = make_double2(tw[j].real(), tw[j].imag());
            RT(upload(p, (void **)&p->tw64[a], tw64.data(), nn * sizeof(double2)));
        }
        RT(upload(p, (void **)&p->kt[a], kr.data(), nn * sizeof(R)));
    }
    // per stored moment: l, the adjoint-gradient weight c_l^2 and the
    // dot-product weight 2l+1, both doubled for m > 0 in the real layout
    // (the m and -m moments contribute equally)
    std::vector<int> lof(p->M);
    std::vector<R> wl(p->M);
    std::vector<double> mw(p->M);
    for (int l = 0; l <= p->d.N; ++l)
        for (int m = p->real ? 0 : -l; m <= l; ++m) {
            const int j = p->real ? l * (l + 1) / 2 + m : l * l + l + m;
            const double pair = (p->real && m > 0) ? 2.0 : 1.0;
            lof[j] = l;
            wl[j] = (R)(pair * (2.0 * l + 1.0) / (4.0 * kPi));
            mw[j] = pair * (2.0 * l + 1.0);
        }
    RT(upload(p, (void **)&p->lof, lof.data(), p->M * sizeof(int)));
    RT(upload(p, (void **)&p->wl, wl.data(), p->M * sizeof(R)));
    RT(upload(p, (void **)&p->mw, mw.data(), p->M * sizeof(double)));
    auto rows = p->real ? coupling_rows_real(p->d.N) : coupling_rows(p->d.N);
    RT(upload(p, (void **)&p->coup, rows.data(), rows.size() * sizeof(CouplingRow)));
    // folded media (mu_a, mu_s, g, interior)
    std::vector<double> mub;
    std::vector<uint8_t> mask;
    layer_profile(p->d.nx, p->d.ny, p->d.nz, p->d.pml_cells, p->d.pml_mu0, p->d.pml_mu1, mub, mask);
    using M4 = typename Media4<R>::type;
    std::vector<M4> med(p->V);
    std::vector<double> ae(p->V), se(p->V);
    for (size_t v = 0; v < p->V; ++v) {
        ae[v] = mask[v] ? mub[v] : p->mua[v];
        se[v] = mask[v] ? 0.0 : p->mus[v];
        med[v].x = (R)ae[v];
        med[v].y = (R)se[v];
        med[v].z = (R)p->g[v];
        med[v].w = mask[v] ? (R)0 : (R)1;
    }
    RT(upload(p, (void **)&p->med, med.data(), p->V * sizeof(M4)));
    // D_l = mu_a + mu_s (1 - g^l) per l, each z plane stored [x slot][y slot],
    // for the fused plane kernel (planes it takes: see plane_fits)
    // x slot px holds x = px / (nx/4) + 4 (px % (nx/4)) (4-point DIF phase
    // first); y slot py holds y = py / SY + (ny/SY) (py % SY) (ny/SY-point
    // phase first)
    if (plane_fits<R>(p->d.nx, p->d.ny)) {
        const int x1 = 4, x2 = p->d.nx / 4, y2 = plane_sy(p->d.ny), y1 = p->d.ny / y2;
        const int nx = p->d.nx, ny = p->d.ny, L = p->d.N + 1;
        const size_t ne = (size_t)nx * ny;
        std::vector<R> dl((size_t)L * p->V);
        for (int z = 0; z < p->d.nz; ++z)
            for (int px = 0; px < nx; ++px)
                for (int py = 0; py < ny; ++py) {
                    const int x = px / x2 + x1 * (px % x2), y = py / y2 + y1 * (py % y2);
                    const size_t v = z * ne + (size_t)y * nx + x;
                    double gl = 1.0;
                    for (int l = 0; l < L; ++l) {
                        dl[(size_t)l * p->V + z * ne + (size_t)px * ny + py] = (R)(ae[v] + se[v] * (1.0 - gl));
                        gl *= p->g[v];
                    }
                }
        RT(upload(p, (void **)&p->dl_slot, dl.data(), dl.size() * sizeof(R)));
    }
    p->classes = media_classes(p->V, ae.data(), se.data(), p->g.data(), mask.data(), 1024);
    // GMRES preconditioner: interior means Dbar_l of D_l, the l <= 1 couplings
    {
        const int L = p->d.N + 1;
        std::vector<double> dbar(L, 0.0);
        size_t cnt = 0;
        for (size_t v = 0; v < p->V; ++v) {
            if (mask[v]) continue;
            double gl = 1.0;
            for (int l = 0; l < L; ++l) {
                dbar[l] += ae[v] + se[v] * (1.0 - gl);
                gl *= p->g[v];
            }
            ++cnt;
        }
        for (int l = 0; l < L; ++l) dbar[l] = cnt ? dbar[l] / (double)cnt : 1.0;
        std::vector<R> sc(p->M);
        for (int j = 0; j < p->M; ++j) sc[j] = lof[j] >= 2 ? (R)(1.0 / dbar[lof[j]]) : (R)1;
        RT(upload(p, &p->prec_scale, sc.data(), p->M * sizeof(R)));
        p->plow = PrecLow{};
        p->plow.d0 = dbar[0];
        p->plow.d1 = L > 1 ? dbar[1] : 1.0;
        if (L > 1) {
            const auto full = coupling_rows(p->d.N);
            for (int o = 0; o < 4; ++o)
                for (int t = 0; t < full[o].n; ++t)
                    if (full[o].src[t] < 4 && p->plow.nterm < 16) {
                        const int k = p->plow.nterm++;
                        p->plow.o[k] = o;
                        p->plow.s[k] = full[o].src[t];
                        p->plow.type[k] = full[o].type[t];
                        p->plow.coef[k] = full[o].coef[t];
                    }
        }
    }
    return RTE_OK;
}

rte_status validate_desc(const rte_grid_desc *d) {
    if (!d) return fail(RTE_ERR_INVALID_ARG, "null descriptor");
    if (!axis_ok(d->nx) || !axis_ok(d->ny) || !axis_ok(d->nz))
        return fail(RTE_ERR_INVALID_ARG, "grid sizes must be 4..1024 and products of 2, 3, 5");
    if (d->N < 0 || d->N > 21) return fail(RTE_ERR_INVALID_ARG, "N must be in 0..21");
    if (!(d->dx_mm > 0.0) || !(d->c_mm_per_ps > 0.0)) return fail(RTE_ERR_INVALID_ARG, "dx and c must be > 0");
    if (d->precision != RTE_FP32 && d->precision != RTE_FP64) return fail(RTE_ERR_INVALID_ARG, "bad precision");
    if (d->real_radiance != 0 && d->real_radiance != 1) return fail(RTE_ERR_INVALID_ARG, "real_radiance must be 0 or 1");
    if (d->pml_cells < 0 || 2 * d->pml_cells >= std::min(d->nx, std::min(d->ny, d->nz)))
        return fail(RTE_ERR_INVALID_ARG, "layer thicker than half the grid");
    if (d->pml_cells > 0 && !(d->pml_mu0 >= 0.0 && d->pml_mu1 >= 0.0))
        return fail(RTE_ERR_INVALID_ARG, "layer loss must be >= 0");
    return RTE_OK;
}

void prof_drain(rte_plan *p) {
    for (auto &q : p->ev_pend) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, q.a, q.b);
        size_t i = 0;
        while (i < p->prof_names.size() && p->prof_names[i] != q.name) ++i;
        if (i == p->prof_names.size()) {
            p->prof_names.push_back(q.name);
            p->prof_count.push_back(0);
            p->prof_ms.push_back(0.0);
        }
        p->prof_count[i] += 1;
        p->prof_ms[i] += ms;
        p->ev_pool.push_back(q.a);
        p->ev_pool.push_back(q.b);
    }
    p->ev_pend.clear();
}

void destroy(rte_plan *p) {
    if (!p) return;
    prof_drain(p);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->ev_open) cudaEventDestroy(p->ev_open);
    if (p->sub) destroy(p->sub);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap_st) cudaStreamDestroy(p->cap_st);
    for (void *q : {p->psi[0], p->psi[1], p->dz, p->t1, p->med, p->dl_slot, p->tw[0], p->tw[1], p->tw[2], p->tw64[0],
                    p->tw64[1], p->kt[0], p->kt[1],
                    p->kt[2], (void *)p->lof, p->wl, (void *)p->mw, (void *)p->coup, (void *)p->step, (void *)p->flags, p->prec_scale, p->gfac})
        plan_free(p, q);
    for (DevBuf *b : {&p->inj, &p->inj_amp, &p->det, &p->det_out, &p->integ, &p->tap_part, &p->kry, &p->kw, &p->kpz, &p->parts, &p->dres,
                      &p->dcoef, &p->rhs, &p->x64, &p->r64, &p->ckpt, &p->rec, &p->lam[0], &p->lam[1], &p->fwd[0],
                      &p->fwd[1], &p->grad_inj, &p->expE, &p->exp_term, &p->exp_coef, &p->exp_dl})
        release(p, *b);
    cudaStreamSynchronize(p->st);   // the memory is back in the pool when destroy returns
    delete p;
}

rte_status create(const rte_grid_desc *desc, const double *mua, const double *mus, const double *g,
                  cudaStream_t st, rte_plan **out, const Allocator &al) {
    RT(validate_desc(desc));
    if (!mua || !mus || !g || !out) return fail(RTE_ERR_INVALID_ARG, "null argument");
    auto *p = new rte_plan();
    p->al = al;
    p->d = *desc;
    p->Mfull = (desc->N + 1) * (desc->N + 1);
    p->real = desc->real_radiance;
    p->M = p->real ? (desc->N + 1) * (desc->N + 2) / 2 : p->Mfull;
    p->V = (size_t)desc->nx * desc->ny * desc->nz;
    p->n = p->V * p->M;
    p->esz = desc->precision == RTE_FP64 ? 16 : 8;
    p->st = st;
    for (size_t v = 0; v < p->V; ++v) {
        if (!std::isfinite(mua[v]) || !std::isfinite(mus[v]) || !std::isfinite(g[v]) || mua[v] < 0 || mus[v] < 0 ||
            g[v] < -1.0 || g[v] > 1.0) {
            delete p;
            return fail(RTE_ERR_INVALID_ARG, "optical map has a negative, non-finite or out-of-range value");
        }
    }
    p->mua.assign(mua, mua + p->V);
    p->mus.assign(mus, mus + p->V);
    p->g.assign(g, g + p->V);
    radix_plan(desc->nx, &p->fp[0]);
    radix_plan(desc->ny, &p->fp[1]);
    radix_plan(desc->nz, &p->fp[2]);
    const int dims[3] = {desc->nx, desc->ny, desc->nz};
    for (int a = 0; a < 3; ++a) {
        double km = 0.0;
        for (int i = 0; i < dims[a]; ++i) km = std::max(km, std::fabs(wavenumber(i, dims[a], desc->dx_mm)));
        p->kmax += km * km;
    }
    p->kmax = std::sqrt(p->kmax);
    rte_status s = RTE_OK;
    auto tryalloc = [&](void **q, size_t b) {
        if (s != RTE_OK) return;
        cudaError_t e = plan_malloc(p, q, b);
        if (e != cudaSuccess) s = cuda_fail(e, p->al.alloc ? "caller's allocator" : "cudaMallocAsync");
    };
    for (void **q : {&p->psi[0], &p->psi[1], &p->dz, &p->t1}) tryalloc(q, p->n * p->esz);
    tryalloc((void **)&p->step, sizeof(int));
    tryalloc((void **)&p->flags, 2 * sizeof(int));
    if (s == RTE_OK) s = desc->precision == RTE_FP64 ? upload_tables<double>(p) : upload_tables<float>(p);
    if (s == RTE_OK) {
        cudaError_t e = cudaMemsetAsync(p->psi[0], 0, p->n * p->esz, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->step, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->flags, 0, 2 * sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "initialise state");
    }
    if (s != RTE_OK) {
        destroy(p);
        return s;
    }
    *out = p;
    return RTE_OK;
}

rte_status check_dt(rte_plan *p, double dt, int allow_unstable) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(RTE_ERR_INVALID_ARG, "dt must be > 0");
    if (allow_unstable) return RTE_OK;
    if (p->dtstar < 0.0) {
        p->dtstar = stability_from_classes(p->d.N, p->d.c_mm_per_ps, p->kmax, p->classes, 256);
        if (p->dtstar < 0.0) return fail(RTE_ERR_CUDA, "eigenvalue iteration did not converge");
    }
    if (dt > 1.0001 * p->dtstar) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "dt = %.6g ps exceeds the stability limit %.6g ps", dt, p->dtstar);
        return fail(RTE_ERR_UNSTABLE_DT, buf);
    }
    return RTE_OK;
}

// ---------------------------------------------------------------- state io

// Full-layout field (ABI) -> stored moments in `dst` (device). In the real
// layout only the m >= 0 moment planes are copied.
rte_status gather_stored(rte_plan *p, const void *full, void *dst, cudaMemcpyKind kind) {
    const size_t plane = p->V * p->esz;
    if (!p->real) {
        CK(cudaMemcpyAsync(dst, full, p->n * p->esz, kind, p->st));
        return RTE_OK;
    }
    for (int l = 0; l <= p->d.N; ++l)
        for (int m = 0; m <= l; ++m)
            CK(cudaMemcpyAsync((char *)dst + (size_t)(l * (l + 1) / 2 + m) * plane,
                               (const char *)full + (size_t)(l * l + l + m) * plane, plane, kind, p->st));
    return RTE_OK;
}

// Stored moments in `src` (device) -> full-layout field; in the real layout the
// m < 0 moments are rebuilt as (-1)^m conj(psi_{l,-m}).
template <typename R> rte_status scatter_full(rte_plan *p, const void *src, void *full, int where) {
    const size_t plane = p->V * p->esz;
    const cudaMemcpyKind kind = where == RTE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (!p->real) {
        CK(cudaMemcpyAsync(full, src, p->n * p->esz, kind, p->st));
        return RTE_OK;
    }
    for (int l = 0; l <= p->d.N; ++l)
        for (int m = 0; m <= l; ++m)
            CK(cudaMemcpyAsync((char *)full + (size_t)(l * l + l + m) * plane,
                               (const char *)src + (size_t)(l * (l + 1) / 2 + m) * plane, plane, kind, p->st));
    if (where == RTE_DEVICE) {
        k_mirror_moments<R><<<vec_grid((size_t)p->Mfull * p->V), 256, 0, p->st>>>((CT<R> *)full, p->V, p->d.N);
        return after_launch(p, "k_mirror_moments");
    }
    if (p->d.N == 0) return RTE_OK;
    // host field: the m < 0 moments are built on the device in the work
    // buffer dz (free between calls; N (N + 1) / 2 <= M planes) and copied to
    // their places, rather than mirrored by the host afterwards
    const int nneg = p->d.N * (p->d.N + 1) / 2;
    const size_t blocks = std::min<size_t>((p->V + 255) / 256, (size_t)4 * num_sms());
    k_negative_moments<R><<<dim3((unsigned)blocks, nneg), 256, 0, p->st>>>((const CT<R> *)src, (CT<R> *)p->dz, p->V);
    RT(after_launch(p, "k_negative_moments"));
    for (int l = 1; l <= p->d.N; ++l)
        for (int m = 1; m <= l; ++m)
            CK(cudaMemcpyAsync((char *)full + (size_t)(l * l + l - m) * plane,
                               (const char *)p->dz + (size_t)(l * (l - 1) / 2 + m - 1) * plane, plane, kind, p->st));
    return RTE_OK;
}

template <typename R> rte_status set_state_impl(rte_plan *p, const void *psi, int where) {
    CK(cudaMemsetAsync(p->flags, 0, sizeof(int), p->st));   // a new state (a timeout record stays)
    RT(gather_stored(p, psi, p->t1, where == RTE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
    RT(to_tilde<R>(p, p->t1, p->psi[p->cur]));
    CK(cudaStreamSynchronize(p->st));
    return RTE_OK;
}

template <typename R> rte_status get_state_impl(rte_plan *p, void *psi, int where) {
    RT(from_tilde<R>(p, p->psi[p->cur], p->t1, p->t1));
    RT(scatter_full<R>(p, p->t1, psi, where));
    CK(cudaStreamSynchronize(p->st));
    return check_finite(p);   // the state is returned either way
}

template <typename R> rte_status apply_impl(rte_plan *p, const void *in, void *out) {
    void *B = p->psi[1 - p->cur];
    RT(gather_stored(p, in, p->t1, cudaMemcpyDeviceToDevice));
    RT(to_tilde<R>(p, p->t1, B));
    RT(apply_T_tilde<R>(p, B, p->t1, 1.0));
    RT(from_tilde<R>(p, p->t1, p->t1, p->t1));
    RT(scatter_full<R>(p, p->t1, out, RTE_DEVICE));
    return RTE_OK;
}

// ---------------------------------------------------------------- GMRES

// complex Givens G = [[c, s], [-conj(s), c]] with real c
struct Givens {
    double c;
    double sr, si;
};

// Restarted GMRES(m) on T x = b (both psi~ form, plan precision). x starts at 0.
template <typename R>
rte_status gmres_impl(rte_plan *p, const void *b, void *x, int m, int max_iter, double rtol, int *iters_out,
                      double *rel_out, bool *conv_out) {
    using cd = std::complex<double>;
    const size_t vb = p->n * p->esz;
    RT(ensure(p, p->kry, vb * (size_t)(m + 1)));
    RT(ensure(p, p->kw, vb));
    const bool pc = p->prec == RTE_PREC_LOW_ORDER;
    if (pc) RT(ensure(p, p->kpz, vb));
    char *basis = (char *)p->kry.p;
    void *w = p->kw.p;
    void *pz = p->kpz.p;
    CK(cudaMemsetAsync(x, 0, vb, p->st));
    double bn;
    RT(wnorm<R>(p, b, &bn));
    int iters = 0;
    double rel = 1.0;
    bool conv = false;
    if (bn == 0.0) {
        *iters_out = 0;
        *rel_out = 0.0;
        *conv_out = true;
        return RTE_OK;
    }
    std::vector<cd> H((size_t)(m + 1) * m), gv(m + 1), y(m);
    std::vector<Givens> rot(m);
    std::vector<double> h(2 * (m + 2)), h2(2 * (m + 2));
    bool first = true;
    while (iters < max_iter) {
        double beta;
        if (first) {
            CK(cudaMemcpyAsync(w, b, vb, cudaMemcpyDeviceToDevice, p->st));
            beta = bn;
            first = false;
        } else {
            RT(apply_T_tilde<R>(p, x, w, 1.0));
            RT((axpby<R, R>(p, b, w, 1.0, 0.0, -1.0, 0.0)));   // w = b - T x
            RT(wnorm<R>(p, w, &beta));
        }
        rel = beta / bn;
        if (rel <= rtol) {
            conv = true;
            break;
        }
        RT((axpby<R, R>(p, w, basis, 1.0 / beta, 0.0, 0.0, 0.0)));
        std::fill(gv.begin(), gv.end(), cd(0.0));
        gv[0] = beta;
        int j = 0;
        for (; j < m && iters < max_iter;) {
            void *vj = basis + (size_t)j * vb;
            void *vn = basis + (size_t)(j + 1) * vb;
            if (pc) {
                RT(apply_prec<R>(p, vj, pz));
                RT(apply_T_tilde<R>(p, pz, w, 1.0));
            } else {
                RT(apply_T_tilde<R>(p, vj, w, 1.0));
            }
            // classical Gram-Schmidt; |w|^2 comes with the projections, and
            // |w - sum h_i v_i|^2 = |w|^2 - sum |h_i|^2 for an orthonormal
            // basis. Unless that shows severe cancellation (the new direction
            // below 1e-3 of |w|^2), one pass suffices and the subtraction
            // writes v_{j+1} already normalised; otherwise project a second
            // time. GMRES tolerates the mild loss of orthogonality of one pass
            // (the true residual is recomputed at every restart, and FP32
            // solves are refined against FP64 residuals): on the 256^3 steady
            // problem the textbook 1/2 threshold reprojected almost every
            // step for the same number of steps.
            RT(wdots<R>(p, basis, j + 1, w, h.data(), 1));
            const double ww = h[2 * (j + 1)];
            double hh = 0.0;
            for (int i = 0; i <= j; ++i) hh += h[2 * i] * h[2 * i] + h[2 * i + 1] * h[2 * i + 1];
            const double rest = ww - hh;
            double hn;
            if (rest > 1e-3 * ww && rest > 0.0) {
                hn = std::sqrt(rest);
                RT(sub_multi<R>(p, basis, j + 1, h.data(), w, vn, 1.0 / hn));
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = cd(h[2 * i], h[2 * i + 1]);
            } else {
                RT(sub_multi<R>(p, basis, j + 1, h.data(), w));
                RT(wdots<R>(p, basis, j + 1, w, h2.data()));
                RT(sub_multi<R>(p, basis, j + 1, h2.data(), w));
                for (int i = 0; i <= j; ++i)
                    H[(size_t)i * m + j] = cd(h[2 * i] + h2[2 * i], h[2 * i + 1] + h2[2 * i + 1]);
                RT(wnorm<R>(p, w, &hn));
                if (hn > 0.0) RT((axpby<R, R>(p, w, vn, 1.0 / hn, 0.0, 0.0, 0.0)));
            }
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                const cd a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                const cd s(rot[i].sr, rot[i].si);
                H[(size_t)i * m + j] = rot[i].c * a + s * bb;
                H[(size_t)(i + 1) * m + j] = -std::conj(s) * a + rot[i].c * bb;
            }
            const cd a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            const double rho = std::sqrt(std::norm(a) + std::norm(bb));
            Givens gr;
            if (std::abs(a) == 0.0) {
                gr.c = 0.0;
                gr.sr = 1.0;
                gr.si = 0.0;
            } else {
                gr.c = std::abs(a) / rho;
                const cd s = a * std::conj(bb) / (std::abs(a) * rho);
                gr.sr = s.real();
                gr.si = s.imag();
            }
            rot[j] = gr;
            const cd s(gr.sr, gr.si);
            H[(size_t)j * m + j] = gr.c * a + s * bb;
            H[(size_t)(j + 1) * m + j] = 0.0;
            const cd g0 = gv[j];
            gv[j] = gr.c * g0;
            gv[j + 1] = -std::conj(s) * g0;
            ++iters;
            ++j;
            rel = std::abs(gv[j]) / bn;
            if (rel <= rtol || hn == 0.0) break;
        }
        for (int i = j - 1; i >= 0; --i) {
            cd acc = gv[i];
            for (int k = i + 1; k < j; ++k) acc -= H[(size_t)i * m + k] * y[k];
            y[i] = acc / H[(size_t)i * m + i];
        }
        std::vector<double> yc(2 * j);
        for (int i = 0; i < j; ++i) {
            yc[2 * i] = y[i].real();
            yc[2 * i + 1] = y[i].imag();
        }
        if (pc) {
            // x += P^-1 (V y); w is free here
            CK(cudaMemsetAsync(w, 0, vb, p->st));
            RT(add_multi<R>(p, basis, j, yc.data(), w));
            RT(apply_prec<R>(p, w, pz));
            RT((axpby<R, R>(p, pz, x, 1.0, 0.0, 1.0, 0.0)));
        } else {
            RT(add_multi<R>(p, basis, j, yc.data(), x));
        }
    }
    if (!conv) {
        RT(apply_T_tilde<R>(p, x, w, 1.0));
        RT((axpby<R, R>(p, b, w, 1.0, 0.0, -1.0, 0.0)));
        double rn;
        RT(wnorm<R>(p, w, &rn));
        rel = rn / bn;
        conv = rel <= rtol;
    }
    *iters_out = iters;
    *rel_out = rel;
    *conv_out = conv;
    return RTE_OK;
}

// right-hand side q~ of the steady problem from the plan's sources (CW amplitude)
template <typename R> rte_status build_rhs(rte_plan *p, void *out) {
    const size_t vb = p->n * p->esz;
    CK(cudaMemsetAsync(p->t1, 0, vb, p->st));
    const int ns = (int)p->src_vox.size();
    if (ns > 0) {
        std::vector<double> val(ns);
        for (int q = 0; q < ns; ++q) val[q] = p->src_amp[q] / (p->d.dx_mm * p->d.dx_mm * p->d.dx_mm);
        DevBuf bv, bm, bval;
        rte_status st = ensure(p, bv, ns * sizeof(long long));
        if (st == RTE_OK) st = ensure(p, bm, ns * sizeof(int));
        if (st == RTE_OK) st = ensure(p, bval, ns * sizeof(double));
        cudaError_t e = cudaSuccess;
        if (st == RTE_OK) {
            e = cudaMemcpyAsync(bv.p, p->src_vox.data(), ns * sizeof(long long), cudaMemcpyHostToDevice, p->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(bm.p, p->src_mom.data(), ns * sizeof(int), cudaMemcpyHostToDevice, p->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(bval.p, val.data(), ns * sizeof(double), cudaMemcpyHostToDevice, p->st);
            if (e == cudaSuccess) {
                prof_begin(p);
                k_scatter_points<R><<<1, 32, 0, p->st>>>((CT<R> *)p->t1, p->V, ns, (const long long *)bv.p,
                                                         (const int *)bm.p, (const double *)bval.p);
                st = after_launch(p, "k_scatter_points");
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
        }
        release(p, bv);
        release(p, bm);
        release(p, bval);
        if (e != cudaSuccess) return cuda_fail(e, "build_rhs");
        if (st != RTE_OK) return st;
    }
    return to_tilde<R>(p, p->t1, out);
}

rte_status make_fp64_twin(rte_plan *p);

template <typename R>
rte_status solve_impl(rte_plan *p, double rtol, int restart, int max_iter, int *iters, double *rel_res) {
    const size_t vb = p->n * p->esz;
    RT(ensure(p, p->rhs, vb));
    RT(build_rhs<R>(p, p->rhs.p));
    void *x = p->psi[p->cur];
    int it = 0;
    double rel = 1.0;
    bool conv = false;
    if (sizeof(R) == 8) {
        RT(gmres_impl<R>(p, p->rhs.p, x, restart, max_iter, rtol, &it, &rel, &conv));
    } else {
        // iterative refinement: FP64 residuals, FP32 GMRES corrections
        RT(make_fp64_twin(p));
        rte_plan *s = p->sub;
        const size_t vb64 = p->n * 16;
        RT(ensure(p, p->x64, vb64));
        RT(ensure(p, p->r64, vb64));
        RT(build_rhs<double>(s, s->psi[0]));     // q~ in FP64 (twin's psi[0])
        CK(cudaMemsetAsync(p->x64.p, 0, vb64, p->st));
        double qn;
        RT(wnorm<double>(s, s->psi[0], &qn));
        void *d32 = p->psi[1 - p->cur];
        for (int outer = 0; outer < 30 && it < max_iter; ++outer) {
            RT(apply_T_tilde<double>(s, p->x64.p, p->r64.p, 1.0));
            RT((axpby<double, double>(s, s->psi[0], p->r64.p, 1.0, 0.0, -1.0, 0.0)));
            double rn;
            RT(wnorm<double>(s, p->r64.p, &rn));
            rel = qn > 0.0 ? rn / qn : 0.0;
            if (rel <= rtol) {
                conv = true;
                break;
            }
            RT((axpby<float, double>(p, p->r64.p, p->rhs.p, 1.0 / rn, 0.0, 0.0, 0.0)));
            int it2 = 0;
            double rel2 = 1.0;
            bool c2 = false;
            const double inner = std::max(1e-4, 0.3 * rtol / rel);
            RT(gmres_impl<float>(p, p->rhs.p, d32, restart, max_iter - it, inner, &it2, &rel2, &c2));
            it += it2;
            RT((axpby<double, float>(s, d32, p->x64.p, rn, 0.0, 1.0, 0.0)));
        }
        if (!conv) {
            RT(apply_T_tilde<double>(s, p->x64.p, p->r64.p, 1.0));
            RT((axpby<double, double>(s, s->psi[0], p->r64.p, 1.0, 0.0, -1.0, 0.0)));
            double rn;
            RT(wnorm<double>(s, p->r64.p, &rn));
            rel = qn > 0.0 ? rn / qn : 0.0;
            conv = rel <= rtol;
        }
        RT((axpby<float, double>(p, p->x64.p, x, 1.0, 0.0, 0.0, 0.0)));
    }
    CK(cudaStreamSynchronize(p->st));
    if (iters) *iters = it;
    if (rel_res) *rel_res = rel;
    if (!std::isfinite(rel)) return fail(RTE_ERR_NONFINITE, "the GMRES residual is not finite");
    return conv ? RTE_OK : fail(RTE_ERR_NOT_CONVERGED, "GMRES did not reach the tolerance");
}

rte_status make_fp64_twin(rte_plan *p) {
    if (p->sub) return RTE_OK;
    rte_grid_desc d = p->d;
    d.precision = RTE_FP64;
    RT(create(&d, p->mua.data(), p->mus.data(), p->g.data(), p->st, &p->sub, p->al));
    p->sub->src_vox = p->src_vox;
    p->sub->src_mom = p->src_mom;
    p->sub->src_amp = p->src_amp;
    p->sub->src_t0 = p->src_t0;
    p->sub->src_fwhm = p->src_fwhm;
    return RTE_OK;
}

// ---------------------------------------------------------------- exponential step

template <typename R> rte_status zdft_all(rte_plan *p, const void *in, void *out, int inverse) {
    return with_line_split(p->d.nz, [&](auto n1, auto n2) -> rte_status {
        constexpr int N1 = decltype(n1)::value, N2 = decltype(n2)::value;
        constexpr int TX = sizeof(R) == 4 ? 16 : 8, NT = TX * N2;
        dim3 grid((p->d.nx + TX - 1) / TX, p->d.ny, p->M);
        prof_begin(p);
        k_zdft_fixed<R, N1, N2, TX, NT><<<grid, NT, 0, p->st>>>((const CT<R> *)in, (CT<R> *)out, geo<R>(p), inverse);
        return after_launch(p, inverse ? "k_zdft_fixed(inverse)" : "k_zdft_fixed(forward)");
    });
}

// nsteps exponential steps of dt (homogeneous periodic medium, no sources)
template <typename R> rte_status expo_impl(rte_plan *p, double dt, int nsteps) {
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(RTE_ERR_INVALID_ARG, "dt must be > 0, nsteps >= 0");
    if (p->real) return fail(RTE_ERR_UNSUPPORTED, "the exponential step needs the full moment layout");
    if (p->d.pml_cells > 0) return fail(RTE_ERR_UNSUPPORTED, "the exponential step needs a medium without a layer");
    if (!p->src_vox.empty()) return fail(RTE_ERR_UNSUPPORTED, "the exponential step takes no sources");
    if (!line_fixed(p->d.nz)) return fail(RTE_ERR_UNSUPPORTED, "the exponential step needs nz in 32, 64, 96, 128, 160, 256");
    if (p->M > 64) return fail(RTE_ERR_UNSUPPORTED, "the exponential step needs N <= 7");
    for (size_t v = 1; v < p->V; ++v)
        if (p->mua[v] != p->mua[0] || p->mus[v] != p->mus[0] || p->g[v] != p->g[0])
            return fail(RTE_ERR_UNSUPPORTED, "the exponential step needs a uniform medium");
    if (nsteps == 0) return RTE_OK;
    const int M = p->M;
    if (p->exp_dt != dt) {
        // per-moment D_l and the streaming terms of Eq. 10 (full layout)
        if (!p->exp_term.p) {
            std::vector<int4> term;
            std::vector<double> coef;
            const auto rows = coupling_rows(p->d.N);
            for (int o = 0; o < M; ++o)
                for (int t = 0; t < rows[o].n; ++t) {
                    term.push_back(make_int4(o, rows[o].src[t], rows[o].type[t], 0));
                    coef.push_back(rows[o].coef[t]);
                }
            std::vector<double> dl(M);
            for (int l = 0; l <= p->d.N; ++l)
                for (int m = -l; m <= l; ++m) dl[l * l + l + m] = p->mua[0] + p->mus[0] * (1.0 - std::pow(p->g[0], l));
            p->exp_nterm = (int)term.size();
            RT(ensure(p, p->exp_term, term.size() * sizeof(int4)));
            RT(ensure(p, p->exp_coef, coef.size() * sizeof(double)));
            RT(ensure(p, p->exp_dl, dl.size() * sizeof(double)));
            CK(cudaMemcpyAsync(p->exp_term.p, term.data(), term.size() * sizeof(int4), cudaMemcpyHostToDevice, p->st));
            CK(cudaMemcpyAsync(p->exp_coef.p, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice,
                               p->st));
            CK(cudaMemcpyAsync(p->exp_dl.p, dl.data(), dl.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
            CK(cudaStreamSynchronize(p->st));   // the host vectors go out of scope
        }
        RT(ensure(p, p->expE, (size_t)M * M * p->V * p->esz));
        ExpoArgs ea;
        ea.M = M;
        ea.nterm = p->exp_nterm;
        ea.term = (const int4 *)p->exp_term.p;
        ea.coef = (const double *)p->exp_coef.p;
        ea.dl = (const double *)p->exp_dl.p;
        ea.cdt = p->d.c_mm_per_ps * dt;
        ea.nsub = 14;   // Taylor degree at |B|_1 <= 1/2: truncation below 1e-16
        const size_t smem = 3 * (size_t)M * M * sizeof(double2);
        CK(allow_smem(k_expm_build<R, 256>, smem));
        prof_begin(p);
        k_expm_build<R, 256><<<(unsigned)p->V, 256, smem, p->st>>>(geo<R>(p), ea, (CT<R> *)p->expE.p);
        RT(after_launch(p, "k_expm_build"));
        p->exp_dt = dt;
    }
    void *A = p->psi[p->cur];
    void *bufs[2] = {p->t1, p->dz};
    RT(zdft_all<R>(p, A, bufs[0], 0));
    int c = 0;
    for (int s = 0; s < nsteps; ++s) {
        prof_begin(p);
        k_expm_apply<R, 4><<<vec_grid(p->V), 256, 0, p->st>>>((const CT<R> *)p->expE.p, (const CT<R> *)bufs[c],
                                                               (CT<R> *)bufs[1 - c], p->V, M);
        RT(after_launch(p, "k_expm_apply"));
        c = 1 - c;
    }
    RT(zdft_all<R>(p, bufs[c], A, 1));
    CK(cudaStreamSynchronize(p->st));
    p->time += nsteps * dt;
    return RTE_OK;
}

// ---------------------------------------------------------------- adjoint

template <typename R>
rte_status forward_impl(rte_plan *p, double dt, int nsteps, int K, const double *lo, const double *hi, double *y) {
    RT(check_dt(p, dt, 0));
    const int nd = (int)p->det_vox.size();
    if (nsteps <= 0 || K <= 0) return fail(RTE_ERR_INVALID_ARG, "nsteps and ckpt_every must be > 0");
    if (nd > 0 && (!lo || !hi || !y)) return fail(RTE_ERR_INVALID_ARG, "gates and y needed with detectors");
    const size_t vb = p->n * p->esz;
    const int nck = (nsteps + K - 1) / K;
    RT(ensure(p, p->ckpt, vb * (size_t)nck));
    p->fw_valid = false;
    p->fw_nsteps = nsteps;
    p->fw_K = K;
    p->fw_dt = dt;
    p->fw_t0 = p->time;
    p->fw_w.assign((size_t)nsteps * nd, 0.0);
    for (int s = 0; s < nsteps; ++s) {
        const double t = p->time + s * dt;
        for (int d = 0; d < nd; ++d)
            if (t >= lo[d] && t <= hi[d]) p->fw_w[(size_t)s * nd + d] = dt;
    }
    const double cdt = p->d.c_mm_per_ps * dt;
    RT(upload_sources<R>(p, dt, nsteps, p->time));
    if (nd > 0) {
        RT(upload_detectors<R>(p));
        RT(ensure(p, p->det_out, (size_t)nsteps * nd * sizeof(double)));
    }
    CK(cudaMemsetAsync(p->step, 0, sizeof(int), p->st));
    XArgs<R> xa = xargs_step<R>(p, cdt, 1);
    const bool fast = use_plane<R>(p) && injections_fit_plane(p, p->src_vox, p->src_mom);
    const PlaneArgs<R> pa = plane_args_step<R>(p, cdt, 1);
    for (int s = 0; s < nsteps; ++s) {
        void *A = p->psi[p->cur], *B = p->psi[1 - p->cur];
        if (s % K == 0)
            CK(cudaMemcpyAsync((char *)p->ckpt.p + (size_t)(s / K) * vb, A, vb, cudaMemcpyDeviceToDevice, p->st));
        if (fast) RT(plane_step<R>(p, A, B, pa, nullptr));
        else RT(one_step<R>(p, A, B, cdt, 1.0, xa, nullptr, 1));
        p->cur = 1 - p->cur;
    }
    if (nd > 0) {
        std::vector<double> det((size_t)nsteps * nd);
        CK(cudaMemcpyAsync(det.data(), p->det_out.p, det.size() * sizeof(double), cudaMemcpyDeviceToHost, p->st));
        CK(cudaStreamSynchronize(p->st));
        for (int d = 0; d < nd; ++d) {
            double acc = 0.0;
            for (int s = 0; s < nsteps; ++s) acc += p->fw_w[(size_t)s * nd + d] * det[(size_t)s * nd + d];
            y[d] = acc;
        }
    }
    CK(cudaStreamSynchronize(p->st));
    p->time += nsteps * dt;
    RT(check_finite(p));
    p->fw_valid = true;
    return RTE_OK;
}

// interior (1 - g^l) per l >= 1 and z plane, [x slot][y slot] like D_l, for
// the mu_s gradient on the plane path
template <typename R> rte_status build_gfac(rte_plan *p) {
    if (p->gfac || p->d.N < 1) return RTE_OK;
    std::vector<double> mub;
    std::vector<uint8_t> mask;
    layer_profile(p->d.nx, p->d.ny, p->d.nz, p->d.pml_cells, p->d.pml_mu0, p->d.pml_mu1, mub, mask);
    const int nx = p->d.nx, ny = p->d.ny, x1 = 4, x2 = nx / 4, y2 = plane_sy(ny), y1 = ny / y2, L = p->d.N + 1;
    const size_t ne = (size_t)nx * ny;
    std::vector<R> gf((size_t)(L - 1) * p->V);
    for (int z = 0; z < p->d.nz; ++z)
        for (int px = 0; px < nx; ++px)
            for (int py = 0; py < ny; ++py) {
                const int x = px / x2 + x1 * (px % x2), y = py / y2 + y1 * (py % y2);
                const size_t v = z * ne + (size_t)y * nx + x;
                double gl = 1.0;
                for (int l = 1; l < L; ++l) {
                    gl *= p->g[v];
                    gf[(size_t)(l - 1) * p->V + z * ne + (size_t)px * ny + py] = mask[v] ? (R)0 : (R)(1.0 - gl);
                }
            }
    RT(upload(p, &p->gfac, gf.data(), gf.size() * sizeof(R)));
    return RTE_OK;
}

template <typename R> rte_status adjoint_impl(rte_plan *p, const double *dLdy, double *ga, double *gs) {
    if (!p->fw_valid) return fail(RTE_ERR_STATE, "rte_adjoint needs a preceding rte_forward");
    const int T = p->fw_nsteps, K = p->fw_K, nd = (int)p->det_vox.size();
    if (nd > 0 && !dLdy) return fail(RTE_ERR_INVALID_ARG, "dL_dy is null");
    if (!ga || !gs) return fail(RTE_ERR_INVALID_ARG, "gradient pointers are null");
    const size_t vb = p->n * p->esz;
    const double dt = p->fw_dt, cdt = p->d.c_mm_per_ps * dt;
    RT(ensure(p, p->rec, vb * (size_t)K));
    for (int i = 0; i < 2; ++i) {
        RT(ensure(p, p->lam[i], vb));
        RT(ensure(p, p->fwd[i], vb));
    }
    CK(cudaMemsetAsync(ga, 0, p->V * sizeof(double), p->st));
    CK(cudaMemsetAsync(gs, 0, p->V * sizeof(double), p->st));
    CK(cudaMemsetAsync(p->lam[0].p, 0, vb, p->st));
    int lc = 0;
    // adjoint injections into lambda~_00: 4 pi * dL/dy_d * w[s][d]
    std::vector<int4> dpts(nd);
    std::vector<double> damp((size_t)T * nd);
    for (int d = 0; d < nd; ++d) dpts[d] = voxel4(p, p->det_vox[d], 0);
    for (int s = 0; s < T; ++s)
        for (int d = 0; d < nd; ++d) damp[(size_t)s * nd + d] = 4.0 * kPi * dLdy[d] * p->fw_w[(size_t)s * nd + d];
    // the plane kernel takes the adjoint steps too when it takes the grid and
    // at most kMaxItemInj detectors share a plane (they inject into lambda_00)
    const bool fast_adj = use_plane<R>(p) && injections_fit_plane(p, p->det_vox, std::vector<int>(nd, 0)) && p->d.N >= 1;
    if (fast_adj) RT(build_gfac<R>(p));
    const int nck = (T + K - 1) / K;
    for (int j = nck - 1; j >= 0; --j) {
        const int s0 = j * K, s1 = std::min(T, (j + 1) * K);
        // recompute the forward segment, recording psi_s in real space
        RT(upload_sources<R>(p, dt, s1 - s0, p->fw_t0 + s0 * dt));
        CK(cudaMemcpyAsync(p->fwd[0].p, (char *)p->ckpt.p + (size_t)j * vb, vb, cudaMemcpyDeviceToDevice, p->st));
        CK(cudaMemsetAsync(p->step, 0, sizeof(int), p->st));
        XArgs<R> xf = xargs_step<R>(p, cdt, 0);
        const bool fast = use_plane<R>(p) && injections_fit_plane(p, p->src_vox, p->src_mom);
        PlaneArgs<R> pf = plane_args_step<R>(p, cdt, 0);
        int fc = 0;
        for (int s = s0; s < s1; ++s) {
            // the X pass (or the plane kernel's X2 phase) records psi_s in real space
            CT<R> *rec = (CT<R> *)((char *)p->rec.p + (size_t)(s - s0) * vb);
            if (fast) {
                pf.rec_out = rec;
                RT(plane_step<R>(p, p->fwd[fc].p, p->fwd[1 - fc].p, pf, nullptr));
            } else {
                xf.rec_out = rec;
                RT(one_step<R>(p, p->fwd[fc].p, p->fwd[1 - fc].p, cdt, 1.0, xf, nullptr, 1));
            }
            fc = 1 - fc;
        }
        // adjoint steps s = s1-1 .. s0 with reversed streaming
        if (nd > 0) {
            std::vector<double> seg((size_t)(s1 - s0) * nd);
            std::copy(damp.begin() + (size_t)s0 * nd, damp.begin() + (size_t)s1 * nd, seg.begin());
            RT(upload_injections<R>(p, dpts, seg, s1 - s0));
        }
        const int last = s1 - s0 - 1;
        CK(cudaMemcpyAsync(p->step, &last, sizeof(int), cudaMemcpyHostToDevice, p->st));
        if (fast_adj) {
            // plane path: reversed streaming (coefS = +c dt), gradient terms in X2
            PlaneArgs<R> pb = plane_args<R>(p, -cdt, 1.0, cdt);
            pb.pl[0].step = p->step;
            if (nd > 0) {
                pb.pl[0].ninj = nd;
                pb.pl[0].inj = (const int4 *)p->inj.p;
                pb.pl[0].inj_amp = (const R *)p->inj_amp.p;
            }
            pb.grad_a = ga;
            pb.grad_s = gs;
            pb.grad_scale = (R)(-cdt);
            pb.wl = (const R *)p->wl;
            pb.gfac = (const R *)p->gfac;
            for (int s = s1 - 1; s >= s0; --s) {
                pb.rec_in = (const CT<R> *)((char *)p->rec.p + (size_t)(s - s0) * vb);
                RT(plane_step<R>(p, p->lam[lc].p, p->lam[1 - lc].p, pb, nullptr, -1));
                lc = 1 - lc;
            }
            CK(cudaStreamSynchronize(p->st));
            continue;
        }
        XArgs<R> xb = xargs_plain<R>(p);
        xb.inv_in = 1;
        xb.pointwise = 1;
        xb.fwd_out = 1;
        xb.coefD = (R)(-cdt);
        xb.step = p->step;
        if (nd > 0) {
            xb.ninj = nd;
            xb.inj = (const int4 *)p->inj.p;
            xb.inj_amp = (const R *)p->inj_amp.p;
        }
        xb.grad_a = ga;
        xb.grad_s = gs;
        xb.grad_scale = (R)(-cdt);
        for (int s = s1 - 1; s >= s0; --s) {
            xb.rec_in = (const CT<R> *)((char *)p->rec.p + (size_t)(s - s0) * vb);
            RT(one_step<R>(p, p->lam[lc].p, p->lam[1 - lc].p, cdt, -1.0, xb, nullptr, -1));
            lc = 1 - lc;
        }
        CK(cudaStreamSynchronize(p->st));
    }
    if (fast_adj) {
        prof_begin(p);
        k_zero_layer<R><<<vec_grid(p->V), 256, 0, p->st>>>(ga, (const typename Media4<R>::type *)p->med, p->V);
        RT(after_launch(p, "k_zero_layer"));
        CK(cudaStreamSynchronize(p->st));
    }
    return check_finite(p);
}

}  // namespace

namespace rte {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace rte

// ===================================================================== ABI

extern "C" {

const char *rte_status_string(rte_status s) {
    switch (s) {
        case RTE_OK: return "ok";
        case RTE_ERR_INVALID_ARG: return "invalid argument";
        case RTE_ERR_OOM: return "out of device memory";
        case RTE_ERR_UNSTABLE_DT: return "time step above the stability limit";
        case RTE_ERR_NONFINITE: return "non-finite value";
        case RTE_ERR_NOT_CONVERGED: return "not converged";
        case RTE_ERR_TIMEOUT: return "timeout";
        case RTE_ERR_CUDA: return "CUDA error";
        case RTE_ERR_UNSUPPORTED: return "unsupported";
        case RTE_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char *rte_last_error_string(void) { return g_err.c_str(); }
const char *rte_version(void) { return "librte 0.1 (sm_103a)"; }
uint64_t rte_kernel_launch_count(void) { return g_launches.load(); }

rte_status rte_set_allocator(rte_alloc_fn alloc, rte_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return fail(RTE_ERR_INVALID_ARG, "rte_set_allocator: give both callbacks or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return RTE_OK;
}

rte_status rte_plan_create(const rte_grid_desc *desc, const double *mua, const double *mus, const double *g,
                           void *cuda_stream, rte_plan **out) {
    return create(desc, mua, mus, g, (cudaStream_t)cuda_stream, out, current_allocator());
}

rte_status rte_plan_destroy(rte_plan *plan) {
    if (!plan) return fail(RTE_ERR_INVALID_ARG, "null plan");
    cudaStreamSynchronize(plan->st);
    destroy(plan);
    return RTE_OK;
}

rte_status rte_plan_footprint(const rte_grid_desc *d, uint64_t *bytes) {
    RT(validate_desc(d));
    if (!bytes) return fail(RTE_ERR_INVALID_ARG, "null output");
    const uint64_t V = (uint64_t)d->nx * d->ny * d->nz;
    const uint64_t M = d->real_radiance ? (uint64_t)(d->N + 1) * (d->N + 2) / 2 : (uint64_t)(d->N + 1) * (d->N + 1);
    const uint64_t esz = d->precision == RTE_FP64 ? 16 : 8;
    const uint64_t rsz = esz / 2;
    const bool slot = d->precision == RTE_FP64 ? plane_fits<double>(d->nx, d->ny) : plane_fits<float>(d->nx, d->ny);
    *bytes = 4 * M * V * esz + V * 4 * rsz + (slot ? (uint64_t)(d->N + 1) * V * rsz : 0) +
             (uint64_t)(d->nx + d->ny + d->nz) * (esz + rsz) + 4096;
    return RTE_OK;
}

rte_status rte_stability_limit_media(const rte_grid_desc *d, const double *mua, const double *mus, const double *g,
                                     double *dt) {
    RT(validate_desc(d));
    if (!mua || !mus || !g || !dt) return fail(RTE_ERR_INVALID_ARG, "null argument");
    const size_t V = (size_t)d->nx * d->ny * d->nz;
    std::vector<double> mub;
    std::vector<uint8_t> mask;
    layer_profile(d->nx, d->ny, d->nz, d->pml_cells, d->pml_mu0, d->pml_mu1, mub, mask);
    std::vector<double> ae(V), se(V);
    for (size_t v = 0; v < V; ++v) {
        ae[v] = mask[v] ? mub[v] : mua[v];
        se[v] = mask[v] ? 0.0 : mus[v];
    }
    auto cl = media_classes(V, ae.data(), se.data(), g, mask.data(), 1024);
    const int dims[3] = {d->nx, d->ny, d->nz};
    double kmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        double km = 0.0;
        for (int i = 0; i < dims[a]; ++i) km = std::max(km, std::fabs(wavenumber(i, dims[a], d->dx_mm)));
        kmax += km * km;
    }
    const double r = stability_from_classes(d->N, d->c_mm_per_ps, std::sqrt(kmax), cl, 256);
    if (r < 0.0) return fail(RTE_ERR_NOT_CONVERGED, "eigenvalue iteration did not converge");
    *dt = r;
    return RTE_OK;
}

rte_status rte_stability_limit(rte_plan *p, double *dt) {
    if (!p || !dt) return fail(RTE_ERR_INVALID_ARG, "null argument");
    if (p->dtstar < 0.0) {
        p->dtstar = stability_from_classes(p->d.N, p->d.c_mm_per_ps, p->kmax, p->classes, 256);
        if (p->dtstar < 0.0) return fail(RTE_ERR_NOT_CONVERGED, "eigenvalue iteration did not converge");
    }
    *dt = p->dtstar;
    return RTE_OK;
}

rte_status rte_set_state(rte_plan *p, const void *psi, int where) {
    if (!p || !psi || (where != RTE_HOST && where != RTE_DEVICE)) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    p->fw_valid = false;
    return p->d.precision == RTE_FP64 ? set_state_impl<double>(p, psi, where) : set_state_impl<float>(p, psi, where);
}

rte_status rte_get_state(rte_plan *p, void *psi, int where) {
    if (!p || !psi || (where != RTE_HOST && where != RTE_DEVICE)) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    return p->d.precision == RTE_FP64 ? get_state_impl<double>(p, psi, where) : get_state_impl<float>(p, psi, where);
}

rte_status rte_set_time(rte_plan *p, double t) {
    if (!p || !std::isfinite(t)) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    p->time = t;
    return RTE_OK;
}

rte_status rte_get_time(const rte_plan *p, double *t) {
    if (!p || !t) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    *t = p->time;
    return RTE_OK;
}

rte_status rte_set_sources(rte_plan *p, int n, const int64_t *voxel, const int *moment, const double *amp,
                           const double *t0, const double *fwhm) {
    if (!p || n < 0) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    if (n > 0 && (!voxel || !moment || !amp || !t0 || !fwhm)) return fail(RTE_ERR_INVALID_ARG, "null array");
    std::vector<double> mub;
    std::vector<uint8_t> mask;
    if (n > 0 && p->d.pml_cells > 0)
        layer_profile(p->d.nx, p->d.ny, p->d.nz, p->d.pml_cells, p->d.pml_mu0, p->d.pml_mu1, mub, mask);
    std::vector<int> stored(n);
    for (int q = 0; q < n; ++q) {
        if (voxel[q] < 0 || (size_t)voxel[q] >= p->V || moment[q] < 0 || moment[q] >= p->Mfull ||
            !std::isfinite(amp[q]))
            return fail(RTE_ERR_INVALID_ARG, "source index out of range");
        if (!mask.empty() && mask[voxel[q]]) return fail(RTE_ERR_INVALID_ARG, "source inside the layer");
        int l = 0;
        while ((l + 1) * (l + 1) <= moment[q]) ++l;
        const int m = moment[q] - l * l - l;
        if (p->real && m < 0)
            return fail(RTE_ERR_INVALID_ARG, "real-radiance plans take sources with m >= 0 (the pair is implied)");
        stored[q] = p->real ? l * (l + 1) / 2 + m : moment[q];
    }
    p->src_vox.assign(voxel, voxel + n);
    p->src_mom = stored;
    p->src_amp.assign(amp, amp + n);
    p->src_t0.assign(t0, t0 + n);
    p->src_fwhm.assign(fwhm, fwhm + n);
    if (p->sub) {
        p->sub->src_vox = p->src_vox;
        p->sub->src_mom = p->src_mom;
        p->sub->src_amp = p->src_amp;
        p->sub->src_t0 = p->src_t0;
        p->sub->src_fwhm = p->src_fwhm;
    }
    return RTE_OK;
}

rte_status rte_set_detectors(rte_plan *p, int n, const int64_t *voxel) {
    if (!p || n < 0 || (n > 0 && !voxel)) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    for (int q = 0; q < n; ++q)
        if (voxel[q] < 0 || (size_t)voxel[q] >= p->V) return fail(RTE_ERR_INVALID_ARG, "detector out of range");
    p->det_vox.assign(voxel, voxel + n);
    p->fw_valid = false;
    return RTE_OK;
}

rte_status rte_step(rte_plan *p, double dt, int nsteps, int allow_unstable, double *det_series, double *integral) {
    if (!p || nsteps < 0) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    p->fw_valid = false;
    return p->d.precision == RTE_FP64 ? step_impl<double>(p, dt, nsteps, allow_unstable, det_series, integral)
                                      : step_impl<float>(p, dt, nsteps, allow_unstable, det_series, integral);
}

rte_status rte_apply_transport(rte_plan *p, const void *in, void *out) {
    if (!p || !in || !out || in == out) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    rte_status s = p->d.precision == RTE_FP64 ? apply_impl<double>(p, in, out) : apply_impl<float>(p, in, out);
    if (s == RTE_OK) {
        cudaError_t e = cudaStreamSynchronize(p->st);
        if (e != cudaSuccess) return cuda_fail(e, "rte_apply_transport");
    }
    return s;
}

rte_status rte_solve_steady(rte_plan *p, double rtol, int restart, int max_iter, int *iters, double *rel_res) {
    if (!p || !(rtol > 0.0) || restart < 1 || restart > 63 || max_iter < 1)
        return fail(RTE_ERR_INVALID_ARG, "bad argument");
    p->fw_valid = false;
    return p->d.precision == RTE_FP64 ? solve_impl<double>(p, rtol, restart, max_iter, iters, rel_res)
                                      : solve_impl<float>(p, rtol, restart, max_iter, iters, rel_res);
}

rte_status rte_step_exponential(rte_plan *p, double dt, int nsteps) {
    if (!p) return fail(RTE_ERR_INVALID_ARG, "null plan");
    return p->d.precision == RTE_FP64 ? expo_impl<double>(p, dt, nsteps) : expo_impl<float>(p, dt, nsteps);
}

rte_status rte_step_group(rte_plan *const *plans, int nplans, const double *dt_ps, int nsteps,
                          double *const *det_series) {
    if (!plans || !dt_ps || nplans < 1 || nplans > kMaxGroup || nsteps < 0)
        return fail(RTE_ERR_INVALID_ARG, "need 1..8 plans, their dt and nsteps >= 0");
    for (int i = 0; i < nplans; ++i)
        if (!plans[i]) return fail(RTE_ERR_INVALID_ARG, "null plan");
    return plans[0]->d.precision == RTE_FP64 ? step_group_impl<double>(plans, nplans, dt_ps, nsteps, det_series)
                                             : step_group_impl<float>(plans, nplans, dt_ps, nsteps, det_series);
}

rte_status rte_set_schedule(rte_plan *p, int schedule, int graph_steps) {
    if (!p) return fail(RTE_ERR_INVALID_ARG, "null plan");
    if (schedule != RTE_SCHED_AUTO && schedule != RTE_SCHED_PLANE && schedule != RTE_SCHED_SPLIT)
        return fail(RTE_ERR_INVALID_ARG, "schedule must be RTE_SCHED_AUTO, RTE_SCHED_PLANE or RTE_SCHED_SPLIT");
    if (graph_steps != 0 && (graph_steps < 2 || graph_steps > 64 || graph_steps % 2))
        return fail(RTE_ERR_INVALID_ARG, "graph_steps must be 0 or even in 2..64");
    if (schedule == RTE_SCHED_PLANE) {
        const bool ok = p->d.precision == RTE_FP64 ? plane_ok<double>(p) : plane_ok<float>(p);
        if (!ok) return fail(RTE_ERR_UNSUPPORTED, "the fused plane path does not take this grid");
    }
    p->sched = schedule;
    p->gsteps = graph_steps;
    return RTE_OK;
}

rte_status rte_set_preconditioner(rte_plan *p, int kind) {
    if (!p || (kind != RTE_PREC_NONE && kind != RTE_PREC_LOW_ORDER)) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    p->prec = kind;
    return RTE_OK;
}

rte_status rte_forward(rte_plan *p, double dt, int nsteps, int K, const double *lo, const double *hi, double *y) {
    if (!p) return fail(RTE_ERR_INVALID_ARG, "null plan");
    return p->d.precision == RTE_FP64 ? forward_impl<double>(p, dt, nsteps, K, lo, hi, y)
                                      : forward_impl<float>(p, dt, nsteps, K, lo, hi, y);
}

rte_status rte_adjoint(rte_plan *p, const double *dLdy, double *ga, double *gs) {
    if (!p) return fail(RTE_ERR_INVALID_ARG, "null plan");
    return p->d.precision == RTE_FP64 ? adjoint_impl<double>(p, dLdy, ga, gs) : adjoint_impl<float>(p, dLdy, ga, gs);
}

rte_status rte_profile_enable(rte_plan *p, int enable) {
    if (!p) return fail(RTE_ERR_INVALID_ARG, "null plan");
    CK(cudaStreamSynchronize(p->st));
    prof_drain(p);
    p->prof_names.clear();
    p->prof_count.clear();
    p->prof_ms.clear();
    p->prof = enable != 0;
    return RTE_OK;
}

rte_status rte_profile_read(rte_plan *p, int max, char *names, int *launches, double *total_ms, int *n) {
    if (!p || max < 0 || !n) return fail(RTE_ERR_INVALID_ARG, "bad argument");
    CK(cudaStreamSynchronize(p->st));
    prof_drain(p);
    const int k = (int)p->prof_names.size();
    *n = k;
    for (int i = 0; i < k && i < max; ++i) {
        if (names) {
            std::strncpy(names + (size_t)i * 64, p->prof_names[i].c_str(), 63);
            names[(size_t)i * 64 + 63] = 0;
        }
        if (launches) launches[i] = p->prof_count[i];
        if (total_ms) total_ms[i] = p->prof_ms[i];
    }
    return RTE_OK;
}

}  // extern "C"
