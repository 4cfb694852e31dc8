/*
 * rte.h -- C ABI of librte, a single-GPU (sm_103a) implementation of the
 * pseudospectral spherical-harmonic (P_N) transport method of Powell, Cox &
 * Arridge, "A pseudospectral method for solution of the radiative transport
 * equation" (arXiv:1801.06364).
 *
 * The method (paper Sec. II): the radiance is expanded in (N+1)^2 complex
 * orthonormal spherical-harmonic moments psi_l^m(r, t) (Eq. 3); the streaming
 * term s.grad is applied in k-space through the alpha/beta recurrence of
 * Eq. 6 / Eq. 10; the attenuation mu_t - mu_s g^l (Henyey-Greenstein
 * scattering is diagonal in l, Eq. 5) is applied pointwise; a perfectly
 * matched layer (Eq. 12) absorbs outgoing light; time is advanced with the
 * explicit step of Eq. 11 and the steady state is found with a Krylov method
 * on the implicit operator (Sec. II.A).
 *
 * Readings of the paper that fix the arithmetic (the paper leaves them open):
 *   - orthonormal complex Y_l^m with the Condon-Shortley phase; moment index
 *     l*l + l + m;
 *   - forward DFT exp(-i k.r), unnormalised; derivative d/dx_j -> +i k_j
 *     (the printed Eq. 10 carries the opposite sign); the Nyquist wavenumber
 *     of an even axis is set to 0;
 *   - Eq. 11 read as psi <- psi - c dt (F^-1[psidot] + D_l psi) + c dt q with
 *     D_l = mu_a + mu_s (1 - g^l) in the domain and D_l = mu_b in the layer;
 *   - layer profile mu_b(d) = mu0 + (mu1 - mu0)(1 - cos(pi d / W)) / 2 with d
 *     the depth of the cell centre in cells, the largest value over the axes
 *     on which a cell lies in the layer; mu_s = 0 and q = 0 there (Eq. 12).
 *
 * Units: lengths mm, times ps, coefficients 1/mm.
 * Layout of every radiance field crossing this ABI: complex numbers
 * (interleaved re, im) in the plan precision, indexed [M][nz][ny][nx] with x
 * fastest, M = (N+1)^2 moments in the order l*l + l + m.
 * Voxel indices are flat: (z * ny + y) * nx + x.
 *
 * Ownership: the caller owns every pointer it passes and every buffer it
 * reads back; the plan owns its device state, workspace and tables, all
 * allocated stream-ordered on the plan's stream (cudaMallocAsync, or the
 * caller's allocator registered with rte_set_allocator) at plan creation (or
 * on first use by the steady and adjoint solvers) and freed by
 * rte_plan_destroy, so creating or destroying one plan does not wait for
 * the work of plans on other streams.
 * Errors: every call returns an rte_status and never aborts; after
 * RTE_ERR_INVALID_ARG, RTE_ERR_UNSTABLE_DT or RTE_ERR_NOT_CONVERGED the plan
 * stays usable. RTE_ERR_CUDA carries the CUDA error text in
 * rte_last_error_string().
 * Streams: all device work of a plan runs on the stream given at creation
 * (NULL = the legacy default stream). Calls that return host data
 * synchronise that stream.
 * Threads: distinct plans may be driven from distinct host threads at the
 * same time (one thread per plan); kernel attributes that are global to the
 * process are set identically by every caller.
 *
 * Against a minimal plan/step/solve/adjoint interface this ABI differs in
 * two ways: the detector gates are arguments of rte_forward, the checkpointed
 * forward sweep, which rte_adjoint then differentiates (so the gradient call
 * takes only dL/dy and the two output maps); and a caller's caching
 * allocator is registered once for the process (rte_set_allocator) rather
 * than per plan.
 */
#ifndef RTE_H_
#define RTE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RTE_OK = 0,
    RTE_ERR_INVALID_ARG = 1,
    RTE_ERR_OOM = 2,
    RTE_ERR_UNSTABLE_DT = 3,
    /* The state holds a NaN or an infinity. The kernels that write the
     * updated state set a device flag when an output of the kx = 0 column is
     * not finite; a non-finite value anywhere in a z plane reaches that column
     * through the x transform within one step. rte_step reports it when it
     * synchronises (an output pointer is given, or nsteps >= 1024) and every
     * 1024 steps of a longer call; otherwise the flag stays set and the next
     * rte_step that synchronises, rte_get_state, rte_forward or rte_adjoint
     * reports it. Reporting clears the flag, and so does rte_set_state. The
     * plan stays usable: set a finite state and step again. Operator
     * applications (rte_apply_transport, the steady solver) do not raise the
     * flag; rte_solve_steady returns this status for a non-finite residual. */
    RTE_ERR_NONFINITE = 4,
    RTE_ERR_NOT_CONVERGED = 5,
    /* A bulk copy into shared memory did not complete within the plane
     * kernel's bounded wait (about 2^24 tests of its barrier); the kernel
     * abandoned the step and the state is not valid. Reported, and cleared,
     * like RTE_ERR_NONFINITE. Not expected in normal operation. */
    RTE_ERR_TIMEOUT = 6,
    RTE_ERR_CUDA = 7,
    RTE_ERR_UNSUPPORTED = 8,
    RTE_ERR_STATE = 9
} rte_status;

enum { RTE_FP32 = 0, RTE_FP64 = 1 };
enum { RTE_HOST = 0, RTE_DEVICE = 1 };
enum { RTE_PREC_NONE = 0, RTE_PREC_LOW_ORDER = 1 };
enum { RTE_SCHED_AUTO = 0, RTE_SCHED_PLANE = 1, RTE_SCHED_SPLIT = 2 };

/* Grid, angular order, speed of light and layer of one problem. Each of
 * nx, ny, nz must be >= 4, at most 1024, and a product of 2, 3 and 5. */
typedef struct {
    int nx, ny, nz;
    double dx_mm;             /* isotropic voxel size */
    int N;                    /* P_N order, 0 <= N <= 21 */
    double c_mm_per_ps;       /* speed of light in the medium */
    int pml_cells;            /* layer thickness W on every face; 0 = periodic */
    double pml_mu0, pml_mu1;  /* layer loss at the inner edge / at the boundary */
    int precision;            /* RTE_FP32 or RTE_FP64 */
    /* 1 = the radiance is real (every physical problem: real optical maps,
     * real initial state, sources with real amplitudes). Then
     * psi_l^{-m} = (-1)^m conj(psi_l^m) (orthonormal complex harmonics with the
     * Condon-Shortley phase), and the plan stores and updates the m >= 0
     * moments only, (N+1)(N+2)/2 of them; the m < 0 moments of any field
     * passed in are ignored and those of fields passed out are rebuilt from
     * the relation. A source in moment (l, m > 0) then stands for the pair
     * (l, +-m) with amplitudes amp and (-1)^m amp; sources with m < 0 are
     * rejected. 0 = general complex moments, all (N+1)^2 stored. */
    int real_radiance;
} rte_grid_desc;

typedef struct rte_plan rte_plan;

/* Text of a status code. */
const char *rte_status_string(rte_status s);
/* Text of the last CUDA or argument error seen by this thread. */
const char *rte_last_error_string(void);
/* Library version string. */
const char *rte_version(void);

/*
 * Create a plan (Sec. II.A-B): copies the optical maps mua, mus, g (HOST
 * arrays of V = nx*ny*nz doubles) and folds the layer into them (Eq. 12:
 * inside the layer mu_a -> mu_b, mu_s -> 0). The state starts at zero, time
 * at 0. cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Returns RTE_ERR_INVALID_ARG on a bad descriptor or a non-finite or negative
 * coefficient, RTE_ERR_OOM when device memory runs out.
 */
rte_status rte_plan_create(const rte_grid_desc *desc, const double *mua, const double *mus,
                           const double *g, void *cuda_stream, rte_plan **out);
rte_status rte_plan_destroy(rte_plan *plan);

/*
 * Device memory from the caller (the ownership rule of the boundary; the
 * paper has no counterpart). Plans created after this call take every device
 * buffer they own from alloc and give it back through release; plans created
 * before keep the allocator they were created with (an FP64 twin that an
 * FP32 plan creates for its refinement residuals takes its parent's).
 *   alloc(bytes, stream, ctx): device memory of at least `bytes` bytes on the
 *     current device, 256-byte aligned, usable in stream order on `stream`
 *     (the plan's cudaStream_t); NULL when it cannot (the calling rte_
 *     function then returns RTE_ERR_OOM).
 *   release(ptr, stream, ctx): takes back a pointer alloc returned; the plan's
 *     work on `stream` that used it may still be in flight (a stream-ordered
 *     allocator, such as a caching allocator keyed by stream, handles that).
 * The callbacks are called from the thread that calls into the plan, and
 * never while a stream is being captured. alloc = release = NULL returns to
 * cudaMallocAsync / cudaFreeAsync on the plan's stream. Returns
 * RTE_ERR_INVALID_ARG when exactly one of the two is NULL. Host-only.
 */
typedef void *(*rte_alloc_fn)(uint64_t bytes, void *stream, void *ctx);
typedef void (*rte_free_fn)(void *ptr, void *stream, void *ctx);
rte_status rte_set_allocator(rte_alloc_fn alloc, rte_free_fn release, void *ctx);

/* Bytes of device memory a time-domain plan allocates (state, workspace,
 * media, tables), without creating it. Host-only. */
rte_status rte_plan_footprint(const rte_grid_desc *desc, uint64_t *bytes);

/*
 * Largest stable explicit step (Sec. II.A asserts conditional stability of
 * Eq. 11). dt* = min over media classes and |k| = k_max j / 256, j = 0..256,
 * of min over eigenvalues lam of M_k = -c (S(k) + D) of 2 Re(-lam) / |lam|^2.
 * Media classes: the distinct (mu_a, mu_s, g) of the layer and of the domain;
 * a domain with more than 1024 distinct triples is represented by its least
 * damped triple (min mu_a, min mu_s, max g). k_max is the largest grid |k|.
 * rte_stability_limit_media is host-only and needs no GPU.
 */
rte_status rte_stability_limit_media(const rte_grid_desc *desc, const double *mua,
                                     const double *mus, const double *g, double *dt_max_ps);
rte_status rte_stability_limit(rte_plan *plan, double *dt_max_ps);

/* Replace / read the state psi(r) (layout above, plan precision). where is
 * RTE_HOST or RTE_DEVICE. The state lives on the device in a transformed
 * representation; these calls convert. rte_get_state synchronises. */
rte_status rte_set_state(rte_plan *plan, const void *psi, int where);
rte_status rte_get_state(rte_plan *plan, void *psi, int where);
/* Current simulation time (ps) used to evaluate pulsed sources. */
rte_status rte_set_time(rte_plan *plan, double t_ps);
rte_status rte_get_time(const rte_plan *plan, double *t_ps);

/*
 * Point sources (host arrays of n entries): moment `moment` at voxel `voxel`
 * receives the density q(t) = amp * exp(-4 ln2 ((t - t0)/fwhm)^2) / dx^3 per
 * mm^3, or amp / dx^3 when fwhm <= 0 (continuous wave). Sources inside the
 * layer are rejected (Eq. 12 sets q = 0 there). n = 0 clears them.
 */
rte_status rte_set_sources(rte_plan *plan, int n, const int64_t *voxel, const int *moment,
                           const double *amp, const double *t0_ps, const double *fwhm_ps);

/* Detector voxels (host array of n flat indices). Each readout is
 * Re psi_0^0 at that voxel. n = 0 clears them. */
rte_status rte_set_detectors(rte_plan *plan, int n, const int64_t *voxel);

/*
 * nsteps explicit steps of Eq. 11 from the current state and time:
 *   psi <- psi - c dt (F^-1[psidot] + D_l psi) + c dt q(t),  t += dt.
 * Before each step s the state it starts from is read out:
 *   det_series[s * ndet + d] = Re psi_00(detector d)            (HOST, may be NULL)
 *   integral[2 s], integral[2 s + 1] = re, im of sum_r psi_00 dx^3 (HOST, may be NULL)
 * Returns RTE_ERR_UNSTABLE_DT when dt exceeds 1.0001 * rte_stability_limit
 * (computed once per plan) unless allow_unstable != 0. Synchronises when an
 * output pointer is given.
 */
rte_status rte_step(rte_plan *plan, double dt_ps, int nsteps, int allow_unstable,
                    double *det_series, double *integral);

/*
 * nsteps exponential steps of any dt_ps > 0 for a homogeneous medium: the
 * arbitrary-step scheme the paper names for homogeneous media (Sec. V). Per
 * wavevector k the moments advance by E_k = expm(-c dt (S(k) + D)), S(k) the
 * streaming matrix of Eq. 10, D = diag(mu_a + mu_s (1 - g^l)); the state
 * goes to full k-space by a z-DFT and back. E_k is built on the device in
 * FP64 (Taylor series with scaling and squaring) for the first call with a
 * given dt and kept (M^2 V complex elements of plan precision). Needs a
 * uniform medium, no layer, no sources, the full moment layout, N <= 7 and
 * nz in 32, 64, 96, 128, 160, 256; otherwise RTE_ERR_UNSUPPORTED and the
 * plan is unchanged. No readouts; advances the plan time; synchronises.
 */
rte_status rte_step_exponential(rte_plan *plan, double dt_ps, int nsteps);

/*
 * out = T in, T psi = F^-1[psidot] + D_l psi: the transport operator of the
 * paper's stages 1-2 (Sec. III). in and out are DEVICE fields in the ABI
 * layout, plan precision; they may not alias. The plan state is unchanged.
 */
rte_status rte_apply_transport(rte_plan *plan, const void *psi_in, void *psi_out);

/*
 * Steady state (Sec. II.A: a Krylov solve with the implicit operator):
 * T psi = q with q the plan's sources taken at their amplitude (as continuous
 * wave). Restarted GMRES(restart) from psi = 0 in the inner product
 * <u, v> = sum (2l+1) conj(u) v, dot products and norms accumulated in FP64
 * on the device. For RTE_FP32 plans the residual is recomputed with an FP64
 * operator and corrected by FP32 GMRES solves (iterative refinement) until
 * |q - T psi| / |q| <= rtol. The solution replaces the state. iters receives
 * the total Arnoldi steps, rel_res the final relative residual.
 * restart is 1..63. Returns RTE_ERR_NOT_CONVERGED after max_iter steps.
 * GMRES is right-preconditioned as rte_set_preconditioner selects (the
 * residual it reports and tests is that of T psi = q either way).
 */
rte_status rte_solve_steady(rte_plan *plan, double rtol, int restart, int max_iter, int *iters,
                            double *rel_res);

/*
 * nsteps explicit steps (as rte_step) of a group of plans with one launch of
 * each step pass for the whole group: the z-streaming and plane passes run
 * their work items over the plans (the serving loop groups same-shape
 * requests this way). Up to 8 plans; all must share nx, ny, nz, N,
 * precision, real_radiance and the stream they were created on (the work runs
 * there), and take the fused plane path (RTE_ERR_UNSUPPORTED otherwise).
 * Each plan keeps its own media, layer, sources, detectors, state, time and
 * dt: dt_ps[i] is plan i's step (checked against its stability limit as
 * rte_step does). det_series[i] (det_series or its entries may be NULL)
 * receives plan i's readouts as rte_step's det_series. Each plan's results
 * are bitwise the same as from rte_step on that plan alone. Synchronises
 * the stream when a readout pointer is given or nsteps >= 1024, and then
 * reports a non-finite state of any plan as RTE_ERR_NONFINITE.
 */
rte_status rte_step_group(rte_plan *const *plans, int nplans, const double *dt_ps, int nsteps,
                          double *const *det_series);

/*
 * Scheduling of a plan's steps and operator applications (no counterpart in
 * the paper; the serving autotuner sets it per grid, order and precision).
 * schedule: RTE_SCHED_AUTO (the default) takes the fused plane path (a z
 * pass with the streaming coupling, then one fused pass per moment and z
 * plane, 5 sweeps of the state) where the grid allows it and the split passes
 * (z, inverse y, x with the pointwise stage, forward y with the coupling, 10
 * sweeps) elsewhere; RTE_SCHED_PLANE requires the plane path
 * (RTE_ERR_UNSUPPORTED where it does not fit); RTE_SCHED_SPLIT always takes the
 * split passes. The two paths compute the same step with FP32 rounding in a
 * different order. graph_steps: rte_step replays runs of this many steps
 * (even, 2..64; default 2) from one captured CUDA graph; 0 launches every
 * kernel directly. Returns RTE_ERR_INVALID_ARG for other values.
 */
rte_status rte_set_schedule(rte_plan *plan, int schedule, int graph_steps);

/*
 * Right preconditioner of rte_solve_steady's GMRES (no counterpart in the
 * paper, which names only a Krylov method). RTE_PREC_LOW_ORDER (the
 * default): on the l <= 1 moments the exact inverse, per wavevector, of the
 * transport operator of a homogeneous medium with D_l = Dbar_l, the interior
 * mean of mu_a + mu_s (1 - g^l); the l >= 2 moments are divided by Dbar_l.
 * It needs N >= 1 (N = 0 plans apply only the scaling). It pays where the
 * interior dominates the slow modes (diffusive media with small mu_a and a
 * strongly absorbing layer); where a weakly absorbing, non-scattering layer
 * fills most of the grid, plain GMRES can converge faster, because a
 * constant-coefficient operator cannot match both regions. RTE_PREC_NONE:
 * plain GMRES.
 * Returns RTE_ERR_INVALID_ARG for another kind.
 */
rte_status rte_set_preconditioner(rte_plan *plan, int kind);

/*
 * Forward sweep for the adjoint: nsteps explicit steps from the current state
 * and time, keeping a checkpoint of the state every ckpt_every steps, and the
 * gated readouts y_d = sum_s dt * Re psi_00(r_d, t_s) over the pre-step
 * states with gate_lo[d] <= t_s <= gate_hi[d] (HOST arrays of ndet; y is a
 * HOST array of ndet).
 */
rte_status rte_forward(rte_plan *plan, double dt_ps, int nsteps, int ckpt_every,
                       const double *gate_lo, const double *gate_hi, double *y);

/*
 * Gradient of a loss L(y) with respect to mu_a(r) and mu_s(r) by the discrete
 * adjoint of the last rte_forward sweep, given dL/dy (HOST array of ndet).
 * grad_mua and grad_mus are DEVICE arrays of V doubles, overwritten; both
 * are zero in the layer, where mu_a and mu_s do not enter. The adjoint step is
 * the forward pipeline with the streaming sign reversed applied to
 * W^-2 lambda, W = diag(sqrt((2l+1)/4pi)); segments between checkpoints are
 * recomputed. The plan state is left at the end of the forward sweep.
 */
rte_status rte_adjoint(rte_plan *plan, const double *dL_dy, double *grad_mua, double *grad_mus);

/*
 * Per-kernel timing with CUDA events recorded on the plan's stream around
 * every launch (off by default). rte_profile_enable synchronises and clears
 * the records. rte_profile_read synchronises and returns, for up to max
 * distinct kernels, the name (NUL-terminated, 64-byte slots in names), the
 * number of launches and the summed event-to-event milliseconds; n receives
 * the number of distinct kernels recorded.
 */
rte_status rte_profile_enable(rte_plan *plan, int enable);
rte_status rte_profile_read(rte_plan *plan, int max, char *names, int *launches, double *total_ms, int *n);

/*
 * rte_apply_transport_noalloc -- the paper has no counterpart to this entry
 * point. It is for callers that cannot allocate device memory: code that runs
 * inside another framework's memory pool or under a fixed device-memory
 * budget, and plug-ins that are not allowed to call cudaMalloc. It computes
 * the same out = T in as rte_apply_transport, but without a plan: desc, mua,
 * mus and g are as for rte_plan_create (HOST arrays of V doubles), psi_in and
 * psi_out are DEVICE fields in the ABI layout and the desc precision (not
 * aliased), and the work runs on cuda_stream (NULL = legacy default stream).
 * desc->real_radiance must be 0 or 1 but does not change the work: every
 * (N+1)^2 moment is computed.
 * Every table and work buffer lives in one 32 MiB device array compiled into
 * the library, which each GPU that loads the library holds until the process
 * exits; a problem whose tables plus three field-sized buffers exceed it is
 * rejected with RTE_ERR_INVALID_ARG, and rte_last_error_string() gives the
 * bytes it would need. The call makes no cudaMalloc or cudaFree; it looks up
 * the array's device address in the current context on every call. All calls
 * share the one array: calls whose
 * GPU work overlaps (other streams, other host threads) race on it and
 * corrupt each other's results. The call synchronises cuda_stream.
 */
rte_status rte_apply_transport_noalloc(const rte_grid_desc *desc, const double *mua, const double *mus,
                                       const double *g, const void *psi_in, void *psi_out,
                                       void *cuda_stream);

/*
 * Measurement aid (no counterpart in the paper): the FMA throughput of the
 * current device in FLOP/s (2 per fused multiply-add) for precision RTE_FP32
 * or RTE_FP64, from this library's own kernel (8 independent FMA chains per
 * thread, 8 CTAs of 256 threads per SM, about 20 ms). It bounds the FP64
 * explicit step, which is limited by the FP64 pipe on B300. Allocates and
 * frees a few bytes of device memory; runs on the legacy default stream and
 * synchronises it.
 */
rte_status rte_fma_peak(int precision, double *flop_per_s);

/* Device kernels launched by this library since the process started. */
uint64_t rte_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RTE_H_ */
