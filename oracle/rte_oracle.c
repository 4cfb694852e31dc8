/*
 * rte_oracle.c -- plain, slow, FP64 CPU oracle for the pseudospectral P_N
 * radiative-transport method of Powell, Cox & Arridge, "A pseudospectral
 * method for solution of the radiative transport equation" (arXiv:1801.06364).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it. It shares no code with the CUDA
 * library; it has its own DFT/FFT, its own coefficient code and its own
 * solvers, written for readability rather than speed.
 *
 * Conventions (the paper leaves these open; the readings are listed here so
 * that the file stands on its own):
 *   - Moments: complex orthonormal spherical harmonics with the Condon-Shortley
 *     phase, index(l, m) = l*l + l + m, M = (N+1)^2 moments (Eq. 3, Sec. II.A).
 *   - Fields are stored [M][nz][ny][nx], x fastest, complex128.
 *   - Forward DFT uses exp(-i k.r) (Eq. 8, unnormalised); the inverse carries
 *     1/n per axis.
 *   - Spatial derivative d/dx_j becomes +i k_j in k-space. The printed Eq. 10
 *     carries -i k_j, which with the exp(-i k.r) forward transform of Eq. 8 is
 *     the negative of the streaming term of Eq. 6; the oracle follows Eq. 6.
 *   - Wavenumber of index i on an axis of n points: 2*pi*i'/(n*dx) with
 *     i' = i (2i < n), 0 (2i == n, the Nyquist index), i - n (2i > n).
 *   - Time step (Eq. 11, signs read so that the scheme decays):
 *       psi <- psi - c dt ( F^-1[psidot] + D_l psi ) + c dt q,
 *     with D_l = mu_a + mu_s (1 - g^l) inside Omega and D_l = mu_b in the PML
 *     (Eq. 12: there mu_s = 0 and q = 0).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>

typedef double complex zc;

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Angular coefficients, Eq. 6                                              */
/* ------------------------------------------------------------------------ */

int orc_num_moments(int N) { return (N + 1) * (N + 1); }
int orc_moment_index(int l, int m) { return l * l + l + m; }

/* alpha_l^m = sqrt((l+m)(l-m)), Eq. 6 */
double orc_alpha(int l, int m) {
    double p = (double)(l + m) * (double)(l - m);
    return p > 0.0 ? sqrt(p) : 0.0;
}

/* beta_l^m = sqrt((l+m)(l+m-1)), Eq. 6 */
double orc_beta(int l, int m) {
    double p = (double)(l + m) * (double)(l + m - 1);
    return p > 0.0 ? sqrt(p) : 0.0;
}

static int moment_exists(int N, int l, int m) {
    return l >= 0 && l <= N && m >= -l && m <= l;
}

/*
 * The k-space streaming term for output moment (l, m): Eq. 10 with the
 * derivative read as d/dx_j -> +i k_j (see the header). Writes up to six
 * (input moment index, coefficient) pairs; returns how many.
 *
 *  psidot_l^m = 1/(2l+1) * (  i kz [ a_{l+1}^m psi_{l+1}^m + a_l^m psi_{l-1}^m ]
 *                 - 1/2 (i kx + ky) [ b_l^m psi_{l-1}^{m-1} - b_{l+1}^{-m+1} psi_{l+1}^{m-1} ]
 *                 - 1/2 (i kx - ky) [ -b_l^{-m} psi_{l-1}^{m+1} + b_{l+1}^{m+1} psi_{l+1}^{m+1} ] )
 *
 * Terms whose moment lies outside 0 <= l' <= N, |m'| <= l' are dropped (the
 * P_N closure of Sec. II.A).
 */
int orc_streaming_terms(int N, int l, int m, double kx, double ky, double kz,
                        int *src, zc *coef) {
    int n = 0;
    const double inv = 1.0 / (2.0 * l + 1.0);
    const zc ikz = I * kz;
    const zc pxy = I * kx + ky;   /* (d/dx - i d/dy) -> i kx + ky */
    const zc mxy = I * kx - ky;   /* (d/dx + i d/dy) -> i kx - ky */
    if (moment_exists(N, l + 1, m)) {
        src[n] = orc_moment_index(l + 1, m); coef[n] = inv * ikz * orc_alpha(l + 1, m); n++;
    }
    if (moment_exists(N, l - 1, m)) {
        src[n] = orc_moment_index(l - 1, m); coef[n] = inv * ikz * orc_alpha(l, m); n++;
    }
    if (moment_exists(N, l - 1, m - 1)) {
        src[n] = orc_moment_index(l - 1, m - 1); coef[n] = -0.5 * inv * pxy * orc_beta(l, m); n++;
    }
    if (moment_exists(N, l + 1, m - 1)) {
        src[n] = orc_moment_index(l + 1, m - 1); coef[n] = 0.5 * inv * pxy * orc_beta(l + 1, -m + 1); n++;
    }
    if (moment_exists(N, l - 1, m + 1)) {
        src[n] = orc_moment_index(l - 1, m + 1); coef[n] = 0.5 * inv * mxy * orc_beta(l, -m); n++;
    }
    if (moment_exists(N, l + 1, m + 1)) {
        src[n] = orc_moment_index(l + 1, m + 1); coef[n] = -0.5 * inv * mxy * orc_beta(l + 1, m + 1); n++;
    }
    return n;
}

/* out = S(k) in for one k-point (Eq. 10). in/out have M entries. */
void orc_kspace_streaming(int N, double kx, double ky, double kz, const zc *in, zc *out) {
    int src[6];
    zc coef[6];
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            int n = orc_streaming_terms(N, l, m, kx, ky, kz, src, coef);
            zc acc = 0.0;
            for (int t = 0; t < n; ++t) acc += coef[t] * in[src[t]];
            out[orc_moment_index(l, m)] = acc;
        }
}

/* out = S(k)^H in: the conjugate transpose of the same coefficients. */
void orc_kspace_streaming_adjoint(int N, double kx, double ky, double kz, const zc *in, zc *out) {
    int M = orc_num_moments(N);
    int src[6];
    zc coef[6];
    for (int j = 0; j < M; ++j) out[j] = 0.0;
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            int row = orc_moment_index(l, m);
            int n = orc_streaming_terms(N, l, m, kx, ky, kz, src, coef);
            for (int t = 0; t < n; ++t) out[src[t]] += conj(coef[t]) * in[row];
        }
}

/* Dense M x M matrix of S(k), row-major: mat[row*M + col]. */
void orc_streaming_matrix(int N, double kx, double ky, double kz, zc *mat) {
    int M = orc_num_moments(N);
    int src[6];
    zc coef[6];
    memset(mat, 0, sizeof(zc) * (size_t)M * M);
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            int row = orc_moment_index(l, m);
            int n = orc_streaming_terms(N, l, m, kx, ky, kz, src, coef);
            for (int t = 0; t < n; ++t) mat[(size_t)row * M + src[t]] += coef[t];
        }
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms (Eq. 7-8 on the collocation grid, Sec. II.A)  */
/* ------------------------------------------------------------------------ */

double orc_wavenumber(int i, int n, double dx) {
    int ip;
    if (2 * i < n) ip = i;
    else if (2 * i == n) ip = 0;
    else ip = i - n;
    return 2.0 * ORC_PI * (double)ip / ((double)n * dx);
}

/* Textbook O(n^2) DFT: out[k] = sum_j in[j] exp(sign 2 pi i j k / n). */
void orc_dft_naive(const zc *in, zc *out, int n, int sign) {
    for (int k = 0; k < n; ++k) {
        zc acc = 0.0;
        for (int j = 0; j < n; ++j) {
            long jk = ((long)j * k) % n;
            double ang = sign * 2.0 * ORC_PI * (double)jk / (double)n;
            acc += in[j] * (cos(ang) + I * sin(ang));
        }
        out[k] = acc;
    }
}

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * Recursive decimation-in-time FFT for any n: with p the smallest prime factor
 * of n and q = n/p, the p decimated subsequences x[r + p j] are transformed
 * (length q) and combined as X[k] = sum_r w_n^{r k} Y_r[k mod q].
 * tw[j] = exp(sign 2 pi i j / ntw) with n dividing ntw.
 */
static void fft_rec(const zc *x, ptrdiff_t xs, zc *X, int n, const zc *tw, int ntw) {
    if (n == 1) { X[0] = x[0]; return; }
    int p = smallest_factor(n);
    int q = n / p;
    zc *Y = (zc *)malloc(sizeof(zc) * (size_t)n);
    for (int r = 0; r < p; ++r) fft_rec(x + r * xs, xs * p, Y + (size_t)r * q, q, tw, ntw);
    int step = ntw / n;
    for (int k = 0; k < n; ++k) {
        zc acc = 0.0;
        for (int r = 0; r < p; ++r) acc += tw[(size_t)(((long)r * k) % n) * step] * Y[(size_t)r * q + (k % q)];
        X[k] = acc;
    }
    free(Y);
}

static void make_twiddles(zc *tw, int n, int sign) {
    for (int j = 0; j < n; ++j) {
        double ang = sign * 2.0 * ORC_PI * (double)j / (double)n;
        tw[j] = cos(ang) + I * sin(ang);
    }
}

void orc_fft(const zc *in, zc *out, int n, int sign) {
    zc *tw = (zc *)malloc(sizeof(zc) * (size_t)n);
    make_twiddles(tw, n, sign);
    fft_rec(in, 1, out, n, tw, n);
    free(tw);
}

/* Transform every line of a [nz][ny][nx] field along one axis, in place. */
static void fft_axis(zc *f, int nx, int ny, int nz, int axis, int sign, const zc *tw) {
    int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    ptrdiff_t stride = axis == 0 ? 1 : (axis == 1 ? nx : (ptrdiff_t)nx * ny);
    int nlines = nx * ny * nz / n;
    #pragma omp parallel
    {
        zc *a = (zc *)malloc(sizeof(zc) * (size_t)n);
        zc *b = (zc *)malloc(sizeof(zc) * (size_t)n);
        #pragma omp for schedule(static)
        for (int line = 0; line < nlines; ++line) {
            ptrdiff_t base;
            if (axis == 0) base = (ptrdiff_t)line * nx;
            else if (axis == 1) base = (ptrdiff_t)(line / nx) * nx * ny + (line % nx);
            else base = line;
            for (int j = 0; j < n; ++j) a[j] = f[base + j * stride];
            fft_rec(a, 1, b, n, tw, n);
            for (int j = 0; j < n; ++j) f[base + j * stride] = b[j];
        }
        free(a);
        free(b);
    }
}

/* Unnormalised 3D DFT of one [nz][ny][nx] field, in place. */
void orc_fft3d(zc *f, int nx, int ny, int nz, int sign) {
    int dims[3] = {nx, ny, nz};
    for (int axis = 0; axis < 3; ++axis) {
        int n = dims[axis];
        zc *tw = (zc *)malloc(sizeof(zc) * (size_t)n);
        make_twiddles(tw, n, sign);
        fft_axis(f, nx, ny, nz, axis, sign, tw);
        free(tw);
    }
}

/* Brute-force 3D DFT (all V^2 terms), for tiny grids only. */
void orc_dft3d_naive(const zc *in, zc *out, int nx, int ny, int nz, int sign) {
    for (int kz = 0; kz < nz; ++kz)
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx < nx; ++kx) {
                zc acc = 0.0;
                for (int z = 0; z < nz; ++z)
                    for (int y = 0; y < ny; ++y)
                        for (int x = 0; x < nx; ++x) {
                            double ph = (double)x * kx / nx + (double)y * ky / ny + (double)z * kz / nz;
                            double ang = sign * 2.0 * ORC_PI * ph;
                            acc += in[((size_t)z * ny + y) * nx + x] * (cos(ang) + I * sin(ang));
                        }
                out[((size_t)kz * ny + ky) * nx + kx] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* Perfectly matched layer, Sec. II.B (Eq. 12) with a half-cosine profile    */
/* ------------------------------------------------------------------------ */

/* Depth (in cells, cell centres) of index i into a layer W cells thick at
 * either end of an axis of n cells; 0 when i is inside the real domain. */
static double pml_depth(int i, int n, int W) {
    if (i < W) return (double)(W - i) - 0.5;
    if (i >= n - W) return (double)(i - (n - W)) + 0.5;
    return 0.0;
}

/*
 * mu_b(d) = mu0 + (mu1 - mu0) (1 - cos(pi d / W)) / 2 along each axis, the
 * largest over the axes on which the cell lies in the layer. mask = 1 in the
 * layer, 0 in Omega. W = 0 gives no layer.
 */
void orc_pml_profile(int nx, int ny, int nz, int W, double mu0, double mu1,
                     double *mub, unsigned char *mask) {
    int dims[3] = {nx, ny, nz};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int idx[3] = {x, y, z};
                double best = 0.0;
                int in = 0;
                for (int a = 0; a < 3; ++a) {
                    if (W <= 0) continue;
                    if (idx[a] < W || idx[a] >= dims[a] - W) {
                        double d = pml_depth(idx[a], dims[a], W);
                        double v = mu0 + (mu1 - mu0) * 0.5 * (1.0 - cos(ORC_PI * d / W));
                        if (!in || v > best) best = v;
                        in = 1;
                    }
                }
                size_t v = ((size_t)z * ny + y) * nx + x;
                mub[v] = in ? best : 0.0;
                mask[v] = (unsigned char)in;
            }
}

/* ------------------------------------------------------------------------ */
/* Transport operator                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, nx, ny, nz;
    double dx;            /* mm */
    double c;             /* mm/ps */
    const double *mua;    /* [V] absorption inside Omega, mu_b in the PML */
    const double *mus;    /* [V] scattering inside Omega, 0 in the PML */
    const double *g;      /* [V] Henyey-Greenstein anisotropy */
} orc_medium;

/* Attenuation of moment l at voxel v: mu_t - mu_s g^l = mu_a + mu_s (1 - g^l)
 * (Eq. 6, 11; in-scattering of the HG phase function is diagonal, Eq. 5). */
static double damping(const orc_medium *p, size_t v, int l) {
    return p->mua[v] + p->mus[v] * (1.0 - pow(p->g[v], (double)l));
}

/* out = F^-1[ S(k) F[psi] ] for all moments, stage 1 of Sec. III.
 * adjoint != 0 applies S(k)^H instead (used by the adjoint sweep). */
static void apply_streaming_impl(const orc_medium *p, const zc *psi, zc *out, int adjoint) {
    const int N = p->N, M = orc_num_moments(N);
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t V = (size_t)nx * ny * nz;
    zc *hat = (zc *)malloc(sizeof(zc) * V * M);
    memcpy(hat, psi, sizeof(zc) * V * M);
    for (int j = 0; j < M; ++j) orc_fft3d(hat + (size_t)j * V, nx, ny, nz, -1);
    #pragma omp parallel
    {
        zc *a = (zc *)malloc(sizeof(zc) * M);
        zc *b = (zc *)malloc(sizeof(zc) * M);
        #pragma omp for schedule(static)
        for (long kv = 0; kv < (long)V; ++kv) {
            int ix = (int)(kv % nx), iy = (int)((kv / nx) % ny), iz = (int)(kv / ((long)nx * ny));
            double kx = orc_wavenumber(ix, nx, p->dx);
            double ky = orc_wavenumber(iy, ny, p->dx);
            double kz = orc_wavenumber(iz, nz, p->dx);
            for (int j = 0; j < M; ++j) a[j] = hat[(size_t)j * V + kv];
            if (adjoint) orc_kspace_streaming_adjoint(N, kx, ky, kz, a, b);
            else orc_kspace_streaming(N, kx, ky, kz, a, b);
            for (int j = 0; j < M; ++j) out[(size_t)j * V + kv] = b[j];
        }
        free(a);
        free(b);
    }
    free(hat);
    const double scale = 1.0 / (double)V;
    for (int j = 0; j < M; ++j) {
        orc_fft3d(out + (size_t)j * V, nx, ny, nz, +1);
        for (size_t v = 0; v < V; ++v) out[(size_t)j * V + v] *= scale;
    }
}

void orc_apply_streaming(const orc_medium *p, const zc *psi, zc *out) {
    apply_streaming_impl(p, psi, out, 0);
}

/* T psi = F^-1[psidot] + D psi: the transport operator of stages 1-2, Sec. III. */
static void apply_T_impl(const orc_medium *p, const zc *psi, zc *out, int adjoint) {
    const int N = p->N;
    const size_t V = (size_t)p->nx * p->ny * p->nz;
    apply_streaming_impl(p, psi, out, adjoint);
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            size_t j = (size_t)orc_moment_index(l, m);
            for (size_t v = 0; v < V; ++v) out[j * V + v] += damping(p, v, l) * psi[j * V + v];
        }
}

void orc_apply_T(const orc_medium *p, const zc *psi, zc *out) { apply_T_impl(p, psi, out, 0); }
void orc_apply_T_adjoint(const orc_medium *p, const zc *psi, zc *out) { apply_T_impl(p, psi, out, 1); }

/* ------------------------------------------------------------------------ */
/* Sources and the explicit time step, Eq. 11                                */
/* ------------------------------------------------------------------------ */

/* Source density q at time t (units of Eq. 1, per mm^3): a Gaussian pulse of
 * full width at half maximum fwhm centred at t0, or a constant when fwhm <= 0. */
double orc_source_density(double t, double amp, double t0, double fwhm, double dx) {
    double vol = dx * dx * dx;
    if (fwhm <= 0.0) return amp / vol;
    double u = (t - t0) / fwhm;
    return amp * exp(-4.0 * log(2.0) * u * u) / vol;
}

/*
 * nsteps explicit steps of Eq. 11 starting from time t_start:
 *   psi_{s+1} = psi_s - c dt (S psi_s + D psi_s) + c dt q(t_s),
 * t_s = t_start + s dt. Before each step the state psi_s is read out:
 * det_series[s*ndet + d] = Re psi_00(det_voxel[d]) and
 * integral[2s], integral[2s+1] = real and imaginary part of sum_r psi_00(r) dx^3.
 * Either output may be NULL.
 */
void orc_run(const orc_medium *p, zc *psi, double dt, int nsteps, double t_start,
             int nsrc, const int *src_voxel, const int *src_moment, const double *src_amp,
             const double *src_t0, const double *src_fwhm,
             int ndet, const int *det_voxel, double *det_series, double *integral) {
    const int N = p->N, M = orc_num_moments(N);
    const size_t V = (size_t)p->nx * p->ny * p->nz;
    const double cdt = p->c * dt;
    const double vol = p->dx * p->dx * p->dx;
    zc *tpsi = (zc *)malloc(sizeof(zc) * V * M);
    for (int s = 0; s < nsteps; ++s) {
        double t = t_start + s * dt;
        if (det_series)
            for (int d = 0; d < ndet; ++d) det_series[(size_t)s * ndet + d] = creal(psi[det_voxel[d]]);
        if (integral) {
            zc acc = 0.0;
            for (size_t v = 0; v < V; ++v) acc += psi[v];
            integral[2 * s] = creal(acc) * vol;
            integral[2 * s + 1] = cimag(acc) * vol;
        }
        orc_apply_T(p, psi, tpsi);
        for (size_t i = 0; i < V * (size_t)M; ++i) psi[i] -= cdt * tpsi[i];
        for (int q = 0; q < nsrc; ++q) {
            double dens = orc_source_density(t, src_amp[q], src_t0[q], src_fwhm[q], p->dx);
            psi[(size_t)src_moment[q] * V + src_voxel[q]] += cdt * dens;
        }
    }
    free(tpsi);
}

/* ------------------------------------------------------------------------ */
/* Steady state: restarted GMRES on T psi = q (Sec. II.A, "Krylov subspace   */
/* iterative methods" applied to the implicit operator)                      */
/* ------------------------------------------------------------------------ */

/* <u, v> = sum_{l,m,r} (2l+1) conj(u) v: the L2 inner product of the radiance
 * over the sphere (Eq. 3 weights each moment by (2l+1)/4pi). */
static zc wdot(int N, size_t V, const zc *u, const zc *v) {
    zc acc = 0.0;
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            size_t j = (size_t)orc_moment_index(l, m);
            zc part = 0.0;
            for (size_t r = 0; r < V; ++r) part += conj(u[j * V + r]) * v[j * V + r];
            acc += (2.0 * l + 1.0) * part;
        }
    return acc;
}

static double wnorm(int N, size_t V, const zc *u) { return sqrt(creal(wdot(N, V, u, u))); }

/*
 * GMRES(restart) from x0 = 0 in the weighted inner product, modified
 * Gram-Schmidt Arnoldi, complex Givens rotations. Stops when the weighted
 * relative residual |q - T x| / |q| <= rtol or after max_iter Arnoldi steps.
 * Returns 0 on convergence, 1 otherwise.
 */
int orc_gmres(const orc_medium *p, const zc *q, zc *x, int restart, int max_iter, double rtol,
              int *iters_out, double *relres_out) {
    const int N = p->N, M = orc_num_moments(N);
    const size_t V = (size_t)p->nx * p->ny * p->nz, n = V * M;
    const int m = restart;
    zc *basis = (zc *)malloc(sizeof(zc) * n * (size_t)(m + 1));
    zc *w = (zc *)malloc(sizeof(zc) * n);
    zc *H = (zc *)calloc((size_t)(m + 1) * m, sizeof(zc));
    zc *gv = (zc *)calloc((size_t)m + 1, sizeof(zc));
    double *cs = (double *)calloc((size_t)m, sizeof(double));
    zc *sn = (zc *)calloc((size_t)m, sizeof(zc));
    zc *y = (zc *)calloc((size_t)m, sizeof(zc));
    double qn = wnorm(N, V, q);
    int iters = 0, converged = 0;
    double rel = 1.0;
    for (size_t i = 0; i < n; ++i) x[i] = 0.0;
    if (qn == 0.0) { rel = 0.0; converged = 1; }
    while (!converged && iters < max_iter) {
        /* r = q - T x */
        apply_T_impl(p, x, w, 0);
        for (size_t i = 0; i < n; ++i) w[i] = q[i] - w[i];
        double beta = wnorm(N, V, w);
        rel = beta / qn;
        if (rel <= rtol) { converged = 1; break; }
        for (size_t i = 0; i < n; ++i) basis[i] = w[i] / beta;
        for (int i = 0; i <= m; ++i) gv[i] = 0.0;
        gv[0] = beta;
        int j;
        for (j = 0; j < m && iters < max_iter; ++j) {
            zc *vj = basis + (size_t)j * n, *vn = basis + (size_t)(j + 1) * n;
            apply_T_impl(p, vj, w, 0);
            for (int i = 0; i <= j; ++i) {
                zc *vi = basis + (size_t)i * n;
                zc h = wdot(N, V, vi, w);
                H[(size_t)i * m + j] = h;
                for (size_t t = 0; t < n; ++t) w[t] -= h * vi[t];
            }
            double hn = wnorm(N, V, w);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (size_t t = 0; t < n; ++t) vn[t] = w[t] / hn;
            /* previous rotations on column j */
            for (int i = 0; i < j; ++i) {
                zc a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -conj(sn[i]) * a + cs[i] * b;
            }
            /* new rotation zeroing H[j+1][j] */
            zc a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            double rho = sqrt(creal(a * conj(a)) + creal(b * conj(b)));
            if (cabs(a) == 0.0) { cs[j] = 0.0; sn[j] = 1.0; }
            else { cs[j] = cabs(a) / rho; sn[j] = a * conj(b) / (cabs(a) * rho); }
            H[(size_t)j * m + j] = cs[j] * a + sn[j] * b;
            H[(size_t)(j + 1) * m + j] = 0.0;
            zc g0 = gv[j];
            gv[j] = cs[j] * g0;
            gv[j + 1] = -conj(sn[j]) * g0;
            ++iters;
            rel = cabs(gv[j + 1]) / qn;
            if (rel <= rtol || hn == 0.0) { ++j; break; }
        }
        /* back substitution H y = g, then x += V y */
        for (int i = j - 1; i >= 0; --i) {
            zc acc = gv[i];
            for (int k = i + 1; k < j; ++k) acc -= H[(size_t)i * m + k] * y[k];
            y[i] = acc / H[(size_t)i * m + i];
        }
        for (int i = 0; i < j; ++i) {
            zc *vi = basis + (size_t)i * n;
            for (size_t t = 0; t < n; ++t) x[t] += y[i] * vi[t];
        }
    }
    if (!converged) {
        apply_T_impl(p, x, w, 0);
        for (size_t i = 0; i < n; ++i) w[i] = q[i] - w[i];
        rel = wnorm(N, V, w) / qn;
        converged = rel <= rtol;
    }
    if (iters_out) *iters_out = iters;
    if (relres_out) *relres_out = rel;
    free(basis); free(w); free(H); free(gv); free(cs); free(sn); free(y);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the explicit scheme                                   */
/* ------------------------------------------------------------------------ */

/*
 * Forward: psi_{n+1} = A psi_n + c dt q_n, A = I - c dt (S + D), n = 0..T-1.
 * Readouts observe the pre-step states psi_n (n = 0..T-1); the loss gradient
 * with respect to them enters as g_n = sum_d weight[n*ndet + d] e_{00, det_voxel[d]},
 * i.e. weight[n][d] = dL/dRe(psi_{n,00}(r_d)).
 * Adjoint: lambda_T = 0, lambda_n = A^H lambda_{n+1} + g_n (n = T-1..1), with
 * A^H = I - c dt (S^H + D) and S^H = F^-1 S(k)^H F.
 * Gradients (inside Omega; zero in the PML where mu_a, mu_s do not enter):
 *   dL/dmu_a(r) = -c dt sum_{n=0}^{T-1} Re sum_{lm} conj(lambda_{n+1}) psi_n
 *   dL/dmu_s(r) = -c dt sum_{n=0}^{T-1} Re sum_{lm} (1 - g^l) conj(lambda_{n+1}) psi_n
 * All T states are kept in memory (tiny grids only).
 */
void orc_adjoint(const orc_medium *p, const unsigned char *pml_mask, const zc *psi0, double dt,
                 int nsteps, double t_start,
                 int nsrc, const int *src_voxel, const int *src_moment, const double *src_amp,
                 const double *src_t0, const double *src_fwhm,
                 int ndet, const int *det_voxel, const double *weight,
                 double *grad_mua, double *grad_mus) {
    const int N = p->N, M = orc_num_moments(N);
    const size_t V = (size_t)p->nx * p->ny * p->nz, n = V * M;
    const double cdt = p->c * dt;
    zc *traj = (zc *)malloc(sizeof(zc) * n * (size_t)nsteps);
    memcpy(traj, psi0, sizeof(zc) * n);
    for (int s = 0; s + 1 < nsteps; ++s) {
        memcpy(traj + (size_t)(s + 1) * n, traj + (size_t)s * n, sizeof(zc) * n);
        orc_run(p, traj + (size_t)(s + 1) * n, dt, 1, t_start + s * dt, nsrc, src_voxel, src_moment,
                src_amp, src_t0, src_fwhm, 0, NULL, NULL, NULL);
    }
    zc *lam = (zc *)calloc(n, sizeof(zc));   /* lambda_{n+1}, starts as lambda_T = 0 */
    zc *tmp = (zc *)malloc(sizeof(zc) * n);
    for (size_t v = 0; v < V; ++v) { grad_mua[v] = 0.0; grad_mus[v] = 0.0; }
    for (int s = nsteps - 1; s >= 0; --s) {
        const zc *ps = traj + (size_t)s * n;
        for (size_t v = 0; v < V; ++v) {
            if (pml_mask && pml_mask[v]) continue;
            double ga = 0.0, gs = 0.0;
            for (int l = 0; l <= N; ++l)
                for (int m = -l; m <= l; ++m) {
                    size_t j = (size_t)orc_moment_index(l, m) * V + v;
                    double pr = creal(conj(lam[j]) * ps[j]);
                    ga += pr;
                    gs += (1.0 - pow(p->g[v], (double)l)) * pr;
                }
            grad_mua[v] -= cdt * ga;
            grad_mus[v] -= cdt * gs;
        }
        if (s == 0) break;
        /* lambda_s = A^H lambda_{s+1} + g_s */
        apply_T_impl(p, lam, tmp, 1);
        for (size_t i = 0; i < n; ++i) lam[i] -= cdt * tmp[i];
        for (int d = 0; d < ndet; ++d) lam[det_voxel[d]] += weight[(size_t)s * ndet + d];
    }
    free(traj); free(lam); free(tmp);
}
