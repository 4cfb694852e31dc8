// rte_host.h -- host-side planning arithmetic of librte: radix plans,
// twiddle and wavenumber tables, the Eq. 6 coupling table, the layer profile
// (Eq. 12) and the stability limit of the explicit step (Sec. II.A).
#pragma once
#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "rte_types.h"

namespace rte {

// Factor n into Stockham passes of radix 8, 4, 2, 3, 5. False if n has
// another prime factor or n < 2.
bool radix_plan(int n, FftPlan *p);

// DFT wavenumber of index i on an axis of n cells of size dx: 2 pi i' / (n dx),
// i' = i (2i < n), 0 (2i == n), i - n (2i > n).
double wavenumber(int i, int n, double dx);

// tw[j] = exp(-2 pi i j / n), j < n, evaluated in double precision.
std::vector<std::complex<double>> twiddles(int n);

// Eq. 6 coefficients alpha_l^m = sqrt((l+m)(l-m)), beta_l^m = sqrt((l+m)(l+m-1)).
double alpha_coef(int l, int m);
double beta_coef(int l, int m);

// The six couplings of every output moment, k-factors left to the kernels.
std::vector<CouplingRow> coupling_rows(int N);

// The same rows for the real-radiance layout, which stores moments m >= 0
// only at index l(l+1)/2 + m. A source with m' < 0 (only the m - 1 = -1
// neighbour of an m = 0 output) is read as (-1)^{m'} conj(psi~_{l', -m'}(-k)):
// its type becomes 3 (mirror of type 1) or 4 (mirror of type 2) and the sign
// goes into the coefficient.
std::vector<CouplingRow> coupling_rows_real(int N);

// Half-cosine layer loss mu_b and mask (1 in the layer), Eq. 12.
void layer_profile(int nx, int ny, int nz, int W, double mu0, double mu1, std::vector<double> &mub,
                   std::vector<uint8_t> &mask);

// Distinct (mu_a, mu_s, g) triples of the folded media: all layer triples,
// and the domain's triples or, beyond max_interior of them, the single
// least-damped one (min mu_a, min mu_s, max g).
std::vector<std::array<double, 3>> media_classes(size_t V, const double *mua_eff, const double *mus_eff,
                                                 const double *g, const uint8_t *mask, size_t max_interior);

// dt* = min over classes and |k| in {k_max j / nk, j = 0..nk} of
// min over eigenvalues lam of -c (S(k) + D) of 2 Re(-lam) / |lam|^2, using
// the block structure of S along z (blocks of fixed m). Returns -1 when an
// eigenvalue solve fails, 0 when some mode grows for every dt.
double stability_from_classes(int N, double c, double kmax,
                              const std::vector<std::array<double, 3>> &classes, int nk);

// Record the text returned by rte_last_error_string() for this thread.
void set_last_error(const std::string &msg);

// Eigenvalues of a small complex upper-Hessenberg matrix (row-major, destroyed).
bool hessenberg_eigenvalues(int n, std::complex<double> *H, std::complex<double> *ev);

}  // namespace rte
