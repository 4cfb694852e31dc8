// rte_host.cpp -- host-side planning arithmetic of librte (see rte_host.h).
#include "rte_host.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <set>

namespace rte {

static const double kPi = 3.14159265358979323846264338327950288;

bool radix_plan(int n, FftPlan *p) {
    if (n < 2) return false;
    p->n = n;
    p->npass = 0;
    int r = n;
    const int order[5] = {8, 4, 2, 3, 5};
    for (int q = 0; q < 5; ++q) {
        while (r % order[q] == 0) {
            if (p->npass >= 12) return false;
            p->radix[p->npass++] = order[q];
            r /= order[q];
        }
    }
    return r == 1;
}

double wavenumber(int i, int n, double dx) {
    int ip;
    if (2 * i < n) ip = i;
    else if (2 * i == n) ip = 0;
    else ip = i - n;
    return 2.0 * kPi * ip / (n * dx);
}

std::vector<std::complex<double>> twiddles(int n) {
    std::vector<std::complex<double>> t(n);
    for (int j = 0; j < n; ++j) {
        const double a = 2.0 * kPi * j / n;
        t[j] = std::complex<double>(std::cos(a), -std::sin(a));
    }
    return t;
}

double alpha_coef(int l, int m) {
    const double p = double(l + m) * double(l - m);
    return p > 0.0 ? std::sqrt(p) : 0.0;
}

double beta_coef(int l, int m) {
    const double p = double(l + m) * double(l + m - 1);
    return p > 0.0 ? std::sqrt(p) : 0.0;
}

static bool has_moment(int N, int l, int m) { return l >= 0 && l <= N && m >= -l && m <= l; }
static int midx(int l, int m) { return l * l + l + m; }

// Output moment (l, m) of the streaming term (Eq. 6 with d/dx_j -> i k_j):
//   1/(2l+1) [ i kz (a_{l+1}^m psi_{l+1}^m + a_l^m psi_{l-1}^m)
//            - 1/2 (i kx + ky)(b_l^m psi_{l-1}^{m-1} - b_{l+1}^{1-m} psi_{l+1}^{m-1})
//            - 1/2 (i kx - ky)(-b_l^{-m} psi_{l-1}^{m+1} + b_{l+1}^{m+1} psi_{l+1}^{m+1}) ]
// The i kz factor is carried by the z-derivative field (type 0).
std::vector<CouplingRow> coupling_rows(int N) {
    const int M = (N + 1) * (N + 1);
    std::vector<CouplingRow> rows(M);
    for (int l = 0; l <= N; ++l)
        for (int m = -l; m <= l; ++m) {
            CouplingRow &r = rows[midx(l, m)];
            r.n = 0;
            const double f = 1.0 / (2.0 * l + 1.0);
            auto add = [&](int ls, int ms, int type, double c) {
                if (!has_moment(N, ls, ms)) return;
                r.src[r.n] = midx(ls, ms);
                r.type[r.n] = type;
                r.coef[r.n] = c;
                ++r.n;
            };
            add(l + 1, m, 0, f * alpha_coef(l + 1, m));
            add(l - 1, m, 0, f * alpha_coef(l, m));
            add(l - 1, m - 1, 1, -0.5 * f * beta_coef(l, m));
            add(l + 1, m - 1, 1, 0.5 * f * beta_coef(l + 1, 1 - m));
            add(l - 1, m + 1, 2, 0.5 * f * beta_coef(l, -m));
            add(l + 1, m + 1, 2, -0.5 * f * beta_coef(l + 1, m + 1));
        }
    return rows;
}

std::vector<CouplingRow> coupling_rows_real(int N) {
    const auto full = coupling_rows(N);
    std::vector<CouplingRow> rows((size_t)(N + 1) * (N + 2) / 2);
    for (int l = 0; l <= N; ++l)
        for (int m = 0; m <= l; ++m) {
            const CouplingRow &f = full[midx(l, m)];
            CouplingRow &r = rows[(size_t)l * (l + 1) / 2 + m];
            r.n = f.n;
            for (int t = 0; t < f.n; ++t) {
                int ls = 0;
                while ((ls + 1) * (ls + 1) <= f.src[t]) ++ls;
                const int ms = f.src[t] - ls * ls - ls;
                if (ms >= 0) {
                    r.src[t] = ls * (ls + 1) / 2 + ms;
                    r.type[t] = f.type[t];
                    r.coef[t] = f.coef[t];
                } else {
                    r.src[t] = ls * (ls + 1) / 2 - ms;
                    r.type[t] = f.type[t] + 2;
                    r.coef[t] = ((-ms) % 2 ? -1.0 : 1.0) * f.coef[t];
                }
            }
        }
    return rows;
}

void layer_profile(int nx, int ny, int nz, int W, double mu0, double mu1, std::vector<double> &mub,
                   std::vector<uint8_t> &mask) {
    const size_t V = (size_t)nx * ny * nz;
    mub.assign(V, 0.0);
    mask.assign(V, 0);
    if (W <= 0) return;
    const int dims[3] = {nx, ny, nz};
    // per-axis profile of each index: depth d of the cell centre into the layer
    std::vector<double> prof[3];
    std::vector<uint8_t> inl[3];
    for (int a = 0; a < 3; ++a) {
        const int n = dims[a];
        prof[a].assign(n, 0.0);
        inl[a].assign(n, 0);
        for (int i = 0; i < n; ++i) {
            double d;
            if (i < W) d = (W - i) - 0.5;
            else if (i >= n - W) d = (i - (n - W)) + 0.5;
            else continue;
            inl[a][i] = 1;
            prof[a][i] = mu0 + (mu1 - mu0) * 0.5 * (1.0 - std::cos(kPi * d / W));
        }
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int idx[3] = {x, y, z};
                bool in = false;
                double best = 0.0;
                for (int a = 0; a < 3; ++a)
                    if (inl[a][idx[a]]) {
                        if (!in || prof[a][idx[a]] > best) best = prof[a][idx[a]];
                        in = true;
                    }
                const size_t v = ((size_t)z * ny + y) * nx + x;
                mub[v] = in ? best : 0.0;
                mask[v] = in ? 1 : 0;
            }
}

std::vector<std::array<double, 3>> media_classes(size_t V, const double *mua, const double *mus, const double *g,
                                                 const uint8_t *mask, size_t max_interior) {
    std::set<std::array<double, 3>> inner, layer;
    bool overflow = false;
    double amin = std::numeric_limits<double>::infinity(), smin = amin, gmax = -amin;
    for (size_t v = 0; v < V; ++v) {
        const std::array<double, 3> t = {mua[v], mus[v], g[v]};
        if (mask[v]) {
            layer.insert(t);
            continue;
        }
        amin = std::min(amin, t[0]);
        smin = std::min(smin, t[1]);
        gmax = std::max(gmax, t[2]);
        if (!overflow) {
            inner.insert(t);
            if (inner.size() > max_interior) overflow = true;
        }
    }
    std::vector<std::array<double, 3>> out;
    if (overflow) out.push_back({amin, smin, gmax});
    else out.assign(inner.begin(), inner.end());
    out.insert(out.end(), layer.begin(), layer.end());
    return out;
}

bool hessenberg_eigenvalues(int n, std::complex<double> *A, std::complex<double> *ev) {
    using cd = std::complex<double>;
    auto H = [&](int i, int j) -> cd & { return A[(size_t)i * n + j]; };
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += std::norm(A[i]);
    fro = std::sqrt(fro);
    if (fro == 0.0) {
        for (int i = 0; i < n; ++i) ev[i] = 0.0;
        return true;
    }
    std::vector<cd> cs(n), sn(n);
    int hi = n - 1, its = 0, total = 0;
    const double eps = std::numeric_limits<double>::epsilon();
    while (hi >= 0) {
        int lo = hi;
        while (lo > 0) {
            double sc = std::abs(H(lo - 1, lo - 1)) + std::abs(H(lo, lo));
            if (sc == 0.0) sc = fro;
            if (std::abs(H(lo, lo - 1)) <= eps * sc) {
                H(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            ev[hi] = H(hi, hi);
            --hi;
            its = 0;
            continue;
        }
        if (++total > 200 * n) return false;
        // Wilkinson shift from the trailing 2x2 block of the active part
        const cd a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
        const cd tr = a + d, det = a * d - b * c;
        const cd disc = std::sqrt(tr * tr * 0.25 - det);
        const cd m1 = tr * 0.5 + disc, m2 = tr * 0.5 - disc;
        cd mu = (std::abs(m1 - d) < std::abs(m2 - d)) ? m1 : m2;
        if (its == 10 || its == 20) mu = d + 0.75 * std::abs(c);   // exceptional shift
        ++its;
        for (int k = lo; k <= hi; ++k) H(k, k) -= mu;
        // H - mu I = Q R with Givens rotations G_k = [[conj c, conj s], [-s, c]]
        for (int k = lo; k < hi; ++k) {
            const cd x = H(k, k), y = H(k + 1, k);
            const double r = std::hypot(std::abs(x), std::abs(y));
            cd ck = 1.0, sk = 0.0;
            if (r > 0.0) {
                ck = x / r;
                sk = y / r;
            }
            cs[k] = ck;
            sn[k] = sk;
            for (int j = k; j <= hi; ++j) {
                const cd u = H(k, j), v = H(k + 1, j);
                H(k, j) = std::conj(ck) * u + std::conj(sk) * v;
                H(k + 1, j) = -sk * u + ck * v;
            }
        }
        // R Q: apply G_k^H = [[c, -conj s], [s, conj c]] on columns k, k+1
        for (int k = lo; k < hi; ++k) {
            const cd ck = cs[k], sk = sn[k];
            const int imax = std::min(k + 2, hi);
            for (int i = lo; i <= imax; ++i) {
                const cd u = H(i, k), v = H(i, k + 1);
                H(i, k) = u * ck + v * sk;
                H(i, k + 1) = -u * std::conj(sk) + v * std::conj(ck);
            }
        }
        for (int k = lo; k <= hi; ++k) H(k, k) += mu;
    }
    return true;
}

double stability_from_classes(int N, double c, double kmax, const std::vector<std::array<double, 3>> &classes,
                              int nk) {
    using cd = std::complex<double>;
    double best = std::numeric_limits<double>::infinity();
    std::vector<cd> H((size_t)(N + 1) * (N + 1)), ev(N + 1);
    std::vector<double> D(N + 1);
    for (const auto &cl : classes) {
        for (int l = 0; l <= N; ++l) D[l] = cl[0] + cl[1] * (1.0 - std::pow(cl[2], (double)l));
        for (int j = 0; j <= nk; ++j) {
            const double k = kmax * j / nk;
            // k along z: S couples (l, m) with (l +- 1, m) only; one block per m >= 0
            // (the block of -m has the same entries).
            for (int m = 0; m <= N; ++m) {
                const int nb = N + 1 - m;
                std::fill(H.begin(), H.begin() + (size_t)nb * nb, cd(0.0));
                for (int i = 0; i < nb; ++i) {
                    const int l = m + i;
                    H[(size_t)i * nb + i] = -c * D[l];
                    if (i + 1 < nb) {
                        const double al = alpha_coef(l + 1, m);
                        H[(size_t)i * nb + i + 1] = -c * cd(0.0, k) * (al / (2.0 * l + 1.0));
                        H[(size_t)(i + 1) * nb + i] = -c * cd(0.0, k) * (al / (2.0 * l + 3.0));
                    }
                }
                if (!hessenberg_eigenvalues(nb, H.data(), ev.data())) return -1.0;
                for (int i = 0; i < nb; ++i) {
                    const double mag = std::abs(ev[i]);
                    if (!(mag > 0.0)) continue;
                    const double re = -ev[i].real();
                    if (re <= 0.0) return 0.0;
                    best = std::min(best, 2.0 * re / (mag * mag));
                }
            }
        }
    }
    return best;
}

}  // namespace rte
