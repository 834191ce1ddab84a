// host_plan.cpp -- FP64 host planning: prolates, kernel tables, geometry, images, tree.
#include "host_plan.h"

#include <chrono>
#ifdef _OPENMP
#include <omp.h>
#include <parallel/algorithm>
#endif

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>
#include <unordered_set>

#include "pdmk.h"

namespace pdmk {

// ------------------------------- quadrature ---------------------------------------
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z); P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1)
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1; p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// nodes and weights mapped to [a, b]
void gl_interval(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
    gauss_legendre(n, x, w);
    for (int i = 0; i < n; ++i) {
        x[i] = 0.5 * (b - a) * x[i] + 0.5 * (a + b);
        w[i] *= 0.5 * (b - a);
    }
}

// ------------------------------- prolates -----------------------------------------
// The prolate psi_0^c is also the lowest eigenfunction of the Sturm-Liouville operator
// -(d/dx)(1-x^2)(d/dx) + c^2 x^2 that commutes with the integral operator of Eq. (2.3).
// In the basis sqrt(n+1/2) P_n (n even) its matrix is symmetric tridiagonal; the
// entries follow from x^2 P_n expanded by the three-term Legendre recurrence.
static void sym_jacobi_lowest(int K, std::vector<double>& A, std::vector<double>& vec, double* lam) {
    // cyclic Jacobi on a dense K x K symmetric matrix (row-major), all eigenpairs
    std::vector<double> Vm(K * K, 0.0);
    for (int i = 0; i < K; ++i) Vm[i * K + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int i = 0; i < K; ++i)
            for (int j = i + 1; j < K; ++j) off += A[i * K + j] * A[i * K + j];
        if (off < 1e-30) break;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) {
                double apq = A[p * K + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[p * K + p], aqq = A[q * K + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < K; ++k) {
                    double akp = A[k * K + p], akq = A[k * K + q];
                    A[k * K + p] = cs * akp - sn * akq;
                    A[k * K + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < K; ++k) {
                    double apk = A[p * K + k], aqk = A[q * K + k];
                    A[p * K + k] = cs * apk - sn * aqk;
                    A[q * K + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < K; ++k) {
                    double vkp = Vm[k * K + p], vkq = Vm[k * K + q];
                    Vm[k * K + p] = cs * vkp - sn * vkq;
                    Vm[k * K + q] = sn * vkp + cs * vkq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < K; ++i)
        if (A[i * K + i] < A[best * K + best]) best = i;
    *lam = A[best * K + best];
    vec.resize(K);
    for (int k = 0; k < K; ++k) vec[k] = Vm[k * K + best];
}

Pswf pswf_make(double c) {
    Pswf p;
    p.c = c;
    int K = int(c) + 30;
    std::vector<double> A(K * K, 0.0);
    double c2 = c * c;
    for (int k = 0; k < K; ++k) {
        double n = 2.0 * k;
        A[k * K + k] = n * (n + 1.0) + c2 * (2.0 * n * (n + 1.0) - 1.0) / ((2.0 * n + 3.0) * (2.0 * n - 1.0));
        if (k + 1 < K) {
            double o = c2 * (n + 1.0) * (n + 2.0) / ((2.0 * n + 3.0) * std::sqrt((2.0 * n + 1.0) * (2.0 * n + 5.0)));
            A[k * K + k + 1] = o;
            A[(k + 1) * K + k] = o;
        }
    }
    double lam;
    sym_jacobi_lowest(K, A, p.beta, &lam);
    // sign: psi(0) > 0
    p.psi0 = p.eval(0.0);
    if (p.psi0 < 0) {
        for (auto& b : p.beta) b = -b;
        p.psi0 = -p.psi0;
    }
    p.psi1 = p.eval(1.0);
    // int_{-1}^{1} sqrt(1/2) P_0 = sqrt(2); only the n = 0 term integrates to non-zero
    p.c0 = p.beta[0] / std::sqrt(2.0);
    return p;
}

double Pswf::eval(double x) const {
    if (std::fabs(x) > 1.0) return 0.0;
    // sum_k beta_k sqrt(2k + 1/2) P_{2k}(x) by the Legendre recurrence
    double p0 = 1.0, p1 = x, s = beta[0] * std::sqrt(0.5);
    int K = int(beta.size());
    for (int n = 2; n <= 2 * (K - 1); ++n) {
        double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
        if ((n & 1) == 0) s += beta[n / 2] * std::sqrt(n + 0.5) * p2;
    }
    return s;
}

double pswf_calibrate(double eps) {
    double lo = 0.5, hi = 200.0;
    for (int it = 0; it < 80; ++it) {
        double mid = 0.5 * (lo + hi);
        Pswf p = pswf_make(mid);
        double r = p.psi1 / p.psi0;
        if (r > eps) lo = mid; else hi = mid;
        if (hi - lo < 1e-12 * hi) break;
    }
    return 0.5 * (lo + hi);
}

// ------------------------------- Chebyshev ----------------------------------------
double Cheb::eval(double x) const {
    double t = (2.0 * x - a - b) / (b - a);
    double b1 = 0, b2 = 0;
    for (int k = int(coef.size()) - 1; k >= 1; --k) {
        double b0 = 2.0 * t * b1 - b2 + coef[k];
        b2 = b1;
        b1 = b0;
    }
    return t * b1 - b2 + coef[0];
}

template <class F>
Cheb cheb_fit(F f, double a, double b, int n, double tol) {
    Cheb ch;
    ch.a = a;
    ch.b = b;
    std::vector<double> fv(n);
    for (int j = 0; j < n; ++j) {
        double t = std::cos(kPi * (j + 0.5) / n);
        fv[j] = f(0.5 * (b - a) * t + 0.5 * (a + b));
    }
    ch.coef.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double s = 0;
        for (int j = 0; j < n; ++j) s += fv[j] * std::cos(kPi * k * (j + 0.5) / n);
        ch.coef[k] = (k == 0 ? 1.0 : 2.0) * s / n;
    }
    int keep = n;
    while (keep > 2 && std::fabs(ch.coef[keep - 1]) < tol) --keep;
    ch.coef.resize(keep);
    return ch;
}

// derivative of a Chebyshev series (d/dx on [a, b])
static Cheb cheb_deriv(const Cheb& f) {
    Cheb d;
    d.a = f.a;
    d.b = f.b;
    int n = int(f.coef.size());
    if (n < 2) {
        d.coef.assign(1, 0.0);
        return d;
    }
    std::vector<double> c(n + 1, 0.0);
    for (int k = n - 1; k >= 1; --k) c[k - 1] = c[k + 1] + 2.0 * k * f.coef[k];
    c[0] *= 0.5;
    c.resize(n - 1);
    double scale = 2.0 / (f.b - f.a);
    for (auto& v : c) v *= scale;
    d.coef = c;
    return d;
}

// ------------------------------- kernel tables ------------------------------------
double KernelTables::what(double x) const {
    double s = 0;
    for (size_t i = 0; i < gl_x.size(); ++i) s += gl_w[i] * gl_psi[i] * std::cos(x * gl_x[i]);
    return s / psi.c0;
}

KernelTables make_kernel_tables(int d, double eps, double fit_tol) {
    KernelTables kt;
    kt.d = d;
    kt.eps = eps;
    kt.psi = pswf_make(pswf_calibrate(eps));
    const Pswf& P = kt.psi;
    gl_interval(240, 0.0, 1.0, kt.gl_x, kt.gl_w);
    kt.gl_psi.resize(kt.gl_x.size());
    for (size_t i = 0; i < kt.gl_x.size(); ++i) kt.gl_psi[i] = P.eval(kt.gl_x[i]);
    double m2 = 0;
    for (size_t i = 0; i < kt.gl_x.size(); ++i) m2 += kt.gl_w[i] * kt.gl_psi[i] * kt.gl_x[i] * kt.gl_x[i];
    kt.mu2 = m2 / P.c0;
    kt.rhat0 = 0.5 * kt.mu2;
    std::vector<double> gx, gw;
    gl_interval(80, 0.0, 1.0, gx, gw);
    if (d == 3) {
        // phi(t) = (1/c0) int_0^t psi ;  A(s) = phi(t)/t = (1/c0) int_0^1 psi(t tau) dtau
        auto Af = [&](double s) {
            double t = std::sqrt(std::max(s, 0.0)), acc = 0;
            for (size_t i = 0; i < gx.size(); ++i) acc += gw[i] * P.eval(t * gx[i]);
            return acc / P.c0;
        };
        auto Bf = [&](double s) { return P.eval(std::sqrt(std::max(s, 0.0))) / P.c0; };
        kt.A = cheb_fit(Af, 0.0, 1.0, 64, fit_tol);
        kt.B = cheb_fit(Bf, 0.0, 1.0, 64, fit_tol);
        kt.self_coef = P.psi0 / (4.0 * kPi * P.c0);  // Eq. (3.16): W_h(0) = psi(0)/(4 pi c0 h)
    } else {
        // 2D radial smoothing density whose transform is hat-w(|k| h): its charge outside
        // radius t is 1 - Q(t) = (1/c0) int_0^{sqrt(1-t^2)} psi(sqrt(t^2 + v^2)) dv
        //                      = sqrt(1 - t^2) S(t^2),  S(s) = (1/c0) int_0^1 psi(sqrt(s + (1-s) tau^2)) dtau,
        // with S smooth; the device evaluates S and multiplies by sqrt(1 - s).
        auto Sf = [&](double s) {
            s = std::min(std::max(s, 0.0), 1.0);
            double acc = 0;
            for (size_t i = 0; i < gx.size(); ++i)
                acc += gw[i] * P.eval(std::sqrt(std::min(s + (1.0 - s) * gx[i] * gx[i], 1.0)));
            return acc / P.c0;
        };
        kt.B = cheb_fit(Sf, 0.0, 1.0, 64, fit_tol);
        const Cheb Sfit = cheb_fit(Sf, 0.0, 1.0, 64, 0.0);
        // W_1(t) = (1/2pi) int_t^1 Q(u)/u du ; R_1(t) = -log t/(2pi) - W_1(t)
        auto Af = [&](double s) {
            double t = std::sqrt(std::max(s, 0.0)), acc = 0;
            for (size_t i = 0; i < gx.size(); ++i) {
                double u = t + (1.0 - t) * gx[i];
                double Qu = 1.0 - std::sqrt(std::max(1.0 - u * u, 0.0)) * Sfit.eval(u * u);
                acc += gw[i] * (1.0 - t) * (u > 0 ? Qu / u : 0.0);
            }
            return acc / (2.0 * kPi);
        };
        kt.A = cheb_fit(Af, 0.0, 1.0, 96, fit_tol);
        kt.self_coef = Af(0.0);
    }
    return kt;
}

double WindowTables::ft(double nu) const {
    double s = 0;
    for (size_t i = 0; i < gl_x.size(); ++i) {
        double t = gl_x[i];
        s += gl_w[i] * F.eval(t * t) * std::cos(kPi * w * nu * t);
    }
    return w * s;
}

WindowTables make_window(int w, double cw, double fit_tol) {
    WindowTables wt;
    wt.w = w;
    wt.cw = cw;
    Pswf P = pswf_make(cw);
    auto Ff = [&](double s) { return P.eval(std::sqrt(std::max(s, 0.0))) / P.psi0; };
    wt.F = cheb_fit(Ff, 0.0, 1.0, 64, fit_tol);
    wt.dF = cheb_deriv(wt.F);
    gl_interval(240, 0.0, 1.0, wt.gl_x, wt.gl_w);
    return wt;
}

double es_window_ft(int w, double beta, double nu, const std::vector<double>& gx,
                    const std::vector<double>& gw) {
    // nodes gx, gw on [0, pi/2]: phi-hat = w int_0^{pi/2} e^{beta (cos th - 1)} cos(pi w nu sin th) cos th dth
    double s = 0;
    for (size_t i = 0; i < gx.size(); ++i) {
        double th = gx[i];
        s += gw[i] * std::exp(beta * (std::cos(th) - 1.0)) * std::cos(kPi * w * nu * std::sin(th)) * std::cos(th);
    }
    return w * s;
}

// ------------------------------- geometry -----------------------------------------
int make_geometry(int d, const double* Lc, double kappa, double c, Geometry* g) {
    if (d != 2 && d != 3) return PDMK_ERR_BAD_ARG;
    if (!(kappa > 0)) return PDMK_ERR_BAD_ARG;
    g->d = d;
    double cols[3][3] = {{0}};  // cols[j][i] = L(i, j)
    double nrm[3] = {0, 0, 0};
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) {
            double v = Lc[i + j * d];
            if (!std::isfinite(v)) return PDMK_ERR_NONFINITE;
            cols[j][i] = v;
            nrm[j] += v * v;
        }
    for (int j = 0; j < d; ++j) nrm[j] = std::sqrt(nrm[j]);
    // permute by decreasing length (stable), Sec. 3.2
    int perm[3] = {0, 1, 2};
    std::stable_sort(perm, perm + d, [&](int a, int b) { return nrm[a] > nrm[b]; });
    for (int i = 0; i < d; ++i) g->perm[i] = perm[i];
    double A[3][3] = {{0}};
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) A[j][i] = cols[perm[j]][i];
    // Gram-Schmidt: orthonormal e_j; R = E^T A upper triangular with positive diagonal
    double E[3][3] = {{0}};
    double prodn = 1;
    for (int j = 0; j < d; ++j) {
        double v[3] = {A[j][0], A[j][1], d == 3 ? A[j][2] : 0.0};
        for (int pass = 0; pass < 2; ++pass)
            for (int k = 0; k < j; ++k) {
                double dot = 0;
                for (int i = 0; i < d; ++i) dot += v[i] * E[k][i];
                for (int i = 0; i < d; ++i) v[i] -= dot * E[k][i];
            }
        double vn = 0;
        for (int i = 0; i < d; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        prodn *= nrm[perm[j]];
        if (!(vn > 1e-14 * nrm[perm[j]])) return PDMK_ERR_SINGULAR_LATTICE;
        for (int i = 0; i < d; ++i) E[j][i] = v[i] / vn;
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0;
            for (int k = 0; k < d; ++k) s += E[i][k] * A[j][k];
            g->R[i * d + j] = (j < i) ? 0.0 : s;
            g->Q[i * d + j] = E[i][j];
        }
    double V = 1;
    for (int i = 0; i < d; ++i) V *= g->R[i * d + i];
    if (!(V > 1e-14 * prodn)) return PDMK_ERR_SINGULAR_LATTICE;
    g->V = V;
    // inverse of the upper-triangular R by back substitution
    for (int j = 0; j < d; ++j)
        for (int i = d - 1; i >= 0; --i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k < d; ++k) s -= g->R[i * d + k] * g->Rinv[k * d + j];
            g->Rinv[i * d + j] = s / g->R[i * d + i];
        }
    for (int j = 0; j < d; ++j) {
        double s = 0;
        for (int i = 0; i < d; ++i) s += g->R[i * d + j] * g->R[i * d + j];
        g->anorm[j] = std::sqrt(s);
    }
    g->Lmin = g->R[0];
    for (int i = 1; i < d; ++i) g->Lmin = std::min(g->Lmin, g->R[i * d + i]);
    g->rc = g->Lmin / kappa;
    // bounding box of the cell (Eq. (3.5)-(3.9)), cover by cubes (Eq. (3.10)), halo (Eq. (3.12))
    for (int i = 0; i < d; ++i) {
        double width = g->R[i * d + i], xminus = 0;
        for (int k = i + 1; k < d; ++k) {
            width += std::fabs(g->R[i * d + k]);
            xminus += std::min(0.0, g->R[i * d + k]);
        }
        int mi = int(std::ceil(width / g->rc - 1e-9));
        if (mi < 1) mi = 1;
        g->m[i] = mi;
        g->nroot[i] = mi + 2;
        g->lo[i] = xminus - g->rc;
        // Eq. (3.15), rounded up to an even length whose prime factors are at most 13 (the
        // transform's fast paths; the added modes lie outside the active ball and carry no
        // weight)
        int M = 2 * int(std::ceil(c * g->anorm[i] / (2.0 * kPi * g->rc) - 1e-9));
        if (M < 2) M = 2;
        auto smooth13 = [](int v) {
            for (int p : {2, 3, 5, 7, 11, 13})
                while (v % p == 0) v /= p;
            return v == 1;
        };
        while (!smooth13(M)) M += 2;
        g->M[i] = M;
    }
    return PDMK_OK;
}

bool make_periodic_root(Geometry* g, double kappa) {
    const int d = g->d;
    const double a = g->R[0];
    if (!(kappa >= 3.0) || std::fabs(kappa - std::nearbyint(kappa)) > 1e-12) return false;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            const double want = i == j ? a : 0.0;
            if (std::fabs(g->R[i * d + j] - want) > 1e-13 * a) return false;
        }
    const int m = int(std::nearbyint(kappa));
    for (int i = 0; i < d; ++i) {
        g->m[i] = m;
        g->nroot[i] = m;
        g->lo[i] = 0.0;
    }
    g->periodic_root = true;
    return true;
}

void table1_defaults(int d, double eps, const Geometry* g, const double* Lc, double* kappa, int* n_s) {
    // paper Table 1 rows: eps = 1e-3, 1e-6, 1e-9, 1e-12
    static const double row_eps[4] = {1e-3, 1e-6, 1e-9, 1e-12};
    static const int ns2[4] = {30, 40, 40, 60};
    static const int ns3[4] = {80, 200, 500, 600};
    static const double k3[3][4] = {{7, 7, 7, 7}, {5, 5, 3, 3}, {1, 1, 1, 1}};
    int row = 0;
    while (row < 3 && eps < row_eps[row] * 0.999) ++row;
    if (d == 2) {
        *kappa = 7.0;
        *n_s = ns2[row];
        return;
    }
    // regime from the oriented diagonal: number of long axes (> 3 x the shortest)
    double diag[3];
    if (g) {
        for (int i = 0; i < 3; ++i) diag[i] = g->R[i * 3 + i];
    } else {
        Geometry tmp;
        make_geometry(3, Lc, 1.0, 1.0, &tmp);
        for (int i = 0; i < 3; ++i) diag[i] = tmp.R[i * 3 + i];
    }
    double mn = std::min(diag[0], std::min(diag[1], diag[2]));
    int nlong = 0;
    for (int i = 0; i < 3; ++i) nlong += (diag[i] > 3.0 * mn);
    int regime = nlong == 0 ? 0 : (nlong == 1 ? 1 : 2);
    *kappa = k3[regime][row];
    *n_s = ns3[row];
}

// ------------------------------- tree ---------------------------------------------
namespace {
struct BoxKey {
    int level;
    int64_t c[3];
    bool operator==(const BoxKey& o) const {
        return level == o.level && c[0] == o.c[0] && c[1] == o.c[1] && c[2] == o.c[2];
    }
};
struct BoxKeyHash {
    size_t operator()(const BoxKey& k) const {
        uint64_t h = 1469598103934665603ULL ^ uint64_t(k.level);
        for (int i = 0; i < 3; ++i) {
            h ^= uint64_t(k.c[i]) + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
            h *= 1099511628211ULL;
        }
        return size_t(h);
    }
};
struct TmpBox {
    int level;
    int64_t c[3];
    int parent;
    int child0;
    int64_t b, e;  // range in the working index array
};

// Splits box bi of `boxes` into its 2^d children: the box's range of the working arrays
// (idx, and tsc, d scaled coordinates per position) is reordered child by child (a stable
// counting sort), the children are appended to `boxes`, and on_child(key, index) is called
// for each.  (pos - lo) / h_L = 2^L tsc exactly: scaling by a power of two commutes with
// rounding.
template <class OnChild>
static void split_box(int d, std::vector<int64_t>& idx, std::vector<double>& tsc, std::vector<TmpBox>& boxes,
                      int bi, std::vector<int>& lab, std::vector<int64_t>& tmp, std::vector<double>& tsct,
                      OnChild on_child) {
    TmpBox B = boxes[bi];
    const int L = B.level + 1;
    const double s2 = double(1LL << L);
    const int nc = 1 << d;
    int64_t cnt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    auto child_of = [&](int64_t j) {  // working position j
        int ch = 0;
        for (int i = 0; i < d; ++i) {
            const int64_t ci = int64_t(std::floor(tsc[j * d + i] * s2));
            int bit = int(ci - B.c[i] * 2);
            if (bit < 0) bit = 0;
            if (bit > 1) bit = 1;
            ch |= bit << i;
        }
        return ch;
    };
    const int64_t m = B.e - B.b;
    lab.resize(size_t(m));
    tmp.resize(size_t(m));
    tsct.resize(size_t(m) * d);
    for (int64_t j = B.b; j < B.e; ++j) {
        lab[j - B.b] = child_of(j);
        cnt[lab[j - B.b] + 1]++;
    }
    for (int k = 0; k < nc; ++k) cnt[k + 1] += cnt[k];
    int64_t cur[8];
    for (int k = 0; k < nc; ++k) cur[k] = cnt[k];
    for (int64_t j = B.b; j < B.e; ++j) {
        const int64_t o = cur[lab[j - B.b]]++;
        tmp[o] = idx[j];
        for (int i = 0; i < d; ++i) tsct[size_t(o) * d + i] = tsc[size_t(j) * d + i];
    }
    std::copy(tmp.begin(), tmp.begin() + m, idx.begin() + B.b);
    std::copy(tsct.begin(), tsct.begin() + m * d, tsc.begin() + B.b * d);
    const int first = int(boxes.size());
    boxes[bi].child0 = first;
    for (int k = 0; k < nc; ++k) {
        TmpBox C;
        C.level = L;
        C.c[0] = C.c[1] = C.c[2] = 0;
        for (int i = 0; i < d; ++i) C.c[i] = B.c[i] * 2 + ((k >> i) & 1);
        C.parent = bi;
        C.child0 = -1;
        C.b = B.b + cnt[k];
        C.e = B.b + cnt[k + 1];
        boxes.push_back(C);
        on_child(BoxKey{L, {C.c[0], C.c[1], C.c[2]}}, first + k);
    }
}

struct Builder {
    int d;
    const Geometry* g;
    std::vector<double> pos;  // d per image
    std::vector<double> tsc;  // d per working position: (pos - lo) / r_c of image idx[j];
                              // (pos - lo) / h_L = 2^L tsc exactly
    std::vector<double> tsct; // split scratch
    std::vector<int64_t> idx; // working permutation of images
    std::vector<int> lab;     // split scratch
    std::vector<int> split_log;  // boxes split since the log was last cleared
    std::vector<int64_t> tmp;
    std::vector<TmpBox> boxes;
    std::unordered_map<BoxKey, int, BoxKeyHash> map;
    int max_level = 0;
    int nchild() const { return 1 << d; }

    int64_t dim_at(int i, int level) const { return int64_t(g->nroot[i]) << level; }

    int find(int level, const int64_t* c) const {
        BoxKey k{level, {c[0], d > 1 ? c[1] : 0, d > 2 ? c[2] : 0}};
        auto it = map.find(k);
        return it == map.end() ? -1 : it->second;
    }

    void split(int bi) {
        split_box(d, idx, tsc, boxes, bi, lab, tmp, tsct, [&](const BoxKey& k, int id) { map[k] = id; });
        split_log.push_back(bi);
        max_level = std::max(max_level, boxes[bi].level + 1);
    }

    // make the box at (level, c) exist and have children
    void ensure_nonleaf(int level, const int64_t* c) {
        int lv = level;
        int a = -1;
        int64_t cc[3] = {0, 0, 0};
        for (; lv >= 0; --lv) {
            for (int i = 0; i < d; ++i) cc[i] = c[i] >> (level - lv);
            a = find(lv, cc);
            if (a >= 0) break;
        }
        while (boxes[a].level < level) {
            if (boxes[a].child0 < 0) split(a);
            int L = boxes[a].level + 1;
            int k = 0;
            for (int i = 0; i < d; ++i) k |= int((c[i] >> (level - L)) & 1) << i;
            a = boxes[a].child0 + k;
        }
        if (boxes[a].child0 < 0) split(a);
    }
};

// One root box's subtree, refined independently of the others (the splits of a root box only
// permute its own range of the working arrays): its boxes (local index 0 = the root), and
// the keys to enter in the builder's map once the subtrees are merged.
struct LocalTree {
    std::vector<TmpBox> boxes;
    std::vector<std::pair<BoxKey, int>> keys;
    std::vector<int> lab;
    std::vector<int64_t> tmp;
    std::vector<double> tsct;
    int max_level = 0;
};

// Builder::split for a box of a local subtree (the same split_box)
static void split_local(Builder& bld, LocalTree& lt, int bi) {
    split_box(bld.d, bld.idx, bld.tsc, lt.boxes, bi, lt.lab, lt.tmp, lt.tsct,
              [&](const BoxKey& k, int id) { lt.keys.push_back({k, id}); });
    lt.max_level = std::max(lt.max_level, lt.boxes[bi].level + 1);
}
}  // namespace

void image_shifts(const Geometry& g, ImageShifts* out) {
    const int d = g.d;
    // the originals first (shift 0), then every other admissible shift
    std::vector<std::vector<int>> shifts;
    shifts.push_back(std::vector<int>(d, 0));
    std::vector<int> nvec(d, 0);
    // nested loops with n_d outermost (Eq. (3.13))
    auto nmax_at = [&](int i) {
        double off = 0;
        for (int k = i + 1; k < d; ++k) off += g.R[i * d + k] * nvec[k];
        return int(std::ceil(((g.m[i] + 1) * g.rc + std::fabs(off)) / g.R[i * d + i]));
    };
    std::function<void(int)> rec = [&](int lev) {
        int b = nmax_at(lev);
        for (int v = -b; v <= b; ++v) {
            nvec[lev] = v;
            if (lev == 0) {
                bool zero = true;
                for (int k = 0; k < d; ++k) zero &= (nvec[k] == 0);
                if (!zero) shifts.push_back(nvec);
            } else {
                rec(lev - 1);
            }
        }
        nvec[lev] = 0;
    };
    if (!g.periodic_root) rec(d - 1);  // a periodic root holds the originals only
    const int ns = int(shifts.size());
    out->ns = ns;
    for (int a = 0; a < 3; ++a) {
        out->Bx[a] = 0;
        out->dimx[a] = 1;
    }
    for (const auto& sh : shifts)
        for (int a = 0; a < d; ++a) out->Bx[a] = std::max(out->Bx[a], std::abs(sh[a]));
    int64_t ntab = 1;
    for (int a = 0; a < d; ++a) {
        out->dimx[a] = 2 * out->Bx[a] + 1;
        ntab *= out->dimx[a];
    }
    auto flat = [&](const int* nv) {
        int64_t f = 0;
        for (int a = d - 1; a >= 0; --a) f = f * out->dimx[a] + (nv[a] + out->Bx[a]);
        return f;
    };
    out->sidx.assign(static_cast<size_t>(ntab), -1);
    out->trs.assign(size_t(ns) * 3, 0.0);
    for (int k = 0; k < ns; ++k) {
        out->sidx[size_t(flat(shifts[k].data()))] = k;
        for (int a = 0; a < d; ++a)
            for (int kk = a; kk < d; ++kk) out->trs[size_t(k) * 3 + a] += g.R[a * d + kk] * shifts[k][kk];
    }
}

int build_tree(const Geometry& g, int64_t n, const double* u, int n_s, int max_depth, Tree* t,
               SortedSources* s, BuildStats* st) {
    const int d = g.d;
    Builder bld;
    bld.d = d;
    bld.g = &g;
    auto clk = std::chrono::steady_clock::now();
    auto lap = [&](int k) {
        const auto now = std::chrono::steady_clock::now();
        if (st) st->phase_ms[k] = std::chrono::duration<double, std::milli>(now - clk).count();
        clk = now;
    };
    // ---- images (Sec. 3.4): shifts within the bounds of Eq. (3.13), in-box test ----
    std::vector<int64_t> img_orig;
    double hi[3];
    for (int i = 0; i < d; ++i) hi[i] = g.lo[i] + g.nroot[i] * g.rc;
    std::vector<double> x(n * d);
    for (int64_t j = 0; j < n; ++j)
        for (int i = 0; i < d; ++i) {
            double v = 0;
            for (int k = i; k < d; ++k) v += g.R[i * d + k] * u[j * d + k];
            x[j * d + i] = v;
        }
    // Images in shift order, and within a shift in point order.  Each point's admissible
    // shifts are enumerated from the in-box bounds of the triangular frame (axis by axis from
    // the last, with a small slack against rounding) and then accepted by the same test with
    // the same arithmetic as a scan of every listed shift; listed shifts only.
    ImageShifts tab;
    image_shifts(g, &tab);
    const int ns = tab.ns;
    const int* Bx = tab.Bx;
    const int64_t* dimx = tab.dimx;
    auto flat = [&](const int* nv) {
        int64_t f = 0;
        for (int a = d - 1; a >= 0; --a) f = f * dimx[a] + (nv[a] + Bx[a]);
        return f;
    };
    const std::vector<int>& sidx = tab.sidx;
    const std::vector<double>& trs = tab.trs;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    const int64_t chunk = (n + nthr - 1) / std::max(nthr, 1);
    std::vector<std::vector<std::pair<int, int64_t>>> acc(static_cast<size_t>(nthr));
    bool missing = false;
#pragma omp parallel for schedule(static, 1) reduction(|| : missing)
    for (int c = 0; c < nthr; ++c) {
        auto& out = acc[size_t(c)];
        for (int64_t j = c * chunk; j < std::min(n, (c + 1) * chunk); ++j) {
            const double* xj = &x[size_t(j) * d];
            auto accept = [&](int k) {
                bool in = true;
                for (int a = 0; a < d; ++a) {
                    const double p = xj[a] + trs[size_t(k) * 3 + a];
                    in &= (p >= g.lo[a] && p < hi[a]);
                }
                return in;
            };
            if (!accept(0)) { missing = true; continue; }  // the cell lies inside the inner block
            // nested intervals, axis by axis from the last: the bounds carry a slack of 1e-9
            // (far above their rounding) and every candidate then takes the exact test
            auto range = [&](int a, const int* nv, int* lo_n, int* hi_n) {
                double off = 0;
                for (int k = a + 1; k < d; ++k) off += g.R[a * d + k] * nv[k];
                const double raa = g.R[a * d + a];
                const double l = (g.lo[a] - xj[a] - off) / raa, h = (hi[a] - xj[a] - off) / raa;
                const double sl = 1e-9 * (1.0 + std::fabs(l)), sh = 1e-9 * (1.0 + std::fabs(h));
                *lo_n = std::max(-Bx[a], int(std::ceil(l - sl)));
                *hi_n = std::min(Bx[a], int(std::floor(h + sh)));
            };
            int nv[3] = {0, 0, 0};
            int l2 = 0, h2 = 0, l1 = 0, h1 = 0, l0 = 0, h0 = 0;
            if (d == 3) range(2, nv, &l2, &h2);
            for (int v2 = l2; v2 <= h2; ++v2) {
                nv[2] = d == 3 ? v2 : 0;
                range(1, nv, &l1, &h1);
                for (int v1 = l1; v1 <= h1; ++v1) {
                    nv[1] = v1;
                    range(0, nv, &l0, &h0);
                    for (int v0 = l0; v0 <= h0; ++v0) {
                        nv[0] = v0;
                        const int k = sidx[size_t(flat(nv))];
                        if (k > 0 && accept(k)) out.push_back({k, j});
                    }
                }
            }
        }
    }
    if (missing) return PDMK_ERR_INTERNAL;
    // offsets: shift 0 holds the originals in point order; then shift by shift, thread
    // chunks in order (points in increasing order within each)
    std::vector<int64_t> cnt(size_t(ns) * nthr, 0);
    for (int c = 0; c < nthr; ++c)
        for (const auto& pr : acc[size_t(c)]) cnt[size_t(pr.first) * nthr + c]++;
    std::vector<int64_t> off(size_t(ns) * nthr, 0);
    int64_t run = n;
    for (int k = 1; k < ns; ++k)
        for (int c = 0; c < nthr; ++c) {
            off[size_t(k) * nthr + c] = run;
            run += cnt[size_t(k) * nthr + c];
        }
    img_orig.resize(size_t(run));
    bld.pos.resize(size_t(run) * d);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        img_orig[size_t(j)] = j;
        for (int a = 0; a < d; ++a) bld.pos[size_t(j) * d + a] = x[size_t(j) * d + a] + trs[a];
    }
#pragma omp parallel for schedule(static, 1)
    for (int c = 0; c < nthr; ++c) {
        std::vector<int64_t> o(static_cast<size_t>(ns));
        for (int k = 1; k < ns; ++k) o[size_t(k)] = off[size_t(k) * nthr + c];
        for (const auto& pr : acc[size_t(c)]) {
            const int64_t w = o[size_t(pr.first)]++;
            img_orig[size_t(w)] = -(pr.second + 1);
            for (int a = 0; a < d; ++a)
                bld.pos[size_t(w) * d + a] = x[size_t(pr.second) * d + a] + trs[size_t(pr.first) * 3 + a];
        }
    }
    const int64_t nimg = int64_t(img_orig.size());
    bld.tsc.resize(size_t(nimg) * d);
    // position in root-box units, (p - lo) times 1 / r_c (the device build does the same two
    // rounded steps, so both builds put every point in the same box)
    const double inv_rc = 1.0 / g.rc;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nimg; ++j)
        for (int a = 0; a < d; ++a) bld.tsc[size_t(j) * d + a] = (bld.pos[size_t(j) * d + a] - g.lo[a]) * inv_rc;
    bld.map.reserve(size_t(std::max<int64_t>(1024, 4 * nimg / std::max(n_s, 1))));
    lap(0);
    // ---- root boxes: counting sort by root cell ----
    int64_t nroot_tot = 1;
    for (int a = 0; a < d; ++a) nroot_tot *= g.nroot[a];
    std::vector<int64_t> rcell(nimg), rcnt(nroot_tot + 1, 0);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nimg; ++j) {
        int64_t cell = 0;
        for (int a = d - 1; a >= 0; --a) {
            int64_t ci = int64_t(std::floor(bld.tsc[j * d + a]));
            ci = std::min<int64_t>(std::max<int64_t>(ci, 0), g.nroot[a] - 1);
            cell = cell * g.nroot[a] + ci;
        }
        rcell[j] = cell;
    }
    for (int64_t j = 0; j < nimg; ++j) rcnt[rcell[j] + 1]++;
    for (int64_t k = 0; k < nroot_tot; ++k) rcnt[k + 1] += rcnt[k];
    bld.idx.resize(nimg);
    {
        // stable counting sort, in parallel: thread chunks of images in order
        int nt = 1;
#ifdef _OPENMP
        nt = omp_get_max_threads();
#endif
        const int64_t ch = (nimg + nt - 1) / std::max(nt, 1);
        std::vector<int64_t> tc(size_t(nt) * size_t(nroot_tot), 0);
#pragma omp parallel for schedule(static, 1)
        for (int c = 0; c < nt; ++c)
            for (int64_t j = c * ch; j < std::min(nimg, (c + 1) * ch); ++j) tc[size_t(c) * nroot_tot + rcell[j]]++;
        for (int64_t cell = 0; cell < nroot_tot; ++cell) {
            int64_t o = rcnt[cell];
            for (int c = 0; c < nt; ++c) {
                const int64_t v = tc[size_t(c) * nroot_tot + cell];
                tc[size_t(c) * nroot_tot + cell] = o;
                o += v;
            }
        }
#pragma omp parallel for schedule(static, 1)
        for (int c = 0; c < nt; ++c)
            for (int64_t j = c * ch; j < std::min(nimg, (c + 1) * ch); ++j) bld.idx[tc[size_t(c) * nroot_tot + rcell[j]]++] = j;
        std::vector<double> tw(size_t(nimg) * d);
        for (int64_t k = 0; k < nimg; ++k)
            for (int a = 0; a < d; ++a) tw[size_t(k) * d + a] = bld.tsc[size_t(bld.idx[k]) * d + a];
        bld.tsc.swap(tw);
    }
    for (int64_t cell = 0; cell < nroot_tot; ++cell) {
        TmpBox B;
        B.level = 0;
        int64_t r = cell;
        B.c[0] = B.c[1] = B.c[2] = 0;
        for (int a = 0; a < d; ++a) {
            B.c[a] = r % g.nroot[a];
            r /= g.nroot[a];
        }
        B.parent = -1;
        B.child0 = -1;
        B.b = rcnt[cell];
        B.e = rcnt[cell + 1];
        bld.boxes.push_back(B);
        bld.map[BoxKey{0, {B.c[0], B.c[1], B.c[2]}}] = int(cell);
    }
    lap(1);
    // ---- refine boxes holding more than n_s sources (Algorithm 1, step 2) ----
    // Root boxes refine independently (in parallel); their subtrees are then appended in
    // root order.  Box numbering here does not matter: the tree is renumbered canonically
    // (level order, children in order) below.
    {
        std::vector<LocalTree> locals(static_cast<size_t>(nroot_tot));
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r = 0; r < nroot_tot; ++r) {
            LocalTree& lt = locals[size_t(r)];
            lt.boxes.push_back(bld.boxes[size_t(r)]);
            for (size_t bi = 0; bi < lt.boxes.size(); ++bi)
                if (lt.boxes[bi].e - lt.boxes[bi].b > n_s && lt.boxes[bi].level < max_depth)
                    split_local(bld, lt, int(bi));
        }
        for (int64_t r = 0; r < nroot_tot; ++r) {
            LocalTree& lt = locals[size_t(r)];
            const int base = int(bld.boxes.size());
            auto gid = [&](int l) { return l == 0 ? int(r) : base + l - 1; };
            bld.boxes[size_t(r)].child0 = lt.boxes[0].child0 < 0 ? -1 : gid(lt.boxes[0].child0);
            for (size_t l = 1; l < lt.boxes.size(); ++l) {
                TmpBox B = lt.boxes[l];
                B.parent = gid(B.parent);
                B.child0 = B.child0 < 0 ? -1 : gid(B.child0);
                bld.boxes.push_back(B);
            }
            for (const auto& kv : lt.keys) bld.map[kv.first] = gid(kv.second);
            bld.max_level = std::max(bld.max_level, lt.max_level);
            LocalTree().boxes.swap(lt.boxes);
        }
    }
    lap(2);
    // ---- level restriction: every colleague of the parent of a non-leaf box is non-leaf.
    // This keeps the leaves that meet a leaf's colleague neighbourhood within one level of it.
    // The rule's closure is unique and the renumbering below is canonical, so only boxes that
    // became non-leaf since the last sweep need checking: all of them first, then the log.
    std::vector<int> work;
    for (size_t bi = 0; bi < bld.boxes.size(); ++bi) work.push_back(int(bi));
    struct Need {
        int level;
        int64_t c[3];
    };
    int nthb = 1;
#ifdef _OPENMP
    nthb = omp_get_max_threads();
#endif
    std::vector<std::vector<Need>> need(static_cast<size_t>(nthb));
    while (!work.empty()) {
        bld.split_log.clear();
        // find the violations in parallel (read-only), then repair them in order
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            auto& mine = need[size_t(tid)];
            mine.clear();
#pragma omp for schedule(dynamic, 256)
            for (int64_t w = 0; w < int64_t(work.size()); ++w) {
                const TmpBox& Y = bld.boxes[size_t(work[size_t(w)])];
                if (Y.level < 1 || Y.child0 < 0) continue;
                const TmpBox& P = bld.boxes[size_t(Y.parent)];
                int nn = 1;
                for (int a = 0; a < d; ++a) nn *= 3;
                for (int o = 0; o < nn; ++o) {
                    int64_t c[3] = {0, 0, 0};
                    int r = o;
                    bool ok = true;
                    for (int a = 0; a < d; ++a) {
                        c[a] = P.c[a] + (r % 3) - 1;
                        r /= 3;
                        const int64_t dim = bld.dim_at(a, P.level);
                        if (g.periodic_root) c[a] = (c[a] + dim) % dim;  // neighbours across the faces
                        ok &= (c[a] >= 0 && c[a] < dim);
                    }
                    if (!ok) continue;
                    int X = bld.find(P.level, c);
                    if (X >= 0 && bld.boxes[size_t(X)].child0 >= 0) continue;
                    mine.push_back(Need{P.level, {c[0], c[1], c[2]}});
                }
            }
        }
        for (const auto& list : need)
            for (const Need& nd : list) {
                int X = bld.find(nd.level, nd.c);
                if (X >= 0 && bld.boxes[size_t(X)].child0 >= 0) continue;
                bld.ensure_nonleaf(nd.level, nd.c);
            }
        work.swap(bld.split_log);
    }
    lap(3);
    // ---- renumber in level order (children of consecutive parents stay contiguous) ----
    const int nbtot = int(bld.boxes.size());
    std::vector<int> order;
    order.reserve(nbtot);
    for (int k = 0; k < int(nroot_tot); ++k) order.push_back(k);
    std::vector<int> newid(nbtot, -1);
    std::vector<int> lstart;
    lstart.push_back(0);
    size_t head = 0;
    int curlev = 0;
    while (head < order.size()) {
        size_t end = order.size();
        for (size_t k = head; k < end; ++k) {
            int b = order[k];
            if (bld.boxes[b].child0 >= 0)
                for (int c = 0; c < bld.nchild(); ++c) order.push_back(bld.boxes[b].child0 + c);
        }
        head = end;
        lstart.push_back(int(end));
        ++curlev;
        if (order.size() == end) break;
    }
    for (int k = 0; k < nbtot; ++k) newid[order[k]] = k;
    t->d = d;
    for (int a = 0; a < 3; ++a) t->nroot[a] = a < d ? g.nroot[a] : 1;
    t->periodic = g.periodic_root;
    t->nlevels = int(lstart.size()) - 1;
    t->level_start = lstart;
    t->level.resize(nbtot);
    t->coord.assign(size_t(nbtot) * d, 0);
    t->parent.resize(nbtot);
    t->child0.resize(nbtot);
    t->src_begin.resize(nbtot);
    t->src_end.resize(nbtot);
    t->center.resize(size_t(nbtot) * d);
    for (int k = 0; k < nbtot; ++k) {
        const TmpBox& B = bld.boxes[order[k]];
        t->level[k] = B.level;
        for (int a = 0; a < d; ++a) {
            t->coord[size_t(k) * d + a] = B.c[a];
            double h = g.rc / double(1LL << B.level);
            t->center[size_t(k) * d + a] = g.lo[a] + (double(B.c[a]) + 0.5) * h;
        }
        t->parent[k] = B.parent < 0 ? -1 : newid[B.parent];
        t->child0[k] = B.child0 < 0 ? -1 : newid[B.child0];
        t->src_begin[k] = B.b;
        t->src_end[k] = B.e;
    }
    // colleagues
    int nn = 1;
    for (int a = 0; a < d; ++a) nn *= 3;
    t->colleague.assign(size_t(nbtot) * nn, -1);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nbtot; ++k) {
        const TmpBox& B = bld.boxes[order[k]];
        for (int o = 0; o < nn; ++o) {
            int64_t c[3] = {0, 0, 0};
            int r = o;
            bool ok = true;
            for (int a = 0; a < d; ++a) {
                c[a] = B.c[a] + (r % 3) - 1;
                r /= 3;
                const int64_t dim = bld.dim_at(a, B.level);
                if (g.periodic_root) c[a] = (c[a] + dim) % dim;
                ok &= (c[a] >= 0 && c[a] < dim);
            }
            if (!ok) continue;
            int X = bld.find(B.level, c);
            t->colleague[size_t(k) * nn + o] = X < 0 ? -1 : newid[X];
        }
    }
    lap(4);
    // ---- sorted sources and targets (the originals, in sorted order) ----
    s->orig.resize(nimg);
    s->pos.resize(size_t(nimg) * d);
    std::vector<int64_t> is_tgt_prefix(nimg + 1, 0);
    s->tgt_of.clear();
    s->tgt_orig.clear();
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nimg; ++j) {
        int64_t im = bld.idx[j];
        int64_t o = img_orig[im];
        s->orig[j] = o >= 0 ? o : -(o + 1);
        for (int a = 0; a < d; ++a) s->pos[size_t(j) * d + a] = bld.pos[size_t(im) * d + a];
    }
    for (int64_t j = 0; j < nimg; ++j) is_tgt_prefix[j + 1] = is_tgt_prefix[j] + (img_orig[bld.idx[j]] >= 0 ? 1 : 0);
    s->tgt_of.resize(size_t(is_tgt_prefix[nimg]));
    s->tgt_orig.resize(size_t(is_tgt_prefix[nimg]));
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nimg; ++j) {
        const int64_t o = img_orig[bld.idx[j]];
        if (o >= 0) {
            s->tgt_of[is_tgt_prefix[j]] = j;
            s->tgt_orig[is_tgt_prefix[j]] = o;
        }
    }
    t->tgt_begin.resize(nbtot);
    t->tgt_end.resize(nbtot);
    for (int k = 0; k < nbtot; ++k) {
        t->tgt_begin[k] = is_tgt_prefix[t->src_begin[k]];
        t->tgt_end[k] = is_tgt_prefix[t->src_end[k]];
    }
    lap(5);
    if (st) {
        st->n = n;
        st->n_images = nimg;
        st->nboxes = nbtot;
        int nl = 0;
        for (int k = 0; k < nbtot; ++k) nl += t->child0[k] < 0;
        st->nleaves = nl;
        st->depth = t->nlevels - 1;
    }
    return PDMK_OK;
}

void box_direct_list(const Tree& t, int b, std::vector<int>* out, std::vector<int>* shift) {
    const int d = t.d;
    int nn = 1;
    for (int a = 0; a < d; ++a) nn *= 3;
    thread_local std::vector<std::pair<int, int>> lst;  // (leaf, shift code), reused per thread
    lst.clear();
    auto add_leaves_below = [&](int x, int code, auto&& self) -> void {
        if (t.is_leaf(x)) {
            if (t.src_end[x] > t.src_begin[x]) lst.push_back({x, code});
            return;
        }
        for (int c = 0; c < (1 << d); ++c) self(t.child0[x] + c, code, self);
    };
    for (int o = 0; o < nn; ++o) {
        int64_t c[3] = {0, 0, 0};
        int r = o;
        for (int a = 0; a < d; ++a) {
            c[a] = t.coord[size_t(b) * d + a] + (r % 3) - 1;
            r /= 3;
        }
        const int code = t.wrap(t.level[b], c);
        int X = t.colleague[size_t(b) * nn + o];
        if (X >= 0) {
            add_leaves_below(X, code, add_leaves_below);
            continue;
        }
        // no same-level box here: the region is covered by a coarser leaf.  With the level
        // restriction that leaf is one level up, a colleague of b's parent (the colleague at
        // the parent-level cell of c, a leaf whenever it exists); the root level searches
        int found = -1;
        const int pb = t.level[b] > 0 ? t.parent[b] : -1;
        if (pb >= 0) {
            int oi = 0, mul = 1;
            for (int a = 0; a < d; ++a) {
                const int64_t cc = t.coord[size_t(b) * d + a] + ((o / mul) % 3) - 1;  // unwrapped cell
                oi += int((cc >> 1) - t.coord[size_t(pb) * d + a] + 1) * mul;
                mul *= 3;
            }
            found = t.colleague[size_t(pb) * nn + oi];
        } else {
            found = t.locate(t.level[b], c);
        }
        if (found >= 0 && !t.is_leaf(found)) found = -1;
        if (found >= 0 && t.src_end[found] > t.src_begin[found]) lst.push_back({found, code});
    }
    std::sort(lst.begin(), lst.end());
    lst.erase(std::unique(lst.begin(), lst.end()), lst.end());
    out->resize(lst.size());
    if (shift) shift->resize(lst.size());
    for (size_t k = 0; k < lst.size(); ++k) {
        (*out)[k] = lst[k].first;
        if (shift) (*shift)[k] = lst[k].second;
    }
}

void sort_pairs_parallel(std::vector<std::pair<int64_t, int64_t>>* v) {
#ifdef _OPENMP
    __gnu_parallel::sort(v->begin(), v->end());
#else
    std::sort(v->begin(), v->end());
#endif
}

void build_direct_lists(const Tree& t, DirectLists* dl, int64_t* pairs) {
    dl->tleaf.clear();
    dl->list_begin.assign(1, 0);
    dl->list.clear();
    dl->shift.clear();
    for (int b = 0; b < int(t.level.size()); ++b)
        if (t.is_leaf(b) && t.tgt_end[b] > t.tgt_begin[b]) dl->tleaf.push_back(b);
    // each thread builds the lists of a contiguous range of target leaves into its own flat
    // buffers (in leaf order); the buffers are then concatenated in thread order
    const int64_t nl = int64_t(dl->tleaf.size());
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    std::vector<std::vector<int>> tlist(static_cast<size_t>(nthr)), tshift(static_cast<size_t>(nthr));
    std::vector<int64_t> count(static_cast<size_t>(nl) + 1, 0);
    std::vector<int64_t> tpairs(static_cast<size_t>(nthr), 0);
#pragma omp parallel num_threads(nthr)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const int64_t k0 = nl * tid / nthr, k1 = nl * (tid + 1) / nthr;
        std::vector<int> lst, sh;
        std::vector<int>& tl = tlist[size_t(tid)];
        std::vector<int>& ts = tshift[size_t(tid)];
        tl.reserve(size_t(k1 - k0) * 32);
        ts.reserve(size_t(k1 - k0) * 32);
        int64_t np = 0;
        for (int64_t k = k0; k < k1; ++k) {
            const int b = dl->tleaf[size_t(k)];
            box_direct_list(t, b, &lst, &sh);
            int64_t nsrc = 0;
            for (int x : lst) nsrc += t.src_end[x] - t.src_begin[x];
            np += nsrc * (t.tgt_end[b] - t.tgt_begin[b]);
            count[size_t(k) + 1] = int64_t(lst.size());
            tl.insert(tl.end(), lst.begin(), lst.end());
            ts.insert(ts.end(), sh.begin(), sh.end());
        }
        tpairs[size_t(tid)] = np;
    }
    dl->list_begin.resize(size_t(nl) + 1);
    for (int64_t k = 0; k < nl; ++k) dl->list_begin[size_t(k) + 1] = dl->list_begin[size_t(k)] + count[size_t(k) + 1];
    dl->list.resize(size_t(dl->list_begin[size_t(nl)]));
    dl->shift.resize(dl->list.size());
    int64_t np = 0;
    for (int c = 0; c < nthr; ++c) np += tpairs[size_t(c)];
#pragma omp parallel for schedule(static, 1) num_threads(nthr)
    for (int c = 0; c < nthr; ++c) {
        const int64_t base = dl->list_begin[size_t(nl * c / nthr)];
        std::copy(tlist[size_t(c)].begin(), tlist[size_t(c)].end(), dl->list.begin() + base);
        std::copy(tshift[size_t(c)].begin(), tshift[size_t(c)].end(), dl->shift.begin() + base);
    }
    if (pairs) *pairs = np;
}

}  // namespace pdmk

namespace pdmk {
int Tree::wrap(int L, int64_t* c) const {
    if (!periodic) return 13;
    int code = 0, mul = 1;
    for (int a = 0; a < d; ++a) {
        const int64_t dim = nroot[a] << L;
        int n = 0;
        while (c[a] < 0) { c[a] += dim; --n; }
        while (c[a] >= dim) { c[a] -= dim; ++n; }
        code += (n + 1) * mul;
        mul *= 3;
    }
    for (int a = d; a < 3; ++a) { code += mul; mul *= 3; }
    return code;
}

int Tree::locate(int L, const int64_t* cin) const {
    int64_t c[3] = {cin[0], d > 1 ? cin[1] : 0, d > 2 ? cin[2] : 0};
    wrap(L, c);
    int64_t root = 0;
    for (int a = d - 1; a >= 0; --a) {
        int64_t ca = c[a] >> L;
        if (c[a] < 0 || ca >= nroot[a]) return -1;
        root = root * nroot[a] + ca;
    }
    int cur = int(root);
    while (!is_leaf(cur) && level[cur] < L) {
        int Lc = level[cur] + 1;
        int k = 0;
        for (int a = 0; a < d; ++a) k |= int((c[a] >> (L - Lc)) & 1) << a;
        cur = child0[cur] + k;
    }
    return cur;
}
}  // namespace pdmk
