/*
 * ewald_oracle.c -- plain FP64 Ewald summation for periodic Laplace lattice sums.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent oracle against which the
 * CUDA path is checked.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load it.  It shares no code, header, table or constant with the
 * product library, and the product library never calls it.
 *
 * What it computes (paper Sec. 1, Eq. (1.1)-(1.2), tin-foil convention):
 *
 *   Phi(x_i) = sum_{n in Z^d} sum_j' q_j G(x_i - y_j - L n)
 *
 * with G(r) = 1/(4 pi r) in 3D and -log(r)/(2 pi) in 2D, the n = 0, j = self term
 * removed, the k = 0 Fourier mode dropped (the periodic potential is represented by a
 * Fourier series on the reciprocal lattice k_m = 2 pi L^{-T} m, m != 0), and, for a
 * non-neutral set of charges, the uniform neutralising background that makes the
 * potential zero-mean over the cell.  It is evaluated by classical Ewald summation
 * (fast Ewald methods are prior art cited in the paper's introduction):
 *
 *   Phi = sum_{images, r < rcut} q_j S(r)              (short range, real space)
 *       + (1/V) sum_{k != 0, |k| < kcut} g(k) Re[ rho(k) e^{i k.x} ]  (long range)
 *       - q_self * S0                                   (self energy of the split)
 *       - Q / (4 alpha^2 V)                              (zero mean for Q = sum q != 0)
 *
 *   3D: S(r) = erfc(alpha r)/(4 pi r),  S0 = alpha / (2 pi^{3/2})
 *   2D: S(r) = E1(alpha^2 r^2)/(4 pi),  S0 = (gamma + 2 ln alpha)/(4 pi)
 *   g(k) = exp(-k^2/(4 alpha^2)) / k^2,  rho(k) = sum_j q_j e^{-i k.y_j}
 *
 * and the gradient is the analytic derivative of every term.  All sums accumulate in
 * long double.  Cost is O(M * neighbours + (N + M) * modes); it is meant to be slow
 * and obviously correct, not fast.
 *
 * oracle_ewald_bloch (end of file) is the quasi-periodic counterpart (paper Sec. 3.7):
 * image charges carry the Bloch phase e^{i beta.L n}, the reciprocal sum runs over the
 * shifted modes k_m + beta with every mode kept, and no neutrality is needed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_EULER_GAMMA 0.57721566490153286060651209008240243

/* Exponential integral E1(x), x > 0, written from its power series (x <= 1) and its
 * classical continued fraction (x > 1), evaluated backwards from a fixed depth. */
static double orc_e1(double x) {
    if (x <= 1.0) {
        /* E1(x) = -gamma - ln x + sum_{k>=1} (-1)^{k+1} x^k / (k k!) */
        long double sum = 0.0L, term = 1.0L;
        for (int k = 1; k < 60; ++k) {
            term *= -(long double)x / (long double)k; /* (-x)^k / k! */
            long double add = -term / (long double)k;  /* (-1)^{k+1} x^k/(k k!) */
            sum += add;
            if (fabsl(add) < 1e-22L) break;
        }
        return (double)(-(long double)ORC_EULER_GAMMA - logl((long double)x) + sum);
    }
    /* E1(x) = e^{-x} / (x + 1 - 1^2/(x + 3 - 2^2/(x + 5 - 3^2/(x + 7 - ...)))) */
    const int depth = 120;
    long double t = (long double)x + 2.0L * depth + 1.0L;
    for (int k = depth; k >= 1; --k) t = (long double)x + 2.0L * k - 1.0L - (long double)k * k / t;
    return (double)(expl(-(long double)x) / t);
}

double oracle_e1(double x) { return orc_e1(x); }

/* short-range kernel S(r) and S'(r) */
static inline void orc_short(int d, double alpha, double r, double* s, double* ds) {
    if (d == 3) {
        double ar = alpha * r;
        double e = erfc(ar);
        *s = e / (4.0 * ORC_PI * r);
        /* d/dr [erfc(a r)/(4 pi r)] = -[erfc(a r)/r^2 + (2a/sqrt(pi)) e^{-a^2 r^2}/r]/(4 pi) */
        *ds = -(e / (r * r) + 2.0 * alpha / sqrt(ORC_PI) * exp(-ar * ar) / r) / (4.0 * ORC_PI);
    } else {
        double u = alpha * alpha * r * r;
        *s = orc_e1(u) / (4.0 * ORC_PI);
        /* d/dr E1(a^2 r^2)/(4 pi) = -(e^{-u}/u) * 2 a^2 r/(4 pi) = -e^{-u}/(2 pi r) */
        *ds = -exp(-u) / (2.0 * ORC_PI * r);
    }
}

/* Inverse of a d x d column-major matrix (d = 2, 3) by cofactors. Returns det. */
static double orc_inv(int d, const double* L, double* Li) {
#define A(i, j) L[(i) + (j) * d]
    if (d == 2) {
        double det = A(0, 0) * A(1, 1) - A(0, 1) * A(1, 0);
        Li[0] = A(1, 1) / det; Li[2] = -A(0, 1) / det;
        Li[1] = -A(1, 0) / det; Li[3] = A(0, 0) / det;
        return det;
    }
    double c00 = A(1, 1) * A(2, 2) - A(1, 2) * A(2, 1);
    double c01 = A(1, 2) * A(2, 0) - A(1, 0) * A(2, 2);
    double c02 = A(1, 0) * A(2, 1) - A(1, 1) * A(2, 0);
    double det = A(0, 0) * c00 + A(0, 1) * c01 + A(0, 2) * c02;
    double inv[3][3];
    inv[0][0] = c00; inv[1][0] = c01; inv[2][0] = c02;
    inv[0][1] = A(0, 2) * A(2, 1) - A(0, 1) * A(2, 2);
    inv[1][1] = A(0, 0) * A(2, 2) - A(0, 2) * A(2, 0);
    inv[2][1] = A(0, 1) * A(2, 0) - A(0, 0) * A(2, 1);
    inv[0][2] = A(0, 1) * A(1, 2) - A(0, 2) * A(1, 1);
    inv[1][2] = A(0, 2) * A(1, 0) - A(0, 0) * A(1, 2);
    inv[2][2] = A(0, 0) * A(1, 1) - A(0, 1) * A(1, 0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Li[i + j * 3] = inv[i][j] / det;
    return det;
#undef A
}

/*
 * oracle_ewald: potential (and optionally gradient) at m targets.
 *   d        2 or 3
 *   L        d*d column-major lattice matrix, column j = lattice vector a_j
 *   n, y, q  sources: y is n*d row-major (any position; images are implicit), q is n
 *   m, x     targets: x is m*d row-major
 *   self_idx length m: index j of the source that coincides with target i (its n = 0
 *            self pair is excluded and the split's self energy subtracted), or -1
 *   alpha    Ewald splitting parameter; rcut, kcut the real/reciprocal cut-offs
 *   pot      out, m;  grad out, m*d row-major, or NULL
 *   nthreads OpenMP threads (<= 0: runtime default)
 * Returns 0, or -1 on a bad argument / allocation failure.
 */
int oracle_ewald(int d, const double* L, int64_t n, const double* y, const double* q, int64_t m,
                 const double* x, const int64_t* self_idx, double alpha, double rcut, double kcut,
                 double* pot, double* grad, int nthreads) {
    if ((d != 2 && d != 3) || n < 0 || m < 0 || alpha <= 0 || rcut <= 0 || kcut <= 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double Li[9];
    double det = orc_inv(d, L, Li);
    double V = fabs(det);
    if (!(V > 0)) return -1;

    /* fractional coordinates of sources, wrapped into [0,1), and the whole lattice steps
       the wrap took (w_j = floor(L^{-1} y_j)): v locates a source for the binning and the
       structure factors, while a pair's displacement x - y_j - L n is formed from the
       caller's coordinates with the integer shift n, so that nearby points keep their
       exact difference */
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * d);
    int* wj = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1) * d);
    if (!v || !wj) { free(v); free(wj); return -1; }
    for (int64_t j = 0; j < n; ++j)
        for (int a = 0; a < d; ++a) {
            double s = 0;
            for (int b = 0; b < d; ++b) s += Li[a + b * d] * y[j * d + b];
            const double f = floor(s);
            v[j * d + a] = s - f;
            wj[j * d + a] = (int)f;
        }

    long double Qsum = 0;
    for (int64_t j = 0; j < n; ++j) Qsum += q[j];

    /* ---------------- real space: bins in fractional coordinates --------------- */
    /* distance between adjacent lattice planes u_a = const is 1/|row a of L^{-1}| */
    int nb[3] = {1, 1, 1}, R[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
        double rn = 0;
        for (int b = 0; b < d; ++b) rn += Li[a + b * d] * Li[a + b * d];
        double width = 1.0 / sqrt(rn);
        int k = (int)floor(width / rcut);
        if (k < 1) k = 1;
        if (k > 256) k = 256;
        nb[a] = k;
        /* an image within rcut differs by at most rcut/width in fractional coord a */
        R[a] = (int)floor(rcut * nb[a] / width) + 1;
    }
    int64_t nbins = (int64_t)nb[0] * nb[1] * (d == 3 ? nb[2] : 1);
    int64_t* bstart = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
    int64_t* border = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* bcur = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
    if (!bstart || !border || !bcur) { free(v); free(wj); free(bstart); free(border); free(bcur); return -1; }
#define BIN_OF(uu, a) ((int)((uu) * nb[a]) >= nb[a] ? nb[a] - 1 : (int)((uu) * nb[a]))
    for (int64_t j = 0; j < n; ++j) {
        int64_t b = 0;
        for (int a = d - 1; a >= 0; --a) b = b * nb[a] + BIN_OF(v[j * d + a], a);
        bstart[b + 1]++;
    }
    for (int64_t b = 0; b < nbins; ++b) bstart[b + 1] += bstart[b];
    for (int64_t j = 0; j < n; ++j) {
        int64_t b = 0;
        for (int a = d - 1; a >= 0; --a) b = b * nb[a] + BIN_OF(v[j * d + a], a);
        border[bstart[b] + bcur[b]++] = j;
    }
    free(bcur);

    const double rc2 = rcut * rcut;
    double S0 = (d == 3) ? alpha / (2.0 * ORC_PI * sqrt(ORC_PI))
                         : (ORC_EULER_GAMMA + 2.0 * log(alpha)) / (4.0 * ORC_PI);

    /* ---------------- reciprocal space: half-space mode list ------------------- */
    /* |m_a| <= kcut |a_a| / (2 pi) by Cauchy-Schwarz on m_a = a_a . k / (2 pi) */
    int mmax[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
        double an = 0;
        for (int b = 0; b < d; ++b) an += L[b + a * d] * L[b + a * d];
        mmax[a] = (int)ceil(kcut * sqrt(an) / (2.0 * ORC_PI));
    }
    int64_t cap = 1;
    for (int a = 0; a < d; ++a) cap *= (2 * mmax[a] + 1);
    int* modes = (int*)malloc(sizeof(int) * (size_t)cap * 3);
    double* kvec = (double*)malloc(sizeof(double) * (size_t)cap * 3);
    double* gk = (double*)malloc(sizeof(double) * (size_t)cap);
    if (!modes || !kvec || !gk) { free(v); free(wj); free(bstart); free(border); free(modes); free(kvec); free(gk); return -1; }
    int64_t nk = 0;
    int m2lo = (d == 3) ? -mmax[2] : 0, m2hi = (d == 3) ? mmax[2] : 0;
    for (int m0 = 0; m0 <= mmax[0]; ++m0)
        for (int m1 = -mmax[1]; m1 <= mmax[1]; ++m1)
            for (int m2 = m2lo; m2 <= m2hi; ++m2) {
                /* half space: first non-zero component positive */
                if (m0 == 0) {
                    if (m1 < 0) continue;
                    if (m1 == 0 && m2 <= 0) continue;
                }
                int mm[3] = {m0, m1, m2};
                double k[3] = {0, 0, 0}, k2 = 0;
                /* k = 2 pi L^{-T} m : k_b = 2 pi sum_a Li[a][b] m_a */
                for (int b = 0; b < d; ++b) {
                    double s = 0;
                    for (int a = 0; a < d; ++a) s += Li[a + b * d] * mm[a];
                    k[b] = 2.0 * ORC_PI * s;
                    k2 += k[b] * k[b];
                }
                if (k2 > kcut * kcut) continue;
                for (int a = 0; a < 3; ++a) { modes[nk * 3 + a] = mm[a]; kvec[nk * 3 + a] = k[a]; }
                gk[nk] = exp(-k2 / (4.0 * alpha * alpha)) / k2;
                ++nk;
            }

    /* structure factors rho(k) = sum_j q_j e^{-2 pi i m.v_j}, from per-source tables of
       e^{-2 pi i m_a v_a} for 0 <= m_a <= mmax_a (negative m by conjugation) */
    long double* rho_re = (long double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(long double));
    long double* rho_im = (long double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(long double));
    const int64_t blk = 2048;
    int tw = 0;
    for (int a = 0; a < d; ++a) tw += mmax[a] + 1;
    double* tab = (double*)malloc(sizeof(double) * (size_t)blk * tw * 2);
    if (!rho_re || !rho_im || !tab) {
        free(v); free(wj); free(bstart); free(border); free(modes); free(kvec); free(gk);
        free(rho_re); free(rho_im); free(tab); return -1;
    }
    int toff[3] = {0, 0, 0};
    for (int a = 1; a < d; ++a) toff[a] = toff[a - 1] + mmax[a - 1] + 1;
    for (int64_t j0 = 0; j0 < n; j0 += blk) {
        int64_t jn = (n - j0 < blk) ? n - j0 : blk;
#pragma omp parallel for schedule(static)
        for (int64_t jj = 0; jj < jn; ++jj) {
            for (int a = 0; a < d; ++a)
                for (int mm = 0; mm <= mmax[a]; ++mm) {
                    double ph = -2.0 * ORC_PI * mm * v[(j0 + jj) * d + a];
                    tab[(jj * tw + toff[a] + mm) * 2 + 0] = cos(ph);
                    tab[(jj * tw + toff[a] + mm) * 2 + 1] = sin(ph);
                }
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t ik = 0; ik < nk; ++ik) {
            long double sr = 0, si = 0;
            for (int64_t jj = 0; jj < jn; ++jj) {
                double pr = 1.0, pi_ = 0.0;
                for (int a = 0; a < d; ++a) {
                    int mm = modes[ik * 3 + a];
                    double er = tab[(jj * tw + toff[a] + abs(mm)) * 2 + 0];
                    double ei = tab[(jj * tw + toff[a] + abs(mm)) * 2 + 1];
                    if (mm < 0) ei = -ei;
                    double nr = pr * er - pi_ * ei, ni = pr * ei + pi_ * er;
                    pr = nr; pi_ = ni;
                }
                sr += (long double)q[j0 + jj] * pr;
                si += (long double)q[j0 + jj] * pi_;
            }
            rho_re[ik] += sr;
            rho_im[ik] += si;
        }
    }
    free(tab);

    /* ---------------- evaluation at targets ------------------------------------ */
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < m; ++i) {
        const double* xi = x + i * d;
        double u[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            double s = 0;
            for (int b = 0; b < d; ++b) s += Li[a + b * d] * xi[b];
            u[a] = s;
        }
        /* wrapped target and the lattice shift that wraps it */
        double uw[3] = {0, 0, 0};
        int tb[3] = {0, 0, 0}, tw[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            const double f = floor(u[a]);
            uw[a] = u[a] - f;
            tw[a] = (int)f;
            tb[a] = BIN_OF(uw[a], a);
        }
        int64_t self = self_idx ? self_idx[i] : -1;
        long double phi = 0, g[3] = {0, 0, 0};
        int o2lo = (d == 3) ? -R[2] : 0, o2hi = (d == 3) ? R[2] : 0;
        for (int o0 = -R[0]; o0 <= R[0]; ++o0)
            for (int o1 = -R[1]; o1 <= R[1]; ++o1)
                for (int o2 = o2lo; o2 <= o2hi; ++o2) {
                    int off[3] = {o0, o1, o2};
                    int bb[3] = {0, 0, 0}, sh[3] = {0, 0, 0};
                    for (int a = 0; a < d; ++a) {
                        int b = tb[a] + off[a];
                        /* floor division: shift sh and bin bb with b = sh*nb + bb */
                        int s = (b >= 0) ? b / nb[a] : -((-b + nb[a] - 1) / nb[a]);
                        sh[a] = s;
                        bb[a] = b - s * nb[a];
                    }
                    int64_t bidx = 0;
                    for (int a = d - 1; a >= 0; --a) bidx = bidx * nb[a] + bb[a];
                    int zero_shift = 1;
                    for (int a = 0; a < d; ++a) zero_shift &= (sh[a] == 0);
                    for (int64_t t = bstart[bidx]; t < bstart[bidx + 1]; ++t) {
                        int64_t j = border[t];
                        /* x - y_j - L n with n = tw - w_j + sh: the wrapped target minus the
                           shifted wrapped source, written in the caller's coordinates */
                        int nn[3] = {0, 0, 0};
                        for (int a = 0; a < d; ++a) nn[a] = tw[a] - wj[j * d + a] + sh[a];
                        double dx[3] = {0, 0, 0}, r2 = 0;
                        for (int b = 0; b < d; ++b) {
                            double ln = 0;
                            for (int a = 0; a < d; ++a) ln += L[b + a * d] * nn[a];
                            dx[b] = (xi[b] - y[j * d + b]) - ln;
                            r2 += dx[b] * dx[b];
                        }
                        if (r2 > rc2) continue;
                        if (zero_shift && j == self) continue;
                        if (r2 == 0.0) continue; /* coincident non-self pair: undefined, skipped */
                        double r = sqrt(r2), s, ds;
                        orc_short(d, alpha, r, &s, &ds);
                        phi += (long double)q[j] * s;
                        for (int b = 0; b < d; ++b) g[b] += (long double)q[j] * ds * dx[b] / r;
                    }
                }
        /* reciprocal part at the wrapped target (the series is periodic) */
        long double pr_sum = 0, g2[3] = {0, 0, 0};
        for (int64_t ik = 0; ik < nk; ++ik) {
            double kx = 0;
            for (int a = 0; a < d; ++a) kx += 2.0 * ORC_PI * modes[ik * 3 + a] * uw[a];
            double c = cos(kx), sn = sin(kx);
            /* Re[rho e^{ikx}] and Im[rho e^{ikx}] */
            long double re = rho_re[ik] * c - rho_im[ik] * sn;
            long double im = rho_re[ik] * sn + rho_im[ik] * c;
            pr_sum += gk[ik] * re;
            for (int b = 0; b < d; ++b) g2[b] += gk[ik] * kvec[ik * 3 + b] * im;
        }
        /* half-space sum counts k and -k: factor 2 */
        phi += 2.0L * pr_sum / V;
        for (int b = 0; b < d; ++b) g[b] += -2.0L * g2[b] / V;
        if (self >= 0) phi -= (long double)q[self] * S0;
        phi -= Qsum / (4.0L * alpha * alpha * V);
        pot[i] = (double)phi;
        if (grad)
            for (int b = 0; b < d; ++b) grad[i * d + b] = (double)g[b];
    }
#undef BIN_OF
    free(v); free(wj); free(bstart); free(border); free(modes); free(kvec); free(gk);
    free(rho_re); free(rho_im);
    return err;
}

/*
 * oracle_ewald_bloch: quasi-periodic (Bloch) potential and gradient at m targets,
 *
 *   Phi(x) = sum_{n in Z^d} sum_j' q_j e^{i beta.L n} G(x - y_j - L n)
 *
 * (paper Sec. 3.7, the periodised kernel with the Bloch phase), which satisfies
 * Phi(x + L n) = e^{i beta.L n} Phi(x).  Same Ewald split as oracle_ewald, with
 *
 *   real space:  sum_{n, r < rcut} q_j e^{i beta.L n} S(|x - y_j - L n|)
 *   reciprocal:  (1/V) sum_m g(|k_m + beta|) e^{i (k_m + beta).x} sum_j q_j e^{-i (k_m + beta).y_j}
 *                over every mode m (no half space, no mode dropped), |k_m + beta| < kcut
 *   self:        - q_self S0
 *
 * by Poisson summation of sum_n f(z - L n) e^{i beta.L n}.  No neutrality is needed; beta
 * must not be a reciprocal-lattice vector (some k_m + beta = 0): then it returns -2.
 * Written as direct loops over sources, shifts and modes: meant for small N.
 * The potential and gradient are complex: pot_re/pot_im (m), grad_re/grad_im (m*d) or NULL.
 */
int oracle_ewald_bloch(int d, const double* L, int64_t n, const double* y, const double* q, int64_t m,
                       const double* x, const int64_t* self_idx, const double* beta, double alpha,
                       double rcut, double kcut, double* pot_re, double* pot_im, double* grad_re,
                       double* grad_im, int nthreads) {
    if ((d != 2 && d != 3) || n < 0 || m < 0 || alpha <= 0 || rcut <= 0 || kcut <= 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double Li[9];
    double det = orc_inv(d, L, Li);
    double V = fabs(det);
    if (!(V > 0)) return -1;
    /* shifts: |n_a - nearest| <= R_a covers r < rcut (plane spacing 1/|row a of L^{-1}|) */
    int R[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
        double rn = 0;
        for (int b = 0; b < d; ++b) rn += Li[a + b * d] * Li[a + b * d];
        R[a] = (int)ceil(rcut * sqrt(rn)) + 1;
    }
    /* modes: |m_a| <= (kcut + |beta|) |a_a| / (2 pi) */
    double bn = 0;
    for (int b = 0; b < d; ++b) bn += beta[b] * beta[b];
    bn = sqrt(bn);
    int mmax[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
        double an = 0;
        for (int b = 0; b < d; ++b) an += L[b + a * d] * L[b + a * d];
        mmax[a] = (int)ceil((kcut + bn) * sqrt(an) / (2.0 * ORC_PI));
    }
    int64_t cap = 1;
    for (int a = 0; a < d; ++a) cap *= (2 * mmax[a] + 1);
    double* kv = (double*)malloc(sizeof(double) * (size_t)cap * 3);
    double* gk = (double*)malloc(sizeof(double) * (size_t)cap);
    long double* sre = (long double*)calloc((size_t)cap, sizeof(long double));
    long double* sim = (long double*)calloc((size_t)cap, sizeof(long double));
    if (!kv || !gk || !sre || !sim) { free(kv); free(gk); free(sre); free(sim); return -1; }
    int64_t nk = 0;
    int bad = 0;
    int m2lo = (d == 3) ? -mmax[2] : 0, m2hi = (d == 3) ? mmax[2] : 0;
    for (int m0 = -mmax[0]; m0 <= mmax[0]; ++m0)
        for (int m1 = -mmax[1]; m1 <= mmax[1]; ++m1)
            for (int m2 = m2lo; m2 <= m2hi; ++m2) {
                int mm[3] = {m0, m1, m2};
                double k[3] = {0, 0, 0}, k2 = 0;
                for (int b = 0; b < d; ++b) {
                    double s = 0;
                    for (int a = 0; a < d; ++a) s += Li[a + b * d] * mm[a];
                    k[b] = 2.0 * ORC_PI * s + beta[b];
                    k2 += k[b] * k[b];
                }
                if (k2 > kcut * kcut) continue;
                if (!(k2 > 1e-24 * kcut * kcut)) { bad = 1; continue; }
                for (int b = 0; b < 3; ++b) kv[nk * 3 + b] = b < d ? k[b] : 0.0;
                gk[nk] = exp(-k2 / (4.0 * alpha * alpha)) / k2;
                ++nk;
            }
    if (bad) { free(kv); free(gk); free(sre); free(sim); return -2; }
    /* structure factors S(k) = sum_j q_j e^{-i k.y_j}, k = k_m + beta */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t ik = 0; ik < nk; ++ik) {
        long double sr = 0, si = 0;
        for (int64_t j = 0; j < n; ++j) {
            double ph = 0;
            for (int b = 0; b < d; ++b) ph += kv[ik * 3 + b] * y[j * d + b];
            sr += (long double)q[j] * cos(ph);
            si -= (long double)q[j] * sin(ph);
        }
        sre[ik] = sr;
        sim[ik] = si;
    }
    const double rc2 = rcut * rcut;
    const double S0 = (d == 3) ? alpha / (2.0 * ORC_PI * sqrt(ORC_PI))
                               : (ORC_EULER_GAMMA + 2.0 * log(alpha)) / (4.0 * ORC_PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < m; ++i) {
        const double* xi = x + i * d;
        const int64_t self = self_idx ? self_idx[i] : -1;
        long double pr = 0, pim = 0, gr[3] = {0, 0, 0}, gi[3] = {0, 0, 0};
        /* real space */
        for (int64_t j = 0; j < n; ++j) {
            double d0[3] = {0, 0, 0}, f[3] = {0, 0, 0};
            for (int b = 0; b < d; ++b) d0[b] = xi[b] - y[j * d + b];
            int nc[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
                for (int b = 0; b < d; ++b) f[a] += Li[a + b * d] * d0[b];
                nc[a] = (int)floor(f[a] + 0.5);
            }
            int lo2 = (d == 3) ? -R[2] : 0, hi2 = (d == 3) ? R[2] : 0;
            for (int o0 = -R[0]; o0 <= R[0]; ++o0)
                for (int o1 = -R[1]; o1 <= R[1]; ++o1)
                    for (int o2 = lo2; o2 <= hi2; ++o2) {
                        int nn[3] = {nc[0] + o0, nc[1] + o1, d == 3 ? nc[2] + o2 : 0};
                        double dx[3] = {0, 0, 0}, r2 = 0, phase = 0;
                        for (int b = 0; b < d; ++b) {
                            double ln = 0;
                            for (int a = 0; a < d; ++a) ln += L[b + a * d] * nn[a];
                            dx[b] = d0[b] - ln;
                            r2 += dx[b] * dx[b];
                            phase += beta[b] * ln;
                        }
                        if (r2 > rc2) continue;
                        int zero = (nn[0] == 0 && nn[1] == 0 && nn[2] == 0);
                        if (zero && j == self) continue;
                        if (r2 == 0.0) continue;
                        double r = sqrt(r2), s, ds;
                        orc_short(d, alpha, r, &s, &ds);
                        double c = cos(phase), sn = sin(phase);
                        pr += (long double)q[j] * s * c;
                        pim += (long double)q[j] * s * sn;
                        for (int b = 0; b < d; ++b) {
                            gr[b] += (long double)q[j] * ds * dx[b] / r * c;
                            gi[b] += (long double)q[j] * ds * dx[b] / r * sn;
                        }
                    }
        }
        /* reciprocal space: g(k) e^{i k.x} S(k) */
        for (int64_t ik = 0; ik < nk; ++ik) {
            double ph = 0;
            for (int b = 0; b < d; ++b) ph += kv[ik * 3 + b] * xi[b];
            double c = cos(ph), sn = sin(ph);
            long double re = sre[ik] * c - sim[ik] * sn; /* Re[S e^{ikx}] */
            long double im = sre[ik] * sn + sim[ik] * c; /* Im[S e^{ikx}] */
            pr += gk[ik] * re / V;
            pim += gk[ik] * im / V;
            /* grad: i k g S e^{ikx} -> Re = -k g Im, Im = k g Re */
            for (int b = 0; b < d; ++b) {
                gr[b] += -kv[ik * 3 + b] * gk[ik] * im / V;
                gi[b] += kv[ik * 3 + b] * gk[ik] * re / V;
            }
        }
        if (self >= 0) pr -= (long double)q[self] * S0;
        pot_re[i] = (double)pr;
        pot_im[i] = (double)pim;
        if (grad_re && grad_im)
            for (int b = 0; b < d; ++b) {
                grad_re[i * d + b] = (double)gr[b];
                grad_im[i * d + b] = (double)gi[b];
            }
    }
    free(kv); free(gk); free(sre); free(sim);
    return 0;
}
