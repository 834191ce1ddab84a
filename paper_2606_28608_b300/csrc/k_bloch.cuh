// k_bloch.cuh -- quasi-periodic (Bloch) lattice sums (Sec. 3.7):
//     Phi(x) = sum_n sum_j q_j e^{i beta.L n} G(x - y_j - L n),   Phi(x + L n) = e^{i beta.L n} Phi(x).
// The near field keeps its real kernels: every copy of a source in the extended domain (the
// point itself wrapped into the cell, and its images) carries the complex charge
// q_j e^{i beta.d} with d the lattice vector from the given position to the copy, and the
// real and imaginary parts run as two real evaluations.  The smooth part is
//     (1/V) sum_m hat-W_0(|k_m + beta|) e^{i (k_m + beta).x} sum_j q_j e^{-i (k_m + beta).y_j}
// : spreading of the complex strengths q_j e^{-i beta.y_j} (two real spreads), a complex
// transform of the full grid, scaling at the shifted modes with m = 0 kept (no mode vanishes
// when beta is not a reciprocal-lattice vector), the inverse transform, interpolation of the
// periodic factor F and post-modulation by e^{i beta.x}.
#pragma once
#include "kernels_common.cuh"

namespace pdmk {

// charges of one part (0: real, 1: imaginary) for the near field (every sorted copy) and
// for the spreading (every point, strength q e^{-i beta.y})
template <typename T>
__global__ void k_bloch_charges(int part, int d, const double* __restrict__ q, const double* __restrict__ beta,
                                int64_t nsrc, const int* __restrict__ src_orig, const double* __restrict__ disp,
                                T* __restrict__ src4, int64_t nspread, const int* __restrict__ spread_orig,
                                const double* __restrict__ y, T* __restrict__ spread_dq, int64_t ntgt,
                                const int* __restrict__ tgt_orig, T* __restrict__ tgt4) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (int64_t i = i0; i < nsrc; i += stride) {
        double th = 0;
        for (int a = 0; a < d; ++a) th += beta[a] * disp[i * d + a];
        src4[i * 4 + 3] = T(q[src_orig[i]] * (part == 0 ? cos(th) : sin(th)));
    }
    for (int64_t i = i0; i < nspread; i += stride) {
        const int o = spread_orig[i];
        double th = 0;
        for (int a = 0; a < d; ++a) th += beta[a] * y[size_t(o) * d + a];
        spread_dq[i * 4 + 3] = T(q[o] * (part == 0 ? cos(th) : -sin(th)));
    }
    // the whole-grid 2D spreading kernels read the strengths from the target records
    for (int64_t i = i0; i < ntgt; i += stride) {
        const int o = tgt_orig[i];
        double th = 0;
        for (int a = 0; a < d; ++a) th += beta[a] * y[size_t(o) * d + a];
        tgt4[i * 4 + 3] = T(q[o] * (part == 0 ? cos(th) : -sin(th)));
    }
}

struct BlochWeightArgs {
    int d;
    int M0, M1, M2;
    double Rinv[9];       // oriented frame (row-major)
    double beta_o[3];     // beta in the oriented frame
    double rc, c, V;
    const double* glx;    // quadrature nodes on [0, 1]
    const double* glw;    // weights times psi(node) / c0
    int ngl;
    const double* ph;     // window transform per axis index: M0 | M1 | M2 values
};

// weight of every mode of the full grid: hat-W_0(|k_m + beta|) / (V prod_i phi-hat_i(m_i)^2),
// with hat-W_0(k) = hat-w(k r_c) / k^2 inside the active ball |k| r_c <= c and zero beyond it
// and on the Nyquist planes (as the periodic weights); the m = 0 mode keeps its weight
__global__ void k_bloch_weights(BlochWeightArgs a, double* __restrict__ w) {
    const int64_t ncell = int64_t(a.M0) * a.M1 * (a.d == 3 ? a.M2 : 1);
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < ncell; c += int64_t(gridDim.x) * blockDim.x) {
        const int j0 = int(c % a.M0), j1 = int((c / a.M0) % a.M1), j2 = a.d == 3 ? int(c / (int64_t(a.M0) * a.M1)) : 0;
        const int jj[3] = {j0, j1, j2};
        const int MM[3] = {a.M0, a.M1, a.M2};
        bool nyq = false;
        int m[3] = {0, 0, 0};
        for (int i = 0; i < a.d; ++i) {
            if (jj[i] == MM[i] / 2) nyq = true;
            m[i] = jj[i] <= MM[i] / 2 ? jj[i] : jj[i] - MM[i];
        }
        double val = 0;
        if (!nyq) {
            double k2 = 0;
            for (int b = 0; b < a.d; ++b) {
                double s = 0;
                for (int i = 0; i < a.d; ++i) s += a.Rinv[i * a.d + b] * m[i];
                s = 2.0 * 3.14159265358979323846 * s + a.beta_o[b];
                k2 += s * s;
            }
            const double kk = sqrt(k2);
            if (kk * a.rc <= a.c && k2 > 0) {
                double wh = 0;
                for (int g = 0; g < a.ngl; ++g) wh += a.glw[g] * cos(kk * a.rc * a.glx[g]);
                double den = a.V;
                int off = 0;
                for (int i = 0; i < a.d; ++i) {
                    const double f = a.ph[off + jj[i]];
                    den *= f * f;
                    off += MM[i];
                }
                val = wh / k2 / den;
            }
        }
        w[c] = val;
    }
}

// real and imaginary grids into one complex grid (interleaved), and back after the transforms
__global__ void k_bloch_interleave(const double* __restrict__ re, const double* __restrict__ im,
                                   double* __restrict__ cg, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        cg[2 * i] = re[i];
        cg[2 * i + 1] = im[i];
    }
}
__global__ void k_bloch_scale(double* __restrict__ cg, const double* __restrict__ w, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        cg[2 * i] *= w[i];
        cg[2 * i + 1] *= w[i];
    }
}
template <typename T>
__global__ void k_bloch_deinterleave(const double* __restrict__ cg, T* __restrict__ re, T* __restrict__ im,
                                     int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        re[i] = T(cg[2 * i]);
        im[i] = T(cg[2 * i + 1]);
    }
}

struct BlochAssembleArgs {
    int64_t nt;
    const int* tgt_orig;
    const double* self_w;   // W_{L(i)}(0) per sorted target
    const double* q;        // the caller's charges
    const double* tdisp;    // per sorted target: lattice vector from its given position to its copy (d)
    const double* y;        // the caller's positions (d per point)
    const double* beta;     // caller frame (device, d)
    const double* pn[2];    // near potential (real, imaginary parts), per sorted target
    const double* gn[2];    // near gradient (tree frame), d per sorted target
    const double* pp[2];    // plane-wave part (may be null)
    const double* gp[2];
    const double* pf[2];    // interpolated periodic factor F and its gradient in grid units
    const double* gf[2];
    double G[9];            // R^{-T} diag(M)
    double Qt[9];           // Q^T
    double* pot_out;        // 2 per point (real, imaginary)
    double* grad_out;       // 2 d per point, or null
    int64_t out_first;
};

// Phi(y) = e^{-i beta.d} [near(copy) - W_L(0) q e^{i beta.d}] + e^{i beta.y} F(copy)
// grad   = e^{-i beta.d} grad near(copy) + e^{i beta.y} (i beta F + grad F)
template <int D>
__global__ void __launch_bounds__(256) k_assemble_bloch(BlochAssembleArgs a) {
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < a.nt; t += int64_t(gridDim.x) * blockDim.x) {
        const int i = a.tgt_orig[t];
        if (i < a.out_first) continue;
        const int64_t o = i - a.out_first;
        double thd = 0, thy = 0;
        for (int k = 0; k < D; ++k) {
            thd += a.beta[k] * a.tdisp[t * D + k];
            thy += a.beta[k] * a.y[size_t(i) * D + k];
        }
        const double cd = cos(thd), sd = sin(thd), cy = cos(thy), sy = sin(thy);
        const double qs = a.q[i] * a.self_w[t];
        double nr = a.pn[0][t] - qs * cd, ni = a.pn[1][t] - qs * sd;
        if (a.pp[0]) {
            nr += a.pp[0][t];
            ni += a.pp[1][t];
        }
        const double fr = a.pf[0][t], fi = a.pf[1][t];
        // e^{-i thd} (nr + i ni) + e^{i thy} (fr + i fi)
        a.pot_out[2 * o] = cd * nr + sd * ni + cy * fr - sy * fi;
        a.pot_out[2 * o + 1] = cd * ni - sd * nr + cy * fi + sy * fr;
        if (!a.grad_out) continue;
        double gnr[D], gni[D], gfr[D], gfi[D];
        for (int k = 0; k < D; ++k) {
            double sr = 0, si = 0, ur = a.gn[0][t * D + k], ui = a.gn[1][t * D + k];
            if (a.gp[0]) {
                ur += a.gp[0][t * D + k];
                ui += a.gp[1][t * D + k];
            }
            gnr[k] = ur;
            gni[k] = ui;
            for (int j = 0; j < D; ++j) {
                sr += a.G[k * D + j] * a.gf[0][t * D + j];
                si += a.G[k * D + j] * a.gf[1][t * D + j];
            }
            gfr[k] = sr;
            gfi[k] = si;
        }
        for (int k = 0; k < D; ++k) {
            // caller frame: Q^T of the tree-frame vectors
            double nrk = 0, nik = 0, frk = 0, fik = 0;
            for (int j = 0; j < D; ++j) {
                nrk += a.Qt[k * D + j] * gnr[j];
                nik += a.Qt[k * D + j] * gni[j];
                frk += a.Qt[k * D + j] * gfr[j];
                fik += a.Qt[k * D + j] * gfi[j];
            }
            // i beta F + grad F
            const double br = frk - a.beta[k] * fi, bi = fik + a.beta[k] * fr;
            a.grad_out[(o * D + k) * 2] = cd * nrk + sd * nik + cy * br - sy * bi;
            a.grad_out[(o * D + k) * 2 + 1] = cd * nik - sd * nrk + cy * bi + sy * br;
        }
    }
}

}  // namespace pdmk
