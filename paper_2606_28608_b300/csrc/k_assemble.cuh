// k_assemble.cuh -- charge gathers into the device layouts, the total charge, and the
// final assembly (Eq. (3.16)-(3.17), Algorithm 1 step 5), the potential in FP64:
//   Phi = Phi_near + Phi_pw + Phi_far - W_{L(i)}(0) q_i - Q hat-R_0(0) / V,
// gradient = grad_near + grad_pw + R^{-T} (M * grad_gridcoords Phi_far), rotated back to
// the caller's frame and written in the caller's order.
#pragma once
#include "kernels_common.cuh"

namespace pdmk {

template <typename T>
struct GatherArgs {
    const double* q;       // user charges (device)
    int64_t nsrc;          // sorted sources (with images)
    const int* src_orig;
    T* src4;               // writes .w
    int64_t nspread;
    const int* spread_orig;
    T* spread_dq;          // writes [3]
    int64_t ntgt;
    const int* tgt_orig;
    T* tgt4;               // writes .w
    double* q_tgt;
};

template <typename T>
__global__ void k_gather_charges(GatherArgs<T> a) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (int64_t i = i0; i < a.nsrc; i += stride) a.src4[i * 4 + 3] = T(a.q[a.src_orig[i]]);
    for (int64_t i = i0; i < a.nspread; i += stride) a.spread_dq[i * 4 + 3] = T(a.q[a.spread_orig[i]]);
    for (int64_t i = i0; i < a.ntgt; i += stride) {
        const double qq = a.q[a.tgt_orig[i]];
        a.tgt4[i * 4 + 3] = T(qq);
        a.q_tgt[i] = qq;
    }
}

// Deterministic two-stage sums (fixed block ranges, fixed tree orders):
// out[0] = sum q, out[1] = sum |q|, out[2] = number of non-finite values.
// Stage 1: block b sums its contiguous range into part[3 b .. 3 b + 2].
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_charge_sums_part(const double* q, int64_t n, double* part) {
    __shared__ double s0[kSumThreads], s1[kSumThreads], s2[kSumThreads];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = min(n, int64_t(blockIdx.x) * per), i1 = min(n, i0 + per);
    double a = 0, b = 0, c = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double v = q[i];
        if (isfinite(v)) { a += v; b += fabs(v); } else { c += 1; }
    }
    s0[threadIdx.x] = a; s1[threadIdx.x] = b; s2[threadIdx.x] = c;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
            s2[threadIdx.x] += s2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = s0[0];
        part[3 * blockIdx.x + 1] = s1[0];
        part[3 * blockIdx.x + 2] = s2[0];
    }
}
// Stage 2: one block sums the nb partials.
__global__ void __launch_bounds__(kSumThreads) k_charge_sums_final(const double* part, int nb, double* out) {
    __shared__ double s0[kSumThreads], s1[kSumThreads], s2[kSumThreads];
    double a = 0, b = 0, c = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part[3 * i + 0];
        b += part[3 * i + 1];
        c += part[3 * i + 2];
    }
    s0[threadIdx.x] = a; s1[threadIdx.x] = b; s2[threadIdx.x] = c;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
            s2[threadIdx.x] += s2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s0[0]; out[1] = s1[0]; out[2] = s2[0]; }
}

struct AssembleArgs {
    int64_t nt;
    int d;
    const int* tgt_orig;
    const double* self_w;    // W_{L(i)}(0) per target
    const double* q_tgt;
    const double* pot_near;  const double* grad_near;
    const double* pot_pw;    const double* grad_pw;   // may be null
    const double* pot_far;   const double* gradu_far; // gradient w.r.t. M_i u_i
    const double* qsum;      // device: total charge
    double mean_coef;        // hat-R_0(0) / V
    double G[9];             // R^{-T} diag(M): grad_x = G gradu  (row-major d x d)
    double Qt[9];            // Q^T: user-frame rotation (row-major d x d)
    double* pot_out;         // user order
    double* grad_out;        // user order, d per point, or null
    int64_t out_first;       // caller-order points before this one are not written
};

// The potential (self term, mean correction, the 2D logarithmic cancellation between the
// parts) is summed in FP64.  The gradient parts are summed and rotated back to the caller's
// frame in GT: FP32 on the mixed path (FP64 issue on B300 is a small fraction of FP32, and
// this kernel runs after the branches join, on the critical path), FP64 on the FP64 path.
template <int D, typename GT>
__global__ void __launch_bounds__(256) k_assemble(AssembleArgs a) {
    const double corr = a.qsum[0] * a.mean_coef;
    GT G[D * D], Qt[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) {
        G[k] = GT(a.G[k]);
        Qt[k] = GT(a.Qt[k]);
    }
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < a.nt;
         t += int64_t(gridDim.x) * blockDim.x) {
        double p = a.pot_near[t] + a.pot_far[t] - a.self_w[t] * a.q_tgt[t] - corr;
        if (a.pot_pw) p += a.pot_pw[t];
        if (a.tgt_orig[t] < a.out_first) continue;
        const int64_t o = a.tgt_orig[t] - a.out_first;
        a.pot_out[o] = p;
        if (a.grad_out) {
            GT gu[D], g[D];
#pragma unroll
            for (int j = 0; j < D; ++j) gu[j] = GT(a.gradu_far[t * D + j]);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                GT s = GT(a.grad_near[t * D + i]);
                if (a.grad_pw) s += GT(a.grad_pw[t * D + i]);
#pragma unroll
                for (int j = 0; j < D; ++j) s = fma(G[i * D + j], gu[j], s);
                g[i] = s;
            }
#pragma unroll
            for (int i = 0; i < D; ++i) {
                GT s = GT(0);
#pragma unroll
                for (int j = 0; j < D; ++j) s = fma(Qt[i * D + j], g[j], s);
                a.grad_out[o * D + i] = double(s);
            }
        }
    }
}

}  // namespace pdmk
