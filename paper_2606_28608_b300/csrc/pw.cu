// pw.cu -- plane-wave passes of the difference kernels D_l (Sec. 2.3, Eq. (2.5)-(2.6)) on the
// extended-domain tree (Sec. 3.5: the free-space DMK with the root W_0 step omitted).
//
// Representation.  A box of side h at level l carries
//   * proxy moments  Q[m] = sum_{y in box} q_y prod_i T_{m_i}(t_i(y)),  t = 2 (y - c)/h
//     (Chebyshev moments; the box's sources act on smooth kernels through them),
//   * local coefficients a[m]: the D-field of coarser levels and of its own level inside
//     the box is  sum_m a[m] prod_i T_{m_i}(t_i(x)),
// for 0 <= m_i < p.  Plane waves sample D-hat_l on the grid xi = (2 pi / (3 h)) k,
// |k_i| <= K: the spacing makes the trapezoidal rule alias-free for colleague interactions
// (|x - y|_inf <= 2h, D_l supported in |x - y| <= h), and D-hat_l is negligible beyond
// |xi| = 2c/h.  With these choices every per-level operator is level independent:
//   outgoing  out[k]  = sum_m Q[m] prod_i Co[k_i][m_i],  Co[k][m] = Chebyshev coefficients of
//                       exp(-i (pi/3) k t),
//   translate in_T[k] = h^{2-d} 3^{-d} f(|k|) sum_S exp(-i (2 pi/3) k . delta_S) out_S[k],
//                       f(s) = (w-hat(pi s/3) - w-hat(2 pi s/3)) / (2 pi s/3)^2,
//   incoming  a[m]   += Re sum_k in[k] prod_i conj(Co[k_i][m_i]),
// and the tree passes are exact polynomial re-expansions with the triangular matrices
// S_b[M][m] (T_M((t -/+ 1)/2) in the basis T_m(t)).  Hermitian symmetry keeps k_0 >= 0.
//
// Passes: leaf moments -> merge (deepest level first) -> outgoing (all levels at once) ->
// translate+incoming (all levels at once) -> downward (root first) -> leaf evaluation.
#include <cuda_runtime.h>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <complex>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <cstring>
#include <type_traits>
#include <vector>

#include "k_leaf_tc.cuh"
#include "k_pw.cuh"
#include "kernels_common.cuh"
#include "pdmk.h"

namespace pdmk {

namespace {

template <typename T>
struct C2 {
    T x, y;
};
template <typename T>
__device__ __forceinline__ C2<T> cfma(C2<T> a, C2<T> b, C2<T> acc) {  // acc + a*b
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
template <typename T>
__device__ __forceinline__ C2<T> cfma_conj(C2<T> a, C2<T> b, C2<T> acc) {  // acc + conj(a)*b
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    return acc;
}

struct PwDims {
    int d, p, K, n1, np, pd1, npw, nk1;  // nk1 = n1^{d-1}
};

// ------------------------------------------------------------------ leaf moments
template <typename T, int D>
__global__ void __launch_bounds__(128) k_leaf_moments(const int4* __restrict__ leaves, const T* __restrict__ src4,
                                                      T* __restrict__ Q, PwDims pd, double inv_rc) {
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int kB = 32;
    T* basis = reinterpret_cast<T*>(sm);  // [kB][D][p]
    T* qv = basis + kB * D * pd.p;
    const int4 lf = leaves[blockIdx.x];
    const int p = pd.p;
    const T scale = T(2.0 * inv_rc * double(1LL << lf.w));  // t = 2 (y - c)/h
    T* Qb = Q + size_t(lf.z) * pd.np;
    for (int s0 = 0; s0 < lf.y; s0 += kB) {
        const int ns = min(kB, lf.y - s0);
        __syncthreads();
        for (int it = threadIdx.x; it < ns * D; it += blockDim.x) {
            const int s = it / D, i = it % D;
            const T* y = src4 + size_t(lf.x + s0 + s) * 4;
            const T t = y[i] * scale;
            T* b = basis + (s * D + i) * p;
            T tm1 = T(1), tm = t;
            b[0] = T(1);
            if (p > 1) b[1] = t;
            for (int m = 2; m < p; ++m) {
                const T tn = fma(T(2) * t, tm, -tm1);
                b[m] = tn;
                tm1 = tm;
                tm = tn;
            }
            if (i == 0) qv[s] = y[3];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < pd.np; e += blockDim.x) {
            int r = e;
            const int m_last = r % p;
            r /= p;
            const int m_mid = (D == 3) ? r % p : 0;
            if (D == 3) r /= p;
            const int m_first = r;
            T acc = T(0);
            for (int s = 0; s < ns; ++s) {
                const T* b = basis + s * D * p;
                T v = qv[s] * b[m_first] * b[(D - 1) * p + m_last];
                if (D == 3) v *= b[p + m_mid];
                acc += v;
            }
            Qb[e] += acc;
        }
    }
}

// 3D leaf moments as a small GEMM per leaf (the transpose of k_leaf_eval3d_gemm): one block of
// 256 threads per leaf, sources taken 16 at a time.  For a chunk, X[s][m0] = T_m0(t0_s) and
// B[s][m1 m2] = q_s T_m1(t1_s) T_m2(t2_s) are staged in shared memory (B formed by all threads,
// two products per element), and
//     Q[m0][m1 m2] += sum_s X[s][m0] B[s][m1 m2]          (P^3 multiply-adds per source)
// with a register tile of P/4 rows x P^2/64 columns per thread (columns strided by 64).
template <typename T, int P>
constexpr size_t leaf_moments3d_gemm_smem() {
    return sizeof(T) * (size_t(16) * P * P + size_t(16) * 3 * P + 16);
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_leaf_moments3d_gemm(const int4* __restrict__ leaves,
                                                             const T* __restrict__ src4, T* __restrict__ Q,
                                                             double inv_rc) {
    constexpr int PP = P * P, RT = P / 4, CT = PP / 64, NS = 16;
    static_assert(P % 4 == 0 && PP % 64 == 0, "tile split");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Bs = reinterpret_cast<T*>(smraw);  // [NS][PP]
    T* Tb = Bs + NS * PP;                 // [NS][3][P]  T_m of the three axes
    T* qv = Tb + NS * 3 * P;              // [NS]
    const int tid = threadIdx.x, rg = tid >> 6, cg = tid & 63;
    const int4 lf = leaves[blockIdx.x];   // (first source, count, q slot, level)
    const T scale = T(2.0 * inv_rc * double(1LL << lf.w));  // t = 2 (y - c)/h
    T acc[RT][CT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int k = 0; k < CT; ++k) acc[i][k] = T(0);
    for (int s0 = 0; s0 < lf.y; s0 += NS) {
        const int ns = min(NS, lf.y - s0);
        __syncthreads();  // the previous chunk's B and tables are consumed
        if (tid < 3 * NS) {
            const int sidx = tid / 3, ax = tid - 3 * sidx;
            T t = T(0), q = T(0);
            if (sidx < ns) {
                const T* y = src4 + size_t(lf.x + s0 + sidx) * 4;
                t = y[ax] * scale;
                q = y[3];
            }
            T* row = Tb + (sidx * 3 + ax) * P;
            T tm1 = T(1), tm = t;
            row[0] = T(1);
            row[1] = t;
#pragma unroll
            for (int m = 2; m < P; ++m) {
                const T tn = fma(T(2) * t, tm, -tm1);
                row[m] = tn;
                tm1 = tm;
                tm = tn;
            }
            if (ax == 0) qv[sidx] = q;  // zero for absent sources: their B rows vanish
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < (PP + 255) / 256; ++c) {
            const int col = tid + 256 * c;
            if (col < PP) {
                const int m1 = col / P, m2 = col - (col / P) * P;
#pragma unroll 4
                for (int sidx = 0; sidx < NS; ++sidx) {
                    const T* tr = Tb + sidx * 3 * P;
                    Bs[sidx * PP + col] = qv[sidx] * tr[P + m1] * tr[2 * P + m2];
                }
            }
        }
        __syncthreads();
#pragma unroll 2
        for (int sidx = 0; sidx < NS; ++sidx) {
            T xr[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) xr[i] = Tb[sidx * 3 * P + rg * RT + i];
            const T* brow = Bs + sidx * PP + cg;
#pragma unroll
            for (int k = 0; k < CT; ++k) {
                const T b = brow[64 * k];
#pragma unroll
                for (int i = 0; i < RT; ++i) acc[i][k] = fma(xr[i], b, acc[i][k]);
            }
        }
    }
    T* Qb = Q + size_t(lf.z) * (PP * P);
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int k = 0; k < CT; ++k) Qb[(rg * RT + i) * PP + cg + 64 * k] = acc[i][k];
}

// 3D leaf moments (FP32) with a three-way register tile: thread (a, b, c) owns
// Q[TA a + i][4 b + j][4 c + k], i < TA, j, k < 4.  Sources are taken 32 at a time; per chunk the
// rows q T_m0(t0), T_m1(t1), T_m2(t2) of every source are formed once in shared memory (thread
// per source and axis, the three-term recurrence), and per source a thread forms its 4 TA
// products of the first two rows and adds each times its four third-row values:
//     Q[m0][m1][m2] += (q T_m0(t0_s) T_m1(t1_s)) T_m2(t2_s)      (P^3 multiply-adds per source)
// with three 16-byte (or 8-byte) shared loads per source.  The chunk loop runs over the sources
// present only.
template <int P, int TA>
__global__ void __launch_bounds__((P / TA) * (P / 4) * (P / 4))
    k_leaf_moments3d_t(const int4* __restrict__ leaves, const float* __restrict__ src4, float* __restrict__ Q,
                       double inv_rc) {
    constexpr int NA = P / TA, NB = P / 4, NT = NA * NB * NB, PP = P * P, NS = 32;
    static_assert(P % 4 == 0 && P % TA == 0 && (TA == 2 || TA == 4), "tile split");
    __shared__ __align__(16) float Tt[NS][3][P];  // [source][axis][m]; the charge in the axis-0 row
    const int tid = threadIdx.x;
    const int c = tid % NB, b = (tid / NB) % NB, a = tid / (NB * NB);
    const int4 lf = leaves[blockIdx.x];  // (first source, count, q slot, level)
    const float scale = float(2.0 * inv_rc * double(1LL << lf.w));  // t = 2 (y - c)/h
    float acc[TA][4][4];
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    for (int s0 = 0; s0 < lf.y; s0 += NS) {
        const int ns = min(NS, lf.y - s0);
        __syncthreads();  // the previous chunk's rows are consumed
        for (int r = tid; r < 3 * ns; r += NT) {
            const int sidx = r / 3, ax = r - 3 * sidx;
            const float* y = src4 + size_t(lf.x + s0 + sidx) * 4;
            const float t = y[ax] * scale;
            const float f = ax == 0 ? y[3] : 1.f;
            float* row = &Tt[sidx][ax][0];
            float tm1 = 1.f, tm = t;
            row[0] = f;
            row[1] = f * t;
#pragma unroll
            for (int m = 2; m < P; ++m) {
                const float tn = fmaf(2.f * t, tm, -tm1);
                row[m] = f * tn;
                tm1 = tm;
                tm = tn;
            }
        }
        __syncthreads();
#pragma unroll 2
        for (int sidx = 0; sidx < ns; ++sidx) {
            float xv[TA];
            if constexpr (TA == 4) {
                const float4 x4 = *reinterpret_cast<const float4*>(&Tt[sidx][0][4 * a]);
                xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
            } else {
                const float2 x2 = *reinterpret_cast<const float2*>(&Tt[sidx][0][2 * a]);
                xv[0] = x2.x; xv[1] = x2.y;
            }
            const float4 y4 = *reinterpret_cast<const float4*>(&Tt[sidx][1][4 * b]);
            const float4 z4 = *reinterpret_cast<const float4*>(&Tt[sidx][2][4 * c]);
            const float yv[4] = {y4.x, y4.y, y4.z, y4.w}, zv[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
            for (int i = 0; i < TA; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float xy = xv[i] * yv[j];
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[i][j][k] = fmaf(xy, zv[k], acc[i][j][k]);
                }
        }
    }
    float* Qb = Q + size_t(lf.z) * (PP * P);
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(Qb + size_t(TA * a + i) * PP + (4 * b + j) * P + 4 * c) =
                make_float4(acc[i][j][0], acc[i][j][1], acc[i][j][2], acc[i][j][3]);
}

// ------------------------------------------------------------------ merge / downward
// Re-expansion of one box's Chebyshev array into another's, one axis at a time (slices of
// the first axis through shared memory).  mode 0 (merge): contract the child index m against
// the parent index M: Q_P[M] += sum_m Q_c[m] prod S_b[M_i][m_i].  mode 1 (down):
// a_c[m] += sum_M a_P[M] prod S_b[M_i][m_i].
template <typename T, int D>
__device__ void reexpand(const T* __restrict__ src, T* __restrict__ dst, int bits, int mode, const T* Sm,
                         T* s1, T* s2, const PwDims& pd) {
    const int p = pd.p, pd1 = pd.pd1;
    // S(b)[M][m] at Sm[(b * p + M) * p + m]
    auto S = [&](int b, int M, int m) { return Sm[(b * p + M) * p + m]; };
    const int b0 = bits & 1, b1 = (bits >> 1) & 1, b2 = (bits >> 2) & 1;
    for (int o0 = 0; o0 < p; ++o0) {
        // first axis: s1[r] = sum_j S(...) src[j * pd1 + r]
        for (int r = threadIdx.x; r < pd1; r += blockDim.x) {
            T acc = T(0);
            if (mode == 0) {
                for (int j = 0; j <= o0; ++j) acc = fma(S(b0, o0, j), src[j * pd1 + r], acc);
            } else {
                for (int j = o0; j < p; ++j) acc = fma(S(b0, j, o0), src[j * pd1 + r], acc);
            }
            s1[r] = acc;
        }
        __syncthreads();
        if (D == 2) {
            for (int o1 = threadIdx.x; o1 < p; o1 += blockDim.x) {
                T acc = T(0);
                if (mode == 0) {
                    for (int j = 0; j <= o1; ++j) acc = fma(S(b1, o1, j), s1[j], acc);
                } else {
                    for (int j = o1; j < p; ++j) acc = fma(S(b1, j, o1), s1[j], acc);
                }
                dst[o0 * p + o1] += acc;
            }
        } else {
            for (int it = threadIdx.x; it < p * p; it += blockDim.x) {
                const int o1 = it / p, j2 = it % p;
                T acc = T(0);
                if (mode == 0) {
                    for (int j = 0; j <= o1; ++j) acc = fma(S(b1, o1, j), s1[j * p + j2], acc);
                } else {
                    for (int j = o1; j < p; ++j) acc = fma(S(b1, j, o1), s1[j * p + j2], acc);
                }
                s2[it] = acc;
            }
            __syncthreads();
            for (int it = threadIdx.x; it < p * p; it += blockDim.x) {
                const int o1 = it / p, o2 = it % p;
                T acc = T(0);
                if (mode == 0) {
                    for (int j = 0; j <= o2; ++j) acc = fma(S(b2, o2, j), s2[o1 * p + j], acc);
                } else {
                    for (int j = o2; j < p; ++j) acc = fma(S(b2, j, o2), s2[o1 * p + j], acc);
                }
                dst[(o0 * p + o1) * p + o2] += acc;
            }
        }
        __syncthreads();
    }
}

// merge: one CTA per parent; list entry = [parent q slot, child q slots (2^d, -1 if empty)]
template <typename T, int D>
__global__ void __launch_bounds__(128) k_merge(const int* __restrict__ list, T* __restrict__ Q, const T* __restrict__ Sg,
                                               PwDims pd) {
    extern __shared__ __align__(16) unsigned char sm[];
    T* Sm = reinterpret_cast<T*>(sm);  // 2 p p
    T* s1 = Sm + 2 * pd.p * pd.p;      // pd1
    T* s2 = s1 + pd.pd1;               // p p
    for (int i = threadIdx.x; i < 2 * pd.p * pd.p; i += blockDim.x) Sm[i] = Sg[i];
    __syncthreads();
    const int* e = list + size_t(blockIdx.x) * (1 + (1 << D));
    T* dst = Q + size_t(e[0]) * pd.np;
    for (int c = 0; c < (1 << D); ++c) {
        const int cs = e[1 + c];
        if (cs < 0) continue;
        reexpand<T, D>(Q + size_t(cs) * pd.np, dst, c, 0, Sm, s1, s2, pd);
    }
}

// down: one CTA per parent; list entry = [parent local slot, child local slots (2^d, -1)]
template <typename T, int D>
__global__ void __launch_bounds__(128) k_down(const int* __restrict__ list, T* __restrict__ Lc, const T* __restrict__ Sg,
                                              PwDims pd) {
    extern __shared__ __align__(16) unsigned char sm[];
    T* Sm = reinterpret_cast<T*>(sm);
    T* s1 = Sm + 2 * pd.p * pd.p;
    T* s2 = s1 + pd.pd1;
    for (int i = threadIdx.x; i < 2 * pd.p * pd.p; i += blockDim.x) Sm[i] = Sg[i];
    __syncthreads();
    const int* e = list + size_t(blockIdx.x) * (1 + (1 << D));
    for (int c = 0; c < (1 << D); ++c) {
        const int cs = e[1 + c];
        if (cs < 0) continue;
        reexpand<T, D>(Lc + size_t(e[0]) * pd.np, Lc + size_t(cs) * pd.np, c, 1, Sm, s1, s2, pd);
    }
}

// 3D merge with a compile-time order P: one block of P^2 threads per parent, thread (i, j) <->
// the positions (M1, M2) or (m1, m2) of a P x P slice.  The sum over the eight children
// factors by axis (child c = (b0, b1, b2), bit k of c is b_k):
//   T_{b0 b1}[m1][M2] = sum_{b2, m2} S_b2[M2][m2] Q_c[m0][m1][m2]       (slice m0)
//   U_{b0}[M1][M2]    = sum_{b1, m1} S_b1[M1][m1] T_{b0 b1}[m1][M2]
//   Q_P[M0][M1][M2]  += sum_{b0} S_b0[M0][m0] U_{b0}[M1][M2]           (registers)
// 14 P^4 multiply-adds per parent (a child-by-child separable re-expansion takes 24 P^4).
// S is stored as Sm[b][M][m] and transposed as St[b][m][M] (lanes along the contiguous index).
// Levels with fewer parents than SMs take the four-way k_merge3d_q below; the downward pass
// always runs four ways (k_down3d_q).
template <typename T, int P>
__global__ void __launch_bounds__(P * P, sizeof(T) == 4 ? 2 : 1) k_merge3d_p(const int* __restrict__ list, T* __restrict__ Q,
                                                     const T* __restrict__ Sg) {
    constexpr int PP = P * P, NP = PP * P;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Sm = reinterpret_cast<T*>(smraw);  // [2][P][P]
    T* St = Sm + 2 * PP;                  // [2][P][P] transposed
    T* in = St + 2 * PP;                  // [8][PP] child slices m0
    T* Ts = in + 8 * PP;                  // [4][PP]
    T* Us = Ts + 4 * PP;                  // [2][PP]
    const int tid = threadIdx.x, i = tid / P, j = tid % P;
    for (int k = tid; k < 2 * PP; k += blockDim.x) {
        const T v = Sg[k];
        Sm[k] = v;
        const int b = k / PP, M = (k / P) % P, m = k % P;
        St[(b * P + m) * P + M] = v;
    }
    const int* e = list + size_t(blockIdx.x) * 9;
    int cs[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) cs[c] = e[1 + c];
    T acc[P];
#pragma unroll
    for (int M0 = 0; M0 < P; ++M0) acc[M0] = T(0);
    for (int m0 = 0; m0 < P; ++m0) {
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 8; ++c) in[c * PP + tid] = cs[c] >= 0 ? Q[size_t(cs[c]) * NP + size_t(m0) * PP + tid] : T(0);
        __syncthreads();
        // T_{b0b1}[m1 = i][M2 = j]
        {
            T t4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
                for (int m2 = 0; m2 < P; ++m2) {
                    const T s = St[(b2 * P + m2) * P + j];
#pragma unroll
                    for (int k = 0; k < 4; ++k) t4[k] = fma(s, in[((b2 << 2) | k) * PP + i * P + m2], t4[k]);
                }
#pragma unroll
            for (int k = 0; k < 4; ++k) Ts[k * PP + tid] = t4[k];
        }
        __syncthreads();
        // U_{b0}[M1 = i][M2 = j]
        {
            T u0 = T(0), u1 = T(0);
#pragma unroll
            for (int b1 = 0; b1 < 2; ++b1)
#pragma unroll
                for (int m1 = 0; m1 < P; ++m1) {
                    const T s = Sm[(b1 * P + i) * P + m1];
                    u0 = fma(s, Ts[((b1 << 1) | 0) * PP + m1 * P + j], u0);
                    u1 = fma(s, Ts[((b1 << 1) | 1) * PP + m1 * P + j], u1);
                }
            // Q_P[M0][i][j] += S_0[M0][m0] U_0 + S_1[M0][m0] U_1
#pragma unroll
            for (int M0 = 0; M0 < P; ++M0)
                acc[M0] = fma(Sm[M0 * P + m0], u0, fma(Sm[(P + M0) * P + m0], u1, acc[M0]));
        }
    }
    T* dst = Q + size_t(e[0]) * NP;
#pragma unroll
    for (int M0 = 0; M0 < P; ++M0) dst[size_t(M0) * PP + tid] = acc[M0];
}

// 3D re-expansions split four ways per parent, by the children's first two axis bits
// q = b0 | b1 << 1 (child c = b0 | b1 << 1 | b2 << 2): a block of P^2 threads, thread
// (i, j) <-> positions (M1, M2) or (m1, m2) of a P x P slice, as in k_merge3d_p.
// A parent's work is spread over four blocks instead of one: 16 P^4 multiply-adds instead of
// 14 P^4, for four times the blocks, which the small upper levels of a deep tree need (one
// block per parent left most SMs idle and made every level cost one block's latency).
//   down:  V[M1][M2] = sum_{M0} S_b0[M0][m0] a_P[M0][M1][M2]          (slice m0)
//          W[m1][M2] = sum_{M1} S_b1[M1][m1] V[M1][M2]
//          a_c[m0][m1][m2] += sum_{M2} S_b2[M2][m2] W[m1][M2]        (b2 = 0, 1: two children)
//   merge: T[m1][M2] = sum_{b2, m2} S_b2[M2][m2] Q_c[m0][m1][m2]       (slice m0, two children)
//          U[M1][M2] = sum_{m1} S_b1[M1][m1] T[m1][M2]
//          part_q[M0][M1][M2] += S_b0[M0][m0] U[M1][M2]              (registers)
//          the block that completes a parent adds its four parts in the order q = 0..3.
template <typename T, int P>
__global__ void __launch_bounds__(P * P) k_down3d_q(const int* __restrict__ list, T* __restrict__ Lc,
                                                    const T* __restrict__ Sg) {
    constexpr int PP = P * P, NP = PP * P;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Sm = reinterpret_cast<T*>(smraw);  // [2][P][P]  S[b][M][m]
    T* aP = Sm + 2 * PP;                  // [P][PP]   parent coefficients
    T* Vs = aP + NP;                      // [PP]
    T* Ws = Vs + PP;                      // [PP]
    const int tid = threadIdx.x, i = tid / P, j = tid % P;
    const int q = blockIdx.x & 3, b0 = q & 1, b1 = q >> 1;
    const int* e = list + size_t(blockIdx.x >> 2) * 9;
    const int c0 = e[1 + q], c1 = e[1 + (q | 4)];
    if (c0 < 0 && c1 < 0) return;  // whole block: no child of this quadrant has targets
    for (int k = tid; k < 2 * PP; k += blockDim.x) Sm[k] = Sg[k];
    const T* src = Lc + size_t(e[0]) * NP;
    for (int k = tid; k < NP; k += blockDim.x) aP[k] = src[k];
    const T* S0 = Sm + b0 * PP;  // S_b0[M][m]
    const T* S1 = Sm + b1 * PP;  // S_b1[M][m]
    for (int m0 = 0; m0 < P; ++m0) {
        __syncthreads();
        {
            T v = T(0);
#pragma unroll
            for (int M0 = 0; M0 < P; ++M0) v = fma(S0[M0 * P + m0], aP[M0 * PP + tid], v);
            Vs[tid] = v;
        }
        __syncthreads();
        {
            T w = T(0);
#pragma unroll
            for (int M1 = 0; M1 < P; ++M1) w = fma(S1[M1 * P + i], Vs[M1 * P + j], w);
            Ws[tid] = w;
        }
        __syncthreads();
        T o0 = T(0), o1 = T(0);
#pragma unroll
        for (int M2 = 0; M2 < P; ++M2) {
            const T wv = Ws[i * P + M2];
            o0 = fma(Sm[M2 * P + j], wv, o0);
            o1 = fma(Sm[PP + M2 * P + j], wv, o1);
        }
        if (c0 >= 0) Lc[size_t(c0) * NP + size_t(m0) * PP + tid] += o0;
        if (c1 >= 0) Lc[size_t(c1) * NP + size_t(m0) * PP + tid] += o1;
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(P * P) k_merge3d_q(const int* __restrict__ list, T* __restrict__ Q,
                                                     const T* __restrict__ Sg, T* __restrict__ part,
                                                     int* __restrict__ done) {
    constexpr int PP = P * P, NP = PP * P;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Sm = reinterpret_cast<T*>(smraw);  // [2][P][P]  S[b][M][m]
    T* St = Sm + 2 * PP;                  // [2][P][P]  transposed: St[b][m][M]
    T* in = St + 2 * PP;                  // [2][PP]    the two children's slice m0
    T* Ts = in + 2 * PP;                  // [PP]
    __shared__ int s_last;
    const int tid = threadIdx.x, i = tid / P, j = tid % P;
    const int q = blockIdx.x & 3, b0 = q & 1, b1 = q >> 1;
    const int ent = blockIdx.x >> 2;
    const int* e = list + size_t(ent) * 9;
    const int c0 = e[1 + q], c1 = e[1 + (q | 4)];
    for (int k = tid; k < 2 * PP; k += blockDim.x) {
        const T v = Sg[k];
        Sm[k] = v;
        const int b = k / PP, M = (k / P) % P, m = k % P;
        St[(b * P + m) * P + M] = v;
    }
    T acc[P];
#pragma unroll
    for (int M0 = 0; M0 < P; ++M0) acc[M0] = T(0);
    if (c0 >= 0 || c1 >= 0) {  // block-uniform
        for (int m0 = 0; m0 < P; ++m0) {
            __syncthreads();
            in[tid] = c0 >= 0 ? Q[size_t(c0) * NP + size_t(m0) * PP + tid] : T(0);
            in[PP + tid] = c1 >= 0 ? Q[size_t(c1) * NP + size_t(m0) * PP + tid] : T(0);
            __syncthreads();
            {
                T t = T(0);
#pragma unroll
                for (int m2 = 0; m2 < P; ++m2) {
                    t = fma(St[m2 * P + j], in[i * P + m2], t);
                    t = fma(St[PP + m2 * P + j], in[PP + i * P + m2], t);
                }
                Ts[tid] = t;
            }
            __syncthreads();
            T u = T(0);
#pragma unroll
            for (int m1 = 0; m1 < P; ++m1) u = fma(Sm[(b1 * P + i) * P + m1], Ts[m1 * P + j], u);
#pragma unroll
            for (int M0 = 0; M0 < P; ++M0) acc[M0] = fma(Sm[(b0 * P + M0) * P + m0], u, acc[M0]);
        }
    }
    T* mine = part + (size_t(ent) * 4 + q) * NP;
#pragma unroll
    for (int M0 = 0; M0 < P; ++M0) mine[size_t(M0) * PP + tid] = acc[M0];
    // the block that completes the parent adds the four parts in a fixed order (the counter
    // only decides which block does it) and resets the counter for the next evaluation
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(done + ent, 1) == 3;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const T* p0 = part + size_t(ent) * 4 * NP;
    T* dst = Q + size_t(e[0]) * NP;
    for (int k = tid; k < NP; k += blockDim.x) {
        T v = __ldcg(p0 + k);
        v += __ldcg(p0 + NP + k);
        v += __ldcg(p0 + 2 * NP + k);
        v += __ldcg(p0 + 3 * NP + k);
        dst[k] = v;
    }
    if (tid == 0) done[ent] = 0;
}

// ------------------------------------------------------------------------------------------
// 3D re-expansions with register accumulators and the triangular shift matrices.
// S_b[M][m] (coefficient of T_m in T_M((t -/+ 1)/2)) vanishes for m > M, so every axis
// contraction below runs over the lower triangle only: 7 P^4 multiply-adds per parent in all
// (the full separable form takes 14 P^4).  A thread owns one P x P slice position and keeps P
// accumulators in registers; the contracted operand is one shared (or coalesced global) load
// per P/2 multiply-adds on average, and the matrix rows are read as broadcast vectors.
template <typename T>
struct VecOf;
template <>
struct VecOf<float> { using V = float4; static constexpr int W = 4; };
template <>
struct VecOf<double> { using V = double2; static constexpr int W = 2; };

// component jj of a vector (jj compile-time after unrolling)
__device__ __forceinline__ float vlane(const float4& v, int jj) { return jj == 0 ? v.x : jj == 1 ? v.y : jj == 2 ? v.z : v.w; }
__device__ __forceinline__ double vlane(const double2& v, int jj) { return jj == 0 ? v.x : v.y; }

// The shift matrices S_b[M][m] (index (b p + M) p + m) of the register-tiled 3D orders in
// constant memory.  They depend on p alone; with compile-time indices the re-expansions'
// multiply-adds take them as constant operands, with no shared-memory loads.
__constant__ float c_shift_f16[2 * 16 * 16];
__constant__ float c_shift_f24[2 * 24 * 24];
__constant__ double c_shift_d16[2 * 16 * 16];
template <typename T, int P>
__device__ __forceinline__ T shiftc(int i);
template <>
__device__ __forceinline__ float shiftc<float, 16>(int i) { return c_shift_f16[i]; }
template <>
__device__ __forceinline__ float shiftc<float, 24>(int i) { return c_shift_f24[i]; }
template <>
__device__ __forceinline__ double shiftc<double, 16>(int i) { return c_shift_d16[i]; }
// merge: acc[M] += S_b[M][m] x for M in [m, P)      (b, m compile-time after unrolling)
template <typename T, int P>
__device__ __forceinline__ void tri_merge_c(T (&acc)[P], int b, int m, T x) {
#pragma unroll
    for (int M = 0; M < P; ++M)
        if (M >= m) acc[M] = fma(shiftc<T, P>((b * P + M) * P + m), x, acc[M]);
}
// downward: acc[m] += S_b[M][m] x for m in [0, M]   (b, M compile-time after unrolling)
template <typename T, int P>
__device__ __forceinline__ void tri_down_c(T (&acc)[P], int b, int M, T x) {
#pragma unroll
    for (int m = 0; m < P; ++m)
        if (m <= M) acc[m] = fma(shiftc<T, P>((b * P + M) * P + m), x, acc[m]);
}


// downward pass, two blocks per parent (one per first-axis child bit b0):
//   V[m0][M1 M2]  = sum_{M0 >= m0} S_b0[M0][m0] a_P[M0][M1 M2]      thread (M1 M2)
//   W[m0][m1 M2]  = sum_{M1 >= m1} S_b1[M1][m1] V[m0][M1 M2]        thread (m0 M2), per b1
//   a_c[m0 m1][m2] += sum_{M2 >= m2} S_b2[M2][m2] W[m0 m1][M2]      thread (m0 m1), per b2
// The child's coefficients are added to those its own incoming waves wrote (in-boxes,
// add[c] = 1) or written (leaves, whose only contribution this is), so the local array needs
// no clearing.
template <typename T, int P>
__global__ void __launch_bounds__(P * P) k_down3d_r(const int* __restrict__ list, T* __restrict__ Lc,
                                                    const unsigned char* __restrict__ add) {
    constexpr int PP = P * P, NP = PP * P;
    using V = typename VecOf<T>::V;
    constexpr int VW = VecOf<T>::W;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Vs = reinterpret_cast<T*>(smraw);  // [P][PP]
    T* Ws = Vs + NP;                      // [P][PP]
    const int tid = threadIdx.x, b0 = blockIdx.x & 1;
    const int* e = list + size_t(blockIdx.x >> 1) * 9;
    int ch[2][2];
#pragma unroll
    for (int b1 = 0; b1 < 2; ++b1)
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2) ch[b1][b2] = e[1 + (b0 | (b1 << 1) | (b2 << 2))];
    if (ch[0][0] < 0 && ch[0][1] < 0 && ch[1][0] < 0 && ch[1][1] < 0) return;  // block-uniform
    {
        const T* aP = Lc + size_t(e[0]) * NP;
        T v[P];
#pragma unroll
        for (int m = 0; m < P; ++m) v[m] = T(0);
        if (b0 == 0) {
#pragma unroll
            for (int M0 = 0; M0 < P; ++M0) tri_down_c<T, P>(v, 0, M0, aP[M0 * PP + tid]);
        } else {
#pragma unroll
            for (int M0 = 0; M0 < P; ++M0) tri_down_c<T, P>(v, 1, M0, aP[M0 * PP + tid]);
        }
#pragma unroll
        for (int m0 = 0; m0 < P; ++m0) Vs[m0 * PP + tid] = v[m0];
    }
    __syncthreads();
    const int i = tid / P, j = tid - (tid / P) * P;
#pragma unroll
    for (int b1 = 0; b1 < 2; ++b1) {
        if (ch[b1][0] < 0 && ch[b1][1] < 0) continue;  // block-uniform
        {
            // thread (m0 = i, M2 = j)
            T w[P];
#pragma unroll
            for (int m = 0; m < P; ++m) w[m] = T(0);
#pragma unroll
            for (int M1 = 0; M1 < P; ++M1) tri_down_c<T, P>(w, b1, M1, Vs[i * PP + M1 * P + j]);
#pragma unroll
            for (int m1 = 0; m1 < P; ++m1) Ws[i * PP + m1 * P + j] = w[m1];
        }
        __syncthreads();
        {
            // thread (m0 m1) = tid: its W row over M2
            T wr[P];
#pragma unroll
            for (int k = 0; k < P / VW; ++k) {
                const V v = reinterpret_cast<const V*>(Ws + tid * P)[k];
#pragma unroll
                for (int jj = 0; jj < VW; ++jj) wr[VW * k + jj] = reinterpret_cast<const T*>(&v)[jj];
            }
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2) {
                const int c = ch[b1][b2];
                if (c < 0) continue;
                T o[P];
#pragma unroll
                for (int m = 0; m < P; ++m) o[m] = T(0);
#pragma unroll
                for (int M2 = 0; M2 < P; ++M2) tri_down_c<T, P>(o, b2, M2, wr[M2]);
                V* dst = reinterpret_cast<V*>(Lc + size_t(c) * NP + size_t(tid) * P);
                if (add[c]) {
#pragma unroll
                    for (int k = 0; k < P / VW; ++k) {
                        V d = dst[k];
                        T* dd = reinterpret_cast<T*>(&d);
#pragma unroll
                        for (int jj = 0; jj < VW; ++jj) dd[jj] += o[VW * k + jj];
                        dst[k] = d;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < P / VW; ++k) {
                        V d;
                        T* dd = reinterpret_cast<T*>(&d);
#pragma unroll
                        for (int jj = 0; jj < VW; ++jj) dd[jj] = o[VW * k + jj];
                        dst[k] = d;
                    }
                }
            }
        }
        __syncthreads();  // W is rewritten for the next b1
    }
}

// upward merge, one block per parent, two P^3 buffers A, B in shared memory, per half b0:
//   U_{b0 b1}[m0 m1][M2] = sum_{b2} sum_{m2 <= M2} S_b2[M2][m2] Q_c[m0 m1][m2]   thread (m0 m1)
//   V_{b0}[m0][M1 M2]    = sum_{b1} sum_{m1 <= M1} S_b1[M1][m1] U_{b0 b1}[m0][m1 M2]   thread (m0 M2)
//   Q_P[M0][M1 M2]      += sum_{m0 <= M0} S_b0[M0][m0] V_{b0}[m0][M1 M2]         thread (M1 M2)
// U_{b0 b1} sits in buffer b1; V_{b0} overwrites U_{b0 0} in place (a thread rewrites exactly
// the (m0, M2) slice it read).  The first half present writes the parent's moments, the
// second adds to them (each thread its own elements), so two buffers suffice and FP32 order
// 24 runs two blocks per SM.
template <typename T, int P>
__global__ void __launch_bounds__(P * P, (sizeof(T) == 4 && P == 24) ? 2 : 1)
    k_merge3d_r(const int* __restrict__ list, T* __restrict__ Q) {
    constexpr int PP = P * P, NP = PP * P;
    using V = typename VecOf<T>::V;
    constexpr int VW = VecOf<T>::W;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* buf = reinterpret_cast<T*>(smraw);  // [2][NP]
    const int tid = threadIdx.x, i = tid / P, j = tid - (tid / P) * P;
    const int* e = list + size_t(blockIdx.x) * 9;
    // children present per quarter (b0, b1) and per half b0: absent quarters and halves are
    // skipped (block-uniform)
    int qmask = 0;  // bit 2 b0 + b1: quarter (b0, b1) has a child
#pragma unroll
    for (int b0 = 0; b0 < 2; ++b0)
#pragma unroll
        for (int b1 = 0; b1 < 2; ++b1)
            if (e[1 + (b0 | (b1 << 1))] >= 0 || e[1 + (b0 | (b1 << 1) | 4)] >= 0) qmask |= 1 << (2 * b0 + b1);
    auto quarter = [&](int b0, int b1) { return (qmask >> (2 * b0 + b1)) & 1; };
    auto half = [&](int b0) { return (qmask >> (2 * b0)) & 3; };
    T* dst = Q + size_t(e[0]) * NP;
    bool first = true;
#pragma unroll 1
    for (int b0 = 0; b0 < 2; ++b0) {
        if (!half(b0)) continue;
        // U_{b0 b1} in buffer b1
#pragma unroll 1
        for (int b1 = 0; b1 < 2; ++b1) {
            if (!quarter(b0, b1)) continue;
            // thread (m0 m1) = tid
            T u[P];
#pragma unroll
            for (int m = 0; m < P; ++m) u[m] = T(0);
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2) {
                const int c = e[1 + (b0 | (b1 << 1) | (b2 << 2))];
                if (c < 0) continue;  // absent child
                V cur[P / VW];
                const V* qrow = reinterpret_cast<const V*>(Q + size_t(c) * NP + size_t(tid) * P);
#pragma unroll
                for (int k = 0; k < P / VW; ++k) cur[k] = __ldg(qrow + k);
#pragma unroll
                for (int k = 0; k < P / VW; ++k) {
#pragma unroll
                    for (int jj = 0; jj < VW; ++jj) {
                        const int m2 = VW * k + jj;
                        tri_merge_c<T, P>(u, b2, m2, vlane(cur[k], jj));
                    }
                }
            }
            V* ud = reinterpret_cast<V*>((buf + size_t(b1) * NP) + size_t(tid) * P);
#pragma unroll
            for (int k = 0; k < P / VW; ++k) {
                V v;
#pragma unroll
                for (int jj = 0; jj < VW; ++jj) reinterpret_cast<T*>(&v)[jj] = u[VW * k + jj];
                ud[k] = v;
            }
        }
        __syncthreads();
        {
            // thread (m0 = i, M2 = j)
            T v[P];
#pragma unroll
            for (int m = 0; m < P; ++m) v[m] = T(0);
#pragma unroll
            for (int b1 = 0; b1 < 2; ++b1) {
                if (!quarter(b0, b1)) continue;
#pragma unroll
                for (int m1 = 0; m1 < P; ++m1)
                    tri_merge_c<T, P>(v, b1, m1, (buf + size_t(b1) * NP)[i * PP + m1 * P + j]);
            }
#pragma unroll
            for (int M1 = 0; M1 < P; ++M1) buf[i * PP + M1 * P + j] = v[M1];
        }
        __syncthreads();
        {
            // thread (M1 M2) = tid
            T q[P];
#pragma unroll
            for (int m = 0; m < P; ++m) q[m] = T(0);
            if (b0 == 0) {
#pragma unroll
                for (int m0 = 0; m0 < P; ++m0) tri_merge_c<T, P>(q, 0, m0, buf[m0 * PP + tid]);
            } else {
#pragma unroll
                for (int m0 = 0; m0 < P; ++m0) tri_merge_c<T, P>(q, 1, m0, buf[m0 * PP + tid]);
            }
            if (first) {
#pragma unroll
                for (int M0 = 0; M0 < P; ++M0) dst[size_t(M0) * PP + tid] = q[M0];
            } else {
#pragma unroll
                for (int M0 = 0; M0 < P; ++M0) dst[size_t(M0) * PP + tid] += q[M0];
            }
        }
        first = false;
        __syncthreads();  // the buffers are rewritten by the next half
    }
}

// 2D: the whole re-expansion of all children in two shared-memory phases per parent.
// merge: Q_P[M0][M1] = sum_c sum_{m0<=M0} S_{b0}[M0][m0] sum_{m1<=M1} S_{b1}[M1][m1] Q_c[m0][m1]
template <typename T>
__device__ void merge2d_body(const int* __restrict__ e, T* __restrict__ Q, const T* Sm, T* qc, T* tm,
                             const PwDims& pd) {
    const int p = pd.p, pp = p * p;
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * pp; i += blockDim.x) {
        const int c = i / pp, r = i % pp, cs = e[1 + c];
        qc[i] = cs >= 0 ? Q[size_t(cs) * pd.np + r] : T(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * pp; i += blockDim.x) {
        const int c = i / pp, r = i % pp, m0 = r / p, M1 = r % p, b1 = (c >> 1) & 1;
        const T* S = Sm + (b1 * p + M1) * p;
        const T* q = qc + c * pp + m0 * p;
        T acc = T(0);
        for (int m1 = 0; m1 <= M1; ++m1) acc = fma(S[m1], q[m1], acc);
        tm[i] = acc;
    }
    __syncthreads();
    T* dst = Q + size_t(e[0]) * pd.np;
    for (int r = threadIdx.x; r < pp; r += blockDim.x) {
        const int M0 = r / p, M1 = r % p;
        T acc = T(0);
        for (int c = 0; c < 4; ++c) {
            if (e[1 + c] < 0) continue;
            const T* S = Sm + ((c & 1) * p + M0) * p;
            const T* t = tm + c * pp + M1;
            for (int m0 = 0; m0 <= M0; ++m0) acc = fma(S[m0], t[m0 * p], acc);
        }
        dst[r] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_merge2d(const int* __restrict__ list, T* __restrict__ Q,
                                                 const T* __restrict__ Sg, PwDims pd) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int pp = pd.p * pd.p;
    T* Sm = reinterpret_cast<T*>(sm);  // [2][p][p]
    for (int i = threadIdx.x; i < 2 * pp; i += blockDim.x) Sm[i] = Sg[i];
    merge2d_body<T>(list + size_t(blockIdx.x) * 5, Q, Sm, Sm + 2 * pp, Sm + 6 * pp, pd);
}

// down: a_c[m0][m1] += sum_{M0>=m0} S_{b0}[M0][m0] sum_{M1>=m1} S_{b1}[M1][m1] a_P[M0][M1]
template <typename T>
__device__ void down2d_body(const int* __restrict__ e, T* __restrict__ Lc, const T* Sm, T* ap, T* tm,
                            const PwDims& pd) {
    const int p = pd.p, pp = p * p;
    const T* src = Lc + size_t(e[0]) * pd.np;
    __syncthreads();
    for (int i = threadIdx.x; i < pp; i += blockDim.x) ap[i] = src[i];
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * pp; i += blockDim.x) {
        const int b1 = i / pp, r = i % pp, M0 = r / p, m1 = r % p;
        T acc = T(0);
        for (int M1 = m1; M1 < p; ++M1) acc = fma(Sm[(b1 * p + M1) * p + m1], ap[M0 * p + M1], acc);
        tm[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * pp; i += blockDim.x) {
        const int c = i / pp, r = i % pp, cs = e[1 + c];
        if (cs < 0) continue;
        const int m0 = r / p, m1 = r % p, b0 = c & 1, b1 = (c >> 1) & 1;
        T acc = T(0);
        for (int M0 = m0; M0 < p; ++M0) acc = fma(Sm[(b0 * p + M0) * p + m0], tm[b1 * pp + M0 * p + m1], acc);
        Lc[size_t(cs) * pd.np + r] += acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_down2d(const int* __restrict__ list, T* __restrict__ Lc,
                                                const T* __restrict__ Sg, PwDims pd) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int pp = pd.p * pd.p;
    T* Sm = reinterpret_cast<T*>(sm);  // [2][p][p]
    for (int i = threadIdx.x; i < 2 * pp; i += blockDim.x) Sm[i] = Sg[i];
    down2d_body<T>(list + size_t(blockIdx.x) * 5, Lc, Sm, Sm + 2 * pp, Sm + 3 * pp, pd);
}

// 2D re-expansions with a compile-time order P: register tiles of 4 outputs per thread and
// fully unrolled contractions (the triangular zeros of S are multiplied through: regular
// loops beat the saved flops at this size).
//   merge: R_b0[m0][M1] = sum_{b1,m1} S_b1[M1][m1] Q_(b0,b1)[m0][m1];
//          Q_P[M0][M1]  = sum_{b0,m0} S_b0[M0][m0] R_b0[m0][M1]
//   down:  U_b1[M0][m1] = sum_{M1} S_b1[M1][m1] a_P[M0][M1];
//          a_(b0,b1)[m0][m1] += sum_{M0} S_b0[M0][m0] U_b1[M0][m1]
template <typename T, int P>
__global__ void __launch_bounds__(256) k_merge2d_p(const int* __restrict__ list, T* __restrict__ Q,
                                                   const T* __restrict__ Sg, int np) {
    constexpr int PP = P * P, G = (P + 3) / 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Sm = reinterpret_cast<T*>(smraw);  // S[b][M][m]  [2 PP]
    T* St = Sm + 2 * PP;                  // S[b][m][M]  [2 PP] (transposed)
    T* qc = St + 2 * PP;                  // [4 PP]
    T* R = qc + 4 * PP;                   // [2 PP]
    const int* e = list + size_t(blockIdx.x) * 5;
    for (int i = threadIdx.x; i < 2 * PP; i += blockDim.x) {
        const T v = Sg[i];
        Sm[i] = v;
        const int b = i / PP, M = (i / P) % P, m = i % P;
        St[(b * P + m) * P + M] = v;
    }
    for (int i = threadIdx.x; i < 4 * PP; i += blockDim.x) {
        const int c = i / PP, cs = e[1 + c];
        qc[i] = cs >= 0 ? Q[size_t(cs) * np + (i % PP)] : T(0);
    }
    __syncthreads();
    // phase A: lanes along M1 (St column reads are contiguous, q values are broadcasts)
    for (int it = threadIdx.x; it < 2 * G * P; it += blockDim.x) {
        const int b0 = it / (G * P), rem = it % (G * P), g = rem / P, M1 = rem % P;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int b1 = 0; b1 < 2; ++b1) {
            const T* q = qc + ((b1 << 1) | b0) * PP;
#pragma unroll
            for (int m1 = 0; m1 < P; ++m1) {
                const T s = St[(b1 * P + m1) * P + M1];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m0 = g * 4 + j;
                    if (m0 < P) acc[j] = fma(s, q[m0 * P + m1], acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m0 = g * 4 + j;
            if (m0 < P) R[b0 * PP + m0 * P + M1] = acc[j];
        }
    }
    __syncthreads();
    // phase B: lanes along M1 (R rows contiguous, S values broadcasts)
    T* dst = Q + size_t(e[0]) * np;
    for (int it = threadIdx.x; it < G * P; it += blockDim.x) {
        const int g = it / P, M1 = it % P;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int b0 = 0; b0 < 2; ++b0) {
#pragma unroll
            for (int m0 = 0; m0 < P; ++m0) {
                const T r = R[b0 * PP + m0 * P + M1];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int M0 = g * 4 + j;
                    if (M0 < P) acc[j] = fma(Sm[(b0 * P + M0) * P + m0], r, acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int M0 = g * 4 + j;
            if (M0 < P) dst[M0 * P + M1] = acc[j];
        }
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_down2d_p(const int* __restrict__ list, T* __restrict__ Lc,
                                                  const T* __restrict__ Sg, int np) {
    constexpr int PP = P * P, G = (P + 3) / 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Sm = reinterpret_cast<T*>(smraw);  // [2 PP] | ap [PP] | U [2 PP]
    T* ap = Sm + 2 * PP;
    T* U = ap + PP;
    const int* e = list + size_t(blockIdx.x) * 5;
    const T* src = Lc + size_t(e[0]) * np;
    for (int i = threadIdx.x; i < 2 * PP; i += blockDim.x) Sm[i] = Sg[i];
    for (int i = threadIdx.x; i < PP; i += blockDim.x) ap[i] = src[i];
    __syncthreads();
    // phase A: lanes along m1 (S rows contiguous, a_P values broadcasts)
    for (int it = threadIdx.x; it < 2 * G * P; it += blockDim.x) {
        const int b1 = it / (G * P), rem = it % (G * P), g = rem / P, m1 = rem % P;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int M1 = 0; M1 < P; ++M1) {
            const T s = Sm[(b1 * P + M1) * P + m1];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int M0 = g * 4 + j;
                if (M0 < P) acc[j] = fma(s, ap[M0 * P + M1], acc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int M0 = g * 4 + j;
            if (M0 < P) U[b1 * PP + M0 * P + m1] = acc[j];
        }
    }
    __syncthreads();
    // phase B: lanes along m1 (U rows contiguous, S values broadcasts)
    for (int it = threadIdx.x; it < 4 * G * P; it += blockDim.x) {
        const int c = it / (G * P), rem = it % (G * P), g = rem / P, m1 = rem % P;
        const int cs = e[1 + c];
        if (cs < 0) continue;
        const int b0 = c & 1, b1 = c >> 1;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int M0 = 0; M0 < P; ++M0) {
            const T u = U[b1 * PP + M0 * P + m1];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m0 = g * 4 + j;
                if (m0 < P) acc[j] = fma(Sm[(b0 * P + M0) * P + m0], u, acc[j]);
            }
        }
        T* dst = Lc + size_t(cs) * np;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m0 = g * 4 + j;
            if (m0 < P) dst[m0 * P + m1] += acc[j];
        }
    }
}

// ------------------------------------------------------------------ outgoing plane waves
// entry int2 = (q slot, out slot); out layout [k0 in 0..K][k1 in -K..K][k2 in -K..K]
template <typename T, int D>
__global__ void __launch_bounds__(128) k_pw_out(const int2* __restrict__ list, const T* __restrict__ Q,
                                                C2<T>* __restrict__ out, const C2<T>* __restrict__ Cog, PwDims pd, int KC) {
    extern __shared__ __align__(16) unsigned char sm[];
    C2<T>* Co = reinterpret_cast<C2<T>*>(sm);  // [n1][p], row kk = k + K
    C2<T>* A = Co + pd.n1 * pd.p;              // [KC][pd1]
    C2<T>* B = A + KC * pd.pd1;                // [n1][p]   (3D)
    C2<T>* CoT = B + pd.n1 * pd.p;             // [p][n1]   transposed copy (lanes along k)
    const int p = pd.p, K = pd.K, n1 = pd.n1, pd1 = pd.pd1;
    for (int i = threadIdx.x; i < n1 * p; i += blockDim.x) {
        const C2<T> v = Cog[i];
        Co[i] = v;
        CoT[(i % p) * n1 + i / p] = v;
    }
    __syncthreads();
    const int2 e = list[blockIdx.x];
    const T* q = Q + size_t(e.x) * pd.np;
    C2<T>* o = out + size_t(e.y) * pd.npw;
    for (int kc0 = 0; kc0 <= K; kc0 += KC) {
        const int nk = min(KC, K + 1 - kc0);
        if (D == 2) {
            // 2D: one item per (k0, r); p-term dot products
            for (int it = threadIdx.x; it < nk * pd1; it += blockDim.x) {
                const int j = it / pd1, r = it % pd1;
                C2<T> acc{T(0), T(0)};
                const C2<T>* crow = Co + (kc0 + j + K) * p;
                for (int m0 = 0; m0 < p; ++m0) {
                    const T v = q[m0 * pd1 + r];
                    acc.x = fma(crow[m0].x, v, acc.x);
                    acc.y = fma(crow[m0].y, v, acc.y);
                }
                A[j * pd1 + r] = acc;
            }
        } else
        for (int r = threadIdx.x; r < pd1; r += blockDim.x) {
            C2<T> acc[16];
            for (int j = 0; j < 16; ++j) acc[j] = C2<T>{T(0), T(0)};
            for (int m0 = 0; m0 < p; ++m0) {
                const T v = q[m0 * pd1 + r];
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < nk) {
                        const C2<T> c = Co[(kc0 + j + K) * p + m0];
                        acc[j].x = fma(c.x, v, acc[j].x);
                        acc[j].y = fma(c.y, v, acc[j].y);
                    }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < nk) A[j * pd1 + r] = acc[j];
        }
        __syncthreads();
        if (D == 2) {
            for (int it = threadIdx.x; it < nk * n1; it += blockDim.x) {
                const int j = it / n1, kk1 = it % n1;
                C2<T> acc{T(0), T(0)};
                for (int m1 = 0; m1 < p; ++m1) acc = cfma(CoT[m1 * n1 + kk1], A[j * pd1 + m1], acc);
                o[(kc0 + j) * n1 + kk1] = acc;
            }
            __syncthreads();
        } else {
            for (int j = 0; j < nk; ++j) {
                for (int it = threadIdx.x; it < n1 * p; it += blockDim.x) {
                    const int kk1 = it / p, m2 = it % p;
                    C2<T> acc{T(0), T(0)};
                    for (int m1 = 0; m1 < p; ++m1) acc = cfma(Co[kk1 * p + m1], A[j * pd1 + m1 * p + m2], acc);
                    B[it] = acc;
                }
                __syncthreads();
                for (int it = threadIdx.x; it < n1 * n1; it += blockDim.x) {
                    const int kk1 = it / n1, kk2 = it % n1;
                    C2<T> acc{T(0), T(0)};
                    for (int m2 = 0; m2 < p; ++m2) acc = cfma(Co[kk2 * p + m2], B[kk1 * p + m2], acc);
                    o[((kc0 + j) * n1 + kk1) * n1 + kk2] = acc;
                }
                __syncthreads();
            }
        }
    }
}

// ------------------------------------------------------------------ translate + incoming
// entry: [local slot, level, 3^d colleague out slots (-1: none)]
template <typename T, int D>
__global__ void __launch_bounds__(128) k_pw_in(const int* __restrict__ list, const C2<T>* __restrict__ out,
                                               T* __restrict__ Lc, const C2<T>* __restrict__ Cog,
                                               const C2<T>* __restrict__ phg, const T* __restrict__ fk, PwDims pd,
                                               int KC, double inv_rc) {
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int NC = (D == 3) ? 27 : 9;
    const int p = pd.p, K = pd.K, n1 = pd.n1, pd1 = pd.pd1, nk1 = pd.nk1;
    C2<T>* Co = reinterpret_cast<C2<T>*>(sm);  // [n1][p]
    C2<T>* ph = Co + n1 * p;                   // [3][n1]
    C2<T>* I = ph + 3 * n1;                    // [KC][nk1]
    C2<T>* Ap = I + KC * nk1;                  // [KC][pd1]
    C2<T>* B = Ap + KC * pd1;                  // [n1][p]  (3D)
    __shared__ int coll[NC];
    for (int i = threadIdx.x; i < n1 * p; i += blockDim.x) Co[i] = Cog[i];
    for (int i = threadIdx.x; i < 3 * n1; i += blockDim.x) ph[i] = phg[i];
    const int* e = list + size_t(blockIdx.x) * (2 + NC);
    if (threadIdx.x < NC) coll[threadIdx.x] = e[2 + threadIdx.x];
    __syncthreads();
    const int level = e[1];
    // trapezoidal weight (1/(3h))^d times the h^2 of D-hat_l(xi) = h^2 f(|k|)
    const T wlev = (D == 3) ? T(double(1LL << level) * inv_rc / 27.0) : T(1.0 / 9.0);
    T* a = Lc + size_t(e[0]) * pd.np;
    for (int kc0 = 0; kc0 <= K; kc0 += KC) {
        const int nk = min(KC, K + 1 - kc0);
        // incoming slice: sum over colleagues with the translation phases
        for (int it = threadIdx.x; it < nk * nk1; it += blockDim.x) {
            const int j = it / nk1, rem = it % nk1;
            const int k0 = kc0 + j;
            const int kk1 = (D == 3) ? rem / n1 : rem;
            const int kk2 = (D == 3) ? rem % n1 : 0;
            const T f = fk[size_t(k0) * nk1 + rem];
            C2<T> acc{T(0), T(0)};
            if (f != T(0)) {
                for (int c = 0; c < NC; ++c) {
                    const int s = coll[c];
                    if (s < 0) continue;
                    const int d0 = c % 3, d1 = (c / 3) % 3, d2 = (c / 9) % 3;  // delta + 1
                    C2<T> phz = ph[d0 * n1 + k0 + K];
                    phz = cfma(phz, ph[d1 * n1 + kk1], C2<T>{T(0), T(0)});
                    if (D == 3) phz = cfma(phz, ph[d2 * n1 + kk2], C2<T>{T(0), T(0)});
                    acc = cfma(phz, out[size_t(s) * pd.npw + size_t(k0) * nk1 + rem], acc);
                }
                acc.x *= f * wlev;
                acc.y *= f * wlev;
            }
            I[it] = acc;
        }
        __syncthreads();
        if (D == 2) {
            for (int it = threadIdx.x; it < nk * p; it += blockDim.x) {
                const int j = it / p, m1 = it % p;
                C2<T> acc{T(0), T(0)};
                for (int kk1 = 0; kk1 < n1; ++kk1) acc = cfma_conj(Co[kk1 * p + m1], I[j * nk1 + kk1], acc);
                Ap[j * pd1 + m1] = acc;
            }
            __syncthreads();
        } else {
            for (int j = 0; j < nk; ++j) {
                for (int it = threadIdx.x; it < n1 * p; it += blockDim.x) {
                    const int kk1 = it / p, m2 = it % p;
                    C2<T> acc{T(0), T(0)};
                    for (int kk2 = 0; kk2 < n1; ++kk2)
                        acc = cfma_conj(Co[kk2 * p + m2], I[j * nk1 + kk1 * n1 + kk2], acc);
                    B[it] = acc;
                }
                __syncthreads();
                for (int it = threadIdx.x; it < p * p; it += blockDim.x) {
                    const int m1 = it / p, m2 = it % p;
                    C2<T> acc{T(0), T(0)};
                    for (int kk1 = 0; kk1 < n1; ++kk1) acc = cfma_conj(Co[kk1 * p + m1], B[kk1 * p + m2], acc);
                    Ap[j * pd1 + it] = acc;
                }
                __syncthreads();
            }
        }
        // a[m0][r] += sum_j w(k0) Re(conj(Co[k0][m0]) Ap[j][r]); w = 1 for k0 = 0, else 2
        for (int it = threadIdx.x; it < pd.np; it += blockDim.x) {
            const int m0 = it / pd1, r = it % pd1;
            T acc = T(0);
            for (int j = 0; j < nk; ++j) {
                const int k0 = kc0 + j;
                const C2<T> c = Co[(k0 + K) * p + m0];
                const C2<T> v = Ap[j * pd1 + r];
                const T re = fma(c.x, v.x, c.y * v.y);
                acc = fma(k0 == 0 ? T(1) : T(2), re, acc);
            }
            a[it] += acc;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ 3D compile-time outgoing / incoming
// The parity of the Chebyshev coefficients of exp(-i (pi/3) k t) makes every contraction with
// Co real: Co[k][2j] = ce[|k|][j] (real, even in k), Co[k][2j+1] = i sgn(k) so[|k|][j].  So
// each axis transform works on the half range k >= 0 and forms the pair of modes +-k at once.
// Both kernels take one box per block of P^2 threads, thread (m1, m2), and walk the k0 axis
// (the Hermitian half 0..K) slice by slice.

// Outgoing waves of one box, out[k0][k1][k2] = sum_m Co[k0][m0] Co[k1][m1] Co[k2][m2] q[m]:
//   A[m1][m2]  = sum_j ce[k0][j] q[2j][m1][m2] + i so[k0][j] q[2j+1][m1][m2]   (thread's own q)
//   B[+-k1][m2] = E +- i O,  E = sum_j ce[k1][j] A[2j][m2],  O = sum_j so[k1][j] A[2j+1][m2]
//   out[k0][k1][+-k2] = E' +- i O' over m2 in the same way.
// The modes are stored at their places in the full (K + 1) (2K + 1)^2 layout.
template <typename T, int P, int K>
__global__ void __launch_bounds__(P * P, (sizeof(T) == 4 && P * P <= 576) ? 2 : 1)
    k_pw_out3d_p(const int2* __restrict__ list, const T* __restrict__ Q, C2<T>* __restrict__ out,
                 const C2<T>* __restrict__ Cog, const int2* __restrict__ rowg) {
    constexpr int H = P / 2, KH = K + 1, N1 = 2 * K + 1, PP = P * P;
    __shared__ T ce[KH][H], so[KH][H];
    __shared__ C2<T> A[PP];      // [m1][m2]
    __shared__ C2<T> B[N1][P];   // [k1 + K][m2]
    __shared__ int2 row[KH][N1];  // (unused offset, m): the ball's rows k2 = -m .. m
    const int tid = threadIdx.x;
    for (int i = tid; i < KH * H; i += PP) {
        const int k = i / H, j = i % H;
        ce[k][j] = Cog[(k + K) * P + 2 * j].x;
        so[k][j] = Cog[(k + K) * P + 2 * j + 1].y;
    }
    for (int i = tid; i < KH * N1; i += PP) row[i / N1][i % N1] = rowg[i];
    const int2 e = list[blockIdx.x];
    const T* q = Q + size_t(e.x) * (PP * P);
    C2<T>* o = out + size_t(e.y) * (KH * N1 * N1);
    T qr[P];
#pragma unroll
    for (int m0 = 0; m0 < P; ++m0) qr[m0] = q[m0 * PP + tid];
    __syncthreads();
    for (int k0 = 0; k0 <= K; ++k0) {
        if (row[k0][K].y < 0) break;  // this slice and the later ones lie outside the ball
        {
            T ax = T(0), ay = T(0);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                ax = fma(ce[k0][j], qr[2 * j], ax);
                ay = fma(so[k0][j], qr[2 * j + 1], ay);
            }
            A[tid] = C2<T>{ax, ay};
        }
        __syncthreads();
        if (tid < KH * P && row[k0][K + tid / P].y >= 0) {  // rows +-k1 that meet the ball
            const int k1 = tid / P, m2 = tid % P;
            T ex = T(0), ey = T(0), ox = T(0), oy = T(0);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const C2<T> ae = A[(2 * j) * P + m2], ao = A[(2 * j + 1) * P + m2];
                const T c = ce[k1][j], s = so[k1][j];
                ex = fma(c, ae.x, ex);
                ey = fma(c, ae.y, ey);
                ox = fma(s, ao.x, ox);
                oy = fma(s, ao.y, oy);
            }
            B[K + k1][m2] = C2<T>{ex - oy, ey + ox};  // E + i O
            if (k1 > 0) B[K - k1][m2] = C2<T>{ex + oy, ey - ox};
        }
        __syncthreads();
        for (int it = tid; it < N1 * KH; it += PP) {
            const int kk1 = it / KH, k2 = it % KH;
            const int2 rw = row[k0][kk1];
            if (k2 > rw.y) continue;  // outside the ball: never read
            T ex = T(0), ey = T(0), ox = T(0), oy = T(0);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const C2<T> be = B[kk1][2 * j], bo = B[kk1][2 * j + 1];
                const T c = ce[k2][j], s = so[k2][j];
                ex = fma(c, be.x, ex);
                ey = fma(c, be.y, ey);
                ox = fma(s, bo.x, ox);
                oy = fma(s, bo.y, oy);
            }
            C2<T>* os = o + size_t(k0) * (N1 * N1) + kk1 * N1 + K;
            os[k2] = C2<T>{ex - oy, ey + ox};
            if (k2 > 0) os[-k2] = C2<T>{ex + oy, ey - ox};
        }
        // the next slice rewrites A only: every thread is past the reads of A (barrier above),
        // and B is rewritten only after the next barrier
    }
}

// Outgoing waves of one box over the half ball (FP32; the pairs (E, O) of k_pw_in3d_h's layout),
// the same three contractions as k_pw_out3d_p, each over all of the box's modes at once:
//  1. thread (m1, m2): A[k0][m1][m2] = sum_j ce[k0][j] q[2j][m1][m2] + i so[k0][j] q[2j+1][m1][m2]
//     for every slice k0 that meets the ball (its q in registers);
//  2. thread per (k0, m2; eight k1 >= 0): E = sum_j ce[k1][j] A[2j], O = sum_j so[k1][j] A[2j+1],
//     kept as the pair of rows +-k1 (B(+-k1) = E +- i O);
//  3. thread per (row k0, k1 >= 0; four k2 >= 0): E' = sum_j ce[k2][j] B[2j], O' = sum_j so[k2][j]
//     B[2j+1] for both rows +-k1, stored as (E', O') at the modes' compact indices.
// The tables are transposed (j major, the k axis padded to a multiple of eight) so that one
// 16-byte load gives four k.  Shared memory: A [nk0][P][P] in region 1 (r1 floats), the row pairs
// [rows][P + 1] in region 2, as in k_pw_in3d_h.
template <int P, int K>
__global__ void __launch_bounds__(P * P, P <= 16 ? 2 : 1)
    k_pw_out3d_h(const int2* __restrict__ list, const float* __restrict__ Q, float4* __restrict__ out,
                 const C2<float>* __restrict__ Cog, const int4* __restrict__ rowb, const int2* __restrict__ k0rows,
                 int nhalf, int nk0, int nrowb, int r1) {
    constexpr int H = P / 2, KH = K + 1, PP = P * P, KQ = (KH + 3) / 4, KT = 8 * ((KH + 7) / 8), KE = KT / 8;
    __shared__ __align__(16) float ce[KH][H];
    __shared__ __align__(16) float so[KH][H];
    __shared__ __align__(16) float ceT[H][KT];
    __shared__ __align__(16) float soT[H][KT];
    __shared__ int2 krow[KH];
    extern __shared__ __align__(16) float dsm[];
    float2* Ax = reinterpret_cast<float2*>(dsm);       // [nk0][P][P]
    float4* Bx = reinterpret_cast<float4*>(dsm + r1);  // [nrowb][P + 1] (E, O); the pad spreads rows over banks
    const int tid = threadIdx.x;
    for (int i = tid; i < KH * H; i += PP) {
        const int k = i / H, j = i % H;
        ce[k][j] = Cog[(k + K) * P + 2 * j].x;
        so[k][j] = Cog[(k + K) * P + 2 * j + 1].y;
    }
    for (int i = tid; i < H * KT; i += PP) {
        const int j = i / KT, k = i % KT;
        ceT[j][k] = k < KH ? Cog[(k + K) * P + 2 * j].x : 0.f;
        soT[j][k] = k < KH ? Cog[(k + K) * P + 2 * j + 1].y : 0.f;
    }
    for (int i = tid; i < KH; i += PP) krow[i] = k0rows[i];
    const int2 e = list[blockIdx.x];
    const float* q = Q + size_t(e.x) * (PP * P);
    float qr[P];
#pragma unroll
    for (int m0 = 0; m0 < P; ++m0) qr[m0] = q[m0 * PP + tid];
    __syncthreads();
    // 1. over m0, every slice
    for (int k0 = 0; k0 < nk0; ++k0) {
        float ax = 0.f, ay = 0.f;
#pragma unroll
        for (int j4 = 0; j4 < H; j4 += 4) {
            const float4 c4 = *reinterpret_cast<const float4*>(&ce[k0][j4]);
            const float4 s4 = *reinterpret_cast<const float4*>(&so[k0][j4]);
            ax = fmaf(c4.x, qr[2 * j4 + 0], ax);
            ay = fmaf(s4.x, qr[2 * j4 + 1], ay);
            ax = fmaf(c4.y, qr[2 * j4 + 2], ax);
            ay = fmaf(s4.y, qr[2 * j4 + 3], ay);
            ax = fmaf(c4.z, qr[2 * j4 + 4], ax);
            ay = fmaf(s4.z, qr[2 * j4 + 5], ay);
            ax = fmaf(c4.w, qr[2 * j4 + 6], ax);
            ay = fmaf(s4.w, qr[2 * j4 + 7], ay);
        }
        Ax[size_t(k0) * PP + tid] = make_float2(ax, ay);
    }
    __syncthreads();
    // 2. over m1, eight k1 per thread (m2 fastest across threads)
    for (int t = tid; t < nk0 * P * KE; t += PP) {
        const int m2 = t % P, ke = (t / P) % KE, k0 = t / (KE * P);
        const int2 kr = krow[k0];
        if (8 * ke >= kr.y) continue;
        float ex[8], ey[8], ox[8], oy[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) ex[i] = ey[i] = ox[i] = oy[i] = 0.f;
        const float2* a = Ax + size_t(k0) * PP + m2;
#pragma unroll 2
        for (int j = 0; j < H; ++j) {
            const float2 ae = a[(2 * j) * P], ao = a[(2 * j + 1) * P];
            const float4 c0 = *reinterpret_cast<const float4*>(&ceT[j][8 * ke]);
            const float4 c1 = *reinterpret_cast<const float4*>(&ceT[j][8 * ke + 4]);
            const float4 s0 = *reinterpret_cast<const float4*>(&soT[j][8 * ke]);
            const float4 s1 = *reinterpret_cast<const float4*>(&soT[j][8 * ke + 4]);
            const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                ex[i] = fmaf(cv[i], ae.x, ex[i]);
                ey[i] = fmaf(cv[i], ae.y, ey[i]);
                ox[i] = fmaf(sv[i], ao.x, ox[i]);
                oy[i] = fmaf(sv[i], ao.y, oy[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (8 * ke + i < kr.y) Bx[size_t(kr.x + 8 * ke + i) * (P + 1) + m2] = make_float4(ex[i], ey[i], ox[i], oy[i]);
    }
    __syncthreads();
    // 3. over m2, four k2 per thread, rows +k1 and -k1
    float4* o = out + size_t(e.y) * nhalf;
    for (int t = tid; t < nrowb * KQ; t += PP) {
        const int kq = t % KQ, rb = t / KQ;
        const int4 rw = __ldg(rowb + rb);  // (k0 | k1 << 8 | m << 16, row +k1, row -k1, 0)
        const int k1 = (rw.x >> 8) & 255, m = rw.x >> 16;
        if (4 * kq > m) continue;
        float pe[4][2], po[4][2], ne[4][2], no[4][2];  // (E', O') of rows +k1 / -k1 per k2
#pragma unroll
        for (int i = 0; i < 4; ++i) pe[i][0] = pe[i][1] = po[i][0] = po[i][1] = ne[i][0] = ne[i][1] = no[i][0] = no[i][1] = 0.f;
        const float4* b = Bx + size_t(rb) * (P + 1);
#pragma unroll 4
        for (int j = 0; j < H; ++j) {
            const float4 be = b[2 * j], bo = b[2 * j + 1];  // (E, O) at n2 = 2j, 2j + 1
            // B(+k1) = E + i O, B(-k1) = E - i O
            const float bpe_x = be.x - be.w, bpe_y = be.y + be.z, bne_x = be.x + be.w, bne_y = be.y - be.z;
            const float bpo_x = bo.x - bo.w, bpo_y = bo.y + bo.z, bno_x = bo.x + bo.w, bno_y = bo.y - bo.z;
            const float4 c4 = *reinterpret_cast<const float4*>(&ceT[j][4 * kq]);
            const float4 s4 = *reinterpret_cast<const float4*>(&soT[j][4 * kq]);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                pe[i][0] = fmaf(cv[i], bpe_x, pe[i][0]);
                pe[i][1] = fmaf(cv[i], bpe_y, pe[i][1]);
                po[i][0] = fmaf(sv[i], bpo_x, po[i][0]);
                po[i][1] = fmaf(sv[i], bpo_y, po[i][1]);
                ne[i][0] = fmaf(cv[i], bne_x, ne[i][0]);
                ne[i][1] = fmaf(cv[i], bne_y, ne[i][1]);
                no[i][0] = fmaf(sv[i], bno_x, no[i][0]);
                no[i][1] = fmaf(sv[i], bno_y, no[i][1]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k2 = 4 * kq + i;
            if (k2 > m) break;
            o[rw.y + k2] = make_float4(pe[i][0], pe[i][1], po[i][0], po[i][1]);
            if (k1 > 0) o[rw.z + k2] = make_float4(ne[i][0], ne[i][1], no[i][0], no[i][1]);
        }
    }
}

// Translation + incoming of one in-box (list entry: local slot, level, 27 colleague out slots).
// Per slice k0:
//  1. thread (k1, k2 >= 0) sums the colleagues' waves at (k0, k1, +-k2) with the phases
//     exp(-i (2 pi/3) k.delta), which factor by axis; along each axis the three colleagues
//     combine as X_0 + Re(u) (X_+ + X_-) +- i Im(u) (X_+ - X_-), the sign following the mode.
//     The weighted pair is kept as Sp = I(+k2) + I(-k2), Sm = I(+k2) - I(-k2).
//  2. thread (k1 >= 0, m2): contraction over k2 with conj(Co) (ce Sp for even m2, -i so Sm
//     for odd m2) for the rows +-k1, kept again as the sum Bp and the difference Bm.
//  3. thread (m1, m2): contraction over k1 the same way, then
//     a[2j][m1][m2] += w ce[k0][j] Re(.), a[2j+1][m1][m2] += w so[k0][j] Im(.),
//     w = 1 for k0 = 0, else 2 (the Hermitian half of the k0 axis), in registers.
// Each in-box has one entry: the coefficients are written, not added.
template <typename T, int P, int K>
__global__ void __launch_bounds__(P * P) k_pw_in3d_p(const int* __restrict__ list, const C2<T>* __restrict__ out,
                                                    T* __restrict__ Lc, const C2<T>* __restrict__ Cog,
                                                    const C2<T>* __restrict__ phg, const T* __restrict__ fk,
                                                    double inv_rc) {
    constexpr int H = P / 2, KH = K + 1, N1 = 2 * K + 1, PP = P * P, NK1 = N1 * N1, NPW = KH * NK1;
    __shared__ T ce[KH][H], so[KH][H];
    __shared__ C2<T> u[N1];                  // exp(-i (2 pi/3) k), k = -K..K
    __shared__ C2<T> Sp[N1][KH], Sm[N1][KH];  // [k1 + K][k2]
    __shared__ C2<T> Bp[KH][P], Bm[KH][P];    // [k1][m2]
    __shared__ int coll[27];
    const int tid = threadIdx.x;
    for (int i = tid; i < KH * H; i += PP) {
        const int k = i / H, j = i % H;
        ce[k][j] = Cog[(k + K) * P + 2 * j].x;
        so[k][j] = Cog[(k + K) * P + 2 * j + 1].y;
    }
    for (int i = tid; i < N1; i += PP) u[i] = phg[2 * N1 + i];  // delta = +1
    const int* e = list + size_t(blockIdx.x) * 29;
    if (tid < 27) coll[tid] = e[2 + tid];
    __syncthreads();
    const int level = e[1];
    // trapezoidal weight (1/(3h))^3 times the h^2 of D-hat_l(xi) = h^2 f(|k|)
    const T wlev = T(double(1LL << level) * inv_rc / 27.0);
    T acc[P];
#pragma unroll
    for (int m = 0; m < P; ++m) acc[m] = T(0);
    const int m1 = tid / P, m2 = tid % P;
    for (int k0 = 0; k0 <= K; ++k0) {
        // 1. weighted sums over the colleagues, modes (k0, k1, +-k2)
        for (int it = tid; it < N1 * KH; it += PP) {
            const int kk1 = it / KH, k2 = it % KH;
            const T fw = fk[size_t(k0) * NK1 + kk1 * N1 + K + k2] * wlev;
            C2<T> ip{T(0), T(0)}, im{T(0), T(0)};
            if (fw != T(0)) {
                const C2<T> u2 = u[K + k2], u1 = u[kk1], u0 = u[K + k0];
                const size_t op = size_t(k0) * NK1 + size_t(kk1) * N1 + K + k2;
                const size_t om = op - 2 * k2;
                const C2<T> z{T(0), T(0)};
                C2<T> tp[3], tm[3];  // per delta0: sums over delta1, delta2
#pragma unroll
                for (int d0 = 0; d0 < 3; ++d0) {
                    C2<T> rp[3], rm[3];  // per delta1: sums over delta2
#pragma unroll
                    for (int d1 = 0; d1 < 3; ++d1) {
                        const int sM = coll[d0 + 3 * d1], s0 = coll[d0 + 3 * d1 + 9], sP = coll[d0 + 3 * d1 + 18];
                        const C2<T> pP = sP >= 0 ? out[size_t(sP) * NPW + op] : z;
                        const C2<T> pM = sM >= 0 ? out[size_t(sM) * NPW + op] : z;
                        const C2<T> p0 = s0 >= 0 ? out[size_t(s0) * NPW + op] : z;
                        const C2<T> mP = sP >= 0 ? out[size_t(sP) * NPW + om] : z;
                        const C2<T> mM = sM >= 0 ? out[size_t(sM) * NPW + om] : z;
                        const C2<T> m0 = s0 >= 0 ? out[size_t(s0) * NPW + om] : z;
                        rp[d1].x = p0.x + u2.x * (pP.x + pM.x) - u2.y * (pP.y - pM.y);
                        rp[d1].y = p0.y + u2.x * (pP.y + pM.y) + u2.y * (pP.x - pM.x);
                        rm[d1].x = m0.x + u2.x * (mP.x + mM.x) + u2.y * (mP.y - mM.y);
                        rm[d1].y = m0.y + u2.x * (mP.y + mM.y) - u2.y * (mP.x - mM.x);
                    }
                    // axis 1: the mode k1 is the same for both members of the pair
                    tp[d0].x = rp[1].x + u1.x * (rp[2].x + rp[0].x) - u1.y * (rp[2].y - rp[0].y);
                    tp[d0].y = rp[1].y + u1.x * (rp[2].y + rp[0].y) + u1.y * (rp[2].x - rp[0].x);
                    tm[d0].x = rm[1].x + u1.x * (rm[2].x + rm[0].x) - u1.y * (rm[2].y - rm[0].y);
                    tm[d0].y = rm[1].y + u1.x * (rm[2].y + rm[0].y) + u1.y * (rm[2].x - rm[0].x);
                }
                ip.x = fw * (tp[1].x + u0.x * (tp[2].x + tp[0].x) - u0.y * (tp[2].y - tp[0].y));
                ip.y = fw * (tp[1].y + u0.x * (tp[2].y + tp[0].y) + u0.y * (tp[2].x - tp[0].x));
                im.x = fw * (tm[1].x + u0.x * (tm[2].x + tm[0].x) - u0.y * (tm[2].y - tm[0].y));
                im.y = fw * (tm[1].y + u0.x * (tm[2].y + tm[0].y) + u0.y * (tm[2].x - tm[0].x));
            }
            if (k2 == 0) {
                Sp[kk1][0] = ip;  // the +-k2 modes coincide
                Sm[kk1][0] = C2<T>{T(0), T(0)};
            } else {
                Sp[kk1][k2] = C2<T>{ip.x + im.x, ip.y + im.y};
                Sm[kk1][k2] = C2<T>{ip.x - im.x, ip.y - im.y};
            }
        }
        __syncthreads();
        // 2. over k2, rows +-k1
        if (tid < KH * P) {
            const int k1 = tid / P, n2 = tid % P, j = n2 >> 1;
            const bool odd = n2 & 1;
            const T* tab = odd ? &so[0][j] : &ce[0][j];
            const C2<T>* sP = odd ? &Sm[K + k1][0] : &Sp[K + k1][0];
            const C2<T>* sN = odd ? &Sm[K - k1][0] : &Sp[K - k1][0];
            T px = T(0), py = T(0), nx = T(0), ny = T(0);
#pragma unroll
            for (int k2 = 0; k2 < KH; ++k2) {
                const T c = tab[k2 * H];
                const C2<T> a = sP[k2], b = sN[k2];
                px = fma(c, a.x, px);
                py = fma(c, a.y, py);
                nx = fma(c, b.x, nx);
                ny = fma(c, b.y, ny);
            }
            // odd m2: times -i
            C2<T> vp = odd ? C2<T>{py, -px} : C2<T>{px, py};
            C2<T> vn = odd ? C2<T>{ny, -nx} : C2<T>{nx, ny};
            if (k1 == 0) vn = C2<T>{T(0), T(0)};
            Bp[k1][n2] = C2<T>{vp.x + vn.x, vp.y + vn.y};
            Bm[k1][n2] = k1 == 0 ? C2<T>{T(0), T(0)} : C2<T>{vp.x - vn.x, vp.y - vn.y};
        }
        __syncthreads();
        // 3. over k1 (thread's own (m1, m2)), then over k0 into the registers
        {
            const bool odd = m1 & 1;
            const int j1 = m1 >> 1;
            const T* tab = odd ? &so[0][j1] : &ce[0][j1];
            const C2<T>* bb = odd ? &Bm[0][m2] : &Bp[0][m2];
            T ax = T(0), ay = T(0);
#pragma unroll
            for (int k1 = 0; k1 < KH; ++k1) {
                const T c = tab[k1 * H];
                const C2<T> v = bb[k1 * P];
                ax = fma(c, v.x, ax);
                ay = fma(c, v.y, ay);
            }
            const T re = odd ? ay : ax, im_ = odd ? -ax : ay;  // odd m1: times -i
            const T w = k0 == 0 ? T(1) : T(2);
            const T wr = w * re, wi = w * im_;
#pragma unroll
            for (int j0 = 0; j0 < H; ++j0) {
                acc[2 * j0] = fma(ce[k0][j0], wr, acc[2 * j0]);
                acc[2 * j0 + 1] = fma(so[k0][j0], wi, acc[2 * j0 + 1]);
            }
        }
        // the next slice rewrites Sp / Sm only (every thread is past step 2); Bp / Bm are
        // rewritten after the next barrier
    }
    T* a = Lc + size_t(e[0]) * (PP * P);
#pragma unroll
    for (int m0 = 0; m0 < P; ++m0) a[m0 * PP + tid] = acc[m0];
}

// Translation + incoming of one in-box over the half ball (FP32, the outgoing waves stored as
// (E, O) pairs: out(+-k2) = E +- i O at the compact index of the mode, k2 >= 0).  Four phases,
// each over all of the box's modes at once (one barrier between phases):
//  A. thread per mode (k0, k1, k2 >= 0): the 27 colleagues' pairs, one 16-byte load each.  With
//     u = exp(-i (2 pi/3) k2) = a + i b, the axis-2 neighbours of a row combine into
//       Xe = E_0 + a (E_+ + E_-) - b (O_+ - O_-),   Xo = O_0 + a (O_+ + O_-) + b (E_+ - E_-),
//     which are (I(+k2) + I(-k2)) / 2 and (I(+k2) - I(-k2)) / 2i for the axis-2 sums I; axes 1
//     and 0 apply the same complex phase to both.  The weight f(|k|) (doubled for k2 > 0, where
//     the two modes are folded into one pair) gives Sp = 2 Xe f, Sm = 2 Xo f (the -i that the
//     odd Chebyshev coefficients carry is absorbed into Sm).
//  B. thread per (row k0, k1 >= 0; four j): the k2 contraction of the rows +-k1,
//       even n2 = 2j: ce[k2][j] Sp,  odd n2 = 2j + 1: so[k2][j] Sm,
//     kept as the sum Bp and the difference Bm of the two rows (row k1 = 0 alone: Bm = 0).
//  C. thread per (k0, m2; four j): the k1 contraction, even m1: ce Bp, odd m1: -i so Bm, times
//     w = 1 for k0 = 0 and 2 otherwise (the Hermitian half of the k0 axis).
//  D. thread (m1, m2): the k0 contraction into P registers, a[2j] += ce[k0][j] Re, a[2j+1] +=
//     so[k0][j] Im, written (each in-box has one entry).
// Shared memory: the modes' (Sp, Sm) [nhalf], reused for C [nk0][P][P] (region 1 of r1 floats),
// then B [rows][P + 1] (region 2).
template <int P, int K>
__global__ void __launch_bounds__(P * P, P <= 16 ? 2 : 1)
    k_pw_in3d_h(const int* __restrict__ list, const float4* __restrict__ out, float* __restrict__ Lc,
                const C2<float>* __restrict__ Cog, const C2<float>* __restrict__ phg, const int* __restrict__ item,
                const float* __restrict__ fh, const int4* __restrict__ rowb, const int2* __restrict__ k0rows,
                int nhalf, int nk0, int nrowb, int r1, double inv_rc) {
    constexpr int H = P / 2, KH = K + 1, N1 = 2 * K + 1, PP = P * P, NQ = H / 4;
    static_assert(H % 4 == 0, "the j axis is taken four at a time");
    __shared__ __align__(16) float ce[KH][H];
    __shared__ __align__(16) float so[KH][H];
    __shared__ C2<float> u[N1];  // exp(-i (2 pi/3) k), k = -K..K
    __shared__ int coll[27];
    __shared__ int2 krow[KH];    // per k0: first row of the k2 contraction, rows (k1 = 0, 1, ..)
    extern __shared__ __align__(16) float dsm[];
    float4* Sx = reinterpret_cast<float4*>(dsm);       // [nhalf] (Sp, Sm)
    float2* Cx = reinterpret_cast<float2*>(dsm);       // [nk0][P][P] (after phase B)
    float4* Bx = reinterpret_cast<float4*>(dsm + r1);  // [nrowb][P + 1] (Bp, Bm); the pad spreads rows over banks
    const int tid = threadIdx.x;
    for (int i = tid; i < KH * H; i += PP) {
        const int k = i / H, j = i % H;
        ce[k][j] = Cog[(k + K) * P + 2 * j].x;
        so[k][j] = Cog[(k + K) * P + 2 * j + 1].y;
    }
    for (int i = tid; i < N1; i += PP) u[i] = phg[2 * N1 + i];  // delta = +1
    for (int i = tid; i < KH; i += PP) krow[i] = k0rows[i];
    const int* e = list + size_t(blockIdx.x) * 29;
    if (tid < 27) coll[tid] = e[2 + tid];
    __syncthreads();
    // trapezoidal weight (1/(3h))^3 times the h^2 of D-hat_l(xi) = h^2 f(|k|)
    const float wlev = float(double(1LL << e[1]) * inv_rc / 27.0);
    // A. translation
    for (int i = tid; i < nhalf; i += PP) {
        const int it = __ldg(item + i);
        const int k0 = it & 255, kk1 = (it >> 8) & 255, k2 = it >> 16;
        const float fw = __ldg(fh + i) * wlev;
        const C2<float> u2 = u[K + k2], u1 = u[kk1], u0 = u[K + k0];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 t[3];  // per delta0: (Xe, Xo) summed over delta1, delta2
#pragma unroll
        for (int d0 = 0; d0 < 3; ++d0) {
            float4 r[3];  // per delta1: summed over delta2
#pragma unroll
            for (int d1 = 0; d1 < 3; ++d1) {
                const int sM = coll[d0 + 3 * d1], s0 = coll[d0 + 3 * d1 + 9], sP = coll[d0 + 3 * d1 + 18];
                const float4 pP = sP >= 0 ? __ldg(out + size_t(sP) * nhalf + i) : z;
                const float4 pM = sM >= 0 ? __ldg(out + size_t(sM) * nhalf + i) : z;
                const float4 p0 = s0 >= 0 ? __ldg(out + size_t(s0) * nhalf + i) : z;
                r[d1].x = p0.x + u2.x * (pP.x + pM.x) - u2.y * (pP.z - pM.z);
                r[d1].y = p0.y + u2.x * (pP.y + pM.y) - u2.y * (pP.w - pM.w);
                r[d1].z = p0.z + u2.x * (pP.z + pM.z) + u2.y * (pP.x - pM.x);
                r[d1].w = p0.w + u2.x * (pP.w + pM.w) + u2.y * (pP.y - pM.y);
            }
            // axis 1: X_0 + u X_+ + conj(u) X_-, for Xe (x, y) and Xo (z, w)
            t[d0].x = r[1].x + u1.x * (r[2].x + r[0].x) - u1.y * (r[2].y - r[0].y);
            t[d0].y = r[1].y + u1.x * (r[2].y + r[0].y) + u1.y * (r[2].x - r[0].x);
            t[d0].z = r[1].z + u1.x * (r[2].z + r[0].z) - u1.y * (r[2].w - r[0].w);
            t[d0].w = r[1].w + u1.x * (r[2].w + r[0].w) + u1.y * (r[2].z - r[0].z);
        }
        float4 v;
        v.x = fw * (t[1].x + u0.x * (t[2].x + t[0].x) - u0.y * (t[2].y - t[0].y));
        v.y = fw * (t[1].y + u0.x * (t[2].y + t[0].y) + u0.y * (t[2].x - t[0].x));
        v.z = fw * (t[1].z + u0.x * (t[2].z + t[0].z) - u0.y * (t[2].w - t[0].w));
        v.w = fw * (t[1].w + u0.x * (t[2].w + t[0].w) + u0.y * (t[2].z - t[0].z));
        Sx[i] = v;
    }
    __syncthreads();
    // B. over k2, rows +-k1 (four j per thread)
    for (int t = tid; t < nrowb * NQ; t += PP) {
        const int q = t % NQ, rb = t / NQ;
        const int4 rw = __ldg(rowb + rb);  // (k0 | k1 << 8 | m << 16, row +k1, row -k1, 0)
        const int k1 = (rw.x >> 8) & 255, m = rw.x >> 16;
        const float4* sp = Sx + rw.y;
        const float4* sn = Sx + rw.z;
        float ep[4][2], en[4][2], op[4][2], on[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) ep[j][0] = ep[j][1] = en[j][0] = en[j][1] = op[j][0] = op[j][1] = on[j][0] = on[j][1] = 0.f;
        for (int k2 = 0; k2 <= m; ++k2) {
            const float4 a = sp[k2], b = sn[k2];
            const float4 c4 = *reinterpret_cast<const float4*>(&ce[k2][4 * q]);
            const float4 s4 = *reinterpret_cast<const float4*>(&so[k2][4 * q]);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ep[j][0] = fmaf(cv[j], a.x, ep[j][0]);
                ep[j][1] = fmaf(cv[j], a.y, ep[j][1]);
                en[j][0] = fmaf(cv[j], b.x, en[j][0]);
                en[j][1] = fmaf(cv[j], b.y, en[j][1]);
                op[j][0] = fmaf(sv[j], a.z, op[j][0]);
                op[j][1] = fmaf(sv[j], a.w, op[j][1]);
                on[j][0] = fmaf(sv[j], b.z, on[j][0]);
                on[j][1] = fmaf(sv[j], b.w, on[j][1]);
            }
        }
        float4* bo = Bx + size_t(rb) * (P + 1) + 8 * q;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k1 == 0) {
                bo[2 * j] = make_float4(ep[j][0], ep[j][1], 0.f, 0.f);
                bo[2 * j + 1] = make_float4(op[j][0], op[j][1], 0.f, 0.f);
            } else {
                bo[2 * j] = make_float4(ep[j][0] + en[j][0], ep[j][1] + en[j][1], ep[j][0] - en[j][0], ep[j][1] - en[j][1]);
                bo[2 * j + 1] =
                    make_float4(op[j][0] + on[j][0], op[j][1] + on[j][1], op[j][0] - on[j][0], op[j][1] - on[j][1]);
            }
        }
    }
    __syncthreads();
    // C. over k1 (four j per thread: m1 = 2j even, 2j + 1 odd), into region 1
    for (int t = tid; t < nk0 * P * NQ; t += PP) {
        const int q = t % NQ, m2 = (t / NQ) % P, k0 = t / (NQ * P);
        const int2 kr = krow[k0];
        float ex[4], ey[4], ox[4], oy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) ex[j] = ey[j] = ox[j] = oy[j] = 0.f;
        const float4* bb = Bx + size_t(kr.x) * (P + 1) + m2;
        for (int k1 = 0; k1 < kr.y; ++k1) {
            const float4 b = bb[size_t(k1) * (P + 1)];
            const float4 c4 = *reinterpret_cast<const float4*>(&ce[k1][4 * q]);
            const float4 s4 = *reinterpret_cast<const float4*>(&so[k1][4 * q]);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ex[j] = fmaf(cv[j], b.x, ex[j]);
                ey[j] = fmaf(cv[j], b.y, ey[j]);
                ox[j] = fmaf(sv[j], b.z, ox[j]);
                oy[j] = fmaf(sv[j], b.w, oy[j]);
            }
        }
        const float w = k0 == 0 ? 1.f : 2.f;
        float2* cc = Cx + size_t(k0) * PP + m2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m1 = 2 * (4 * q + j);
            cc[m1 * P] = make_float2(w * ex[j], w * ey[j]);
            cc[(m1 + 1) * P] = make_float2(w * oy[j], -w * ox[j]);  // odd m1: times -i
        }
    }
    __syncthreads();
    // D. over k0 into registers, thread (m1, m2)
    float acc[P];
#pragma unroll
    for (int m = 0; m < P; ++m) acc[m] = 0.f;
    for (int k0 = 0; k0 < nk0; ++k0) {
        const float2 c = Cx[size_t(k0) * PP + tid];
#pragma unroll
        for (int j4 = 0; j4 < H; j4 += 4) {
            const float4 c4 = *reinterpret_cast<const float4*>(&ce[k0][j4]);
            const float4 s4 = *reinterpret_cast<const float4*>(&so[k0][j4]);
            acc[2 * j4 + 0] = fmaf(c4.x, c.x, acc[2 * j4 + 0]);
            acc[2 * j4 + 1] = fmaf(s4.x, c.y, acc[2 * j4 + 1]);
            acc[2 * j4 + 2] = fmaf(c4.y, c.x, acc[2 * j4 + 2]);
            acc[2 * j4 + 3] = fmaf(s4.y, c.y, acc[2 * j4 + 3]);
            acc[2 * j4 + 4] = fmaf(c4.z, c.x, acc[2 * j4 + 4]);
            acc[2 * j4 + 5] = fmaf(s4.z, c.y, acc[2 * j4 + 5]);
            acc[2 * j4 + 6] = fmaf(c4.w, c.x, acc[2 * j4 + 6]);
            acc[2 * j4 + 7] = fmaf(s4.w, c.y, acc[2 * j4 + 7]);
        }
    }
    float* a = Lc + size_t(e[0]) * (PP * P);
#pragma unroll
    for (int m0 = 0; m0 < P; ++m0) a[m0 * PP + tid] = acc[m0];
}

// 3D leaf evaluation with a compile-time order P: one warp per leaf, a thread per target.  The
// z-axis T_m, T'_m sit in registers, the x- and y-axis ones in shared memory (interleaved by
// thread), and the leaf's coefficient rows are read as vectors (all lanes read the same row:
// one broadcast load per 4 (FP32) or 2 (FP64) coefficients).
template <typename T, int P>
__global__ void __launch_bounds__(32) k_leaf_eval3d_p(const int4* __restrict__ list, const T* __restrict__ Lc,
                                                      const T* __restrict__ tgt4, double* __restrict__ pot,
                                                      double* __restrict__ grad, double inv_rc) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = sizeof(V) / sizeof(T), NV = P / VW;
    static_assert(P % VW == 0, "rows are whole vectors");
    __shared__ T tab[4][P][32];  // [b0, d0, b1, d1][m][lane]
    const int lane = threadIdx.x;
    const int4 e = list[blockIdx.x];
    const T* a = Lc + size_t(e.x) * (P * P * P);
    const double sc = 2.0 * inv_rc * double(1LL << e.w);  // dt/dx = 2/h
    for (int t0 = 0; t0 < e.z; t0 += 32) {
        const int ti = t0 + lane;
        const bool act = ti < e.z;
        T tz[P], dz[P];
        {
            const T* x = tgt4 + size_t(e.y + (act ? ti : 0)) * 4;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const T t = T(double(x[ax]) * sc);
                T tm1 = T(1), tm = t, um1 = T(1), um = T(2) * t;
                T bv[P], dv[P];
                bv[0] = T(1);
                dv[0] = T(0);
                bv[1] = t;
                dv[1] = T(1);
#pragma unroll
                for (int m = 2; m < P; ++m) {
                    const T tn = fma(T(2) * t, tm, -tm1);
                    bv[m] = tn;
                    dv[m] = T(m) * um;  // T'_m = m U_{m-1}
                    const T un = fma(T(2) * t, um, -um1);
                    tm1 = tm;
                    tm = tn;
                    um1 = um;
                    um = un;
                }
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    if (ax < 2) {
                        tab[2 * ax][m][lane] = bv[m];
                        tab[2 * ax + 1][m][lane] = dv[m];
                    } else {
                        tz[m] = bv[m];
                        dz[m] = dv[m];
                    }
                }
            }
        }
        __syncwarp();
        T phi = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll 1
        for (int m0 = 0; m0 < P; ++m0) {
            T s = 0, s1d = 0, s2d = 0;
#pragma unroll 2
            for (int m1 = 0; m1 < P; ++m1) {
                const V* row = reinterpret_cast<const V*>(a + (m0 * P + m1) * P);
                T u = 0, ud = 0;
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const V v = __ldg(row + k);
                    if constexpr (VW == 4) {
                        u = fma(v.x, tz[4 * k], u);
                        ud = fma(v.x, dz[4 * k], ud);
                        u = fma(v.y, tz[4 * k + 1], u);
                        ud = fma(v.y, dz[4 * k + 1], ud);
                        u = fma(v.z, tz[4 * k + 2], u);
                        ud = fma(v.z, dz[4 * k + 2], ud);
                        u = fma(v.w, tz[4 * k + 3], u);
                        ud = fma(v.w, dz[4 * k + 3], ud);
                    } else {
                        u = fma(v.x, tz[2 * k], u);
                        ud = fma(v.x, dz[2 * k], ud);
                        u = fma(v.y, tz[2 * k + 1], u);
                        ud = fma(v.y, dz[2 * k + 1], ud);
                    }
                }
                const T b1 = tab[2][m1][lane], d1 = tab[3][m1][lane];
                s = fma(b1, u, s);
                s1d = fma(d1, u, s1d);
                s2d = fma(b1, ud, s2d);
            }
            const T b0 = tab[0][m0][lane], d0 = tab[1][m0][lane];
            phi = fma(b0, s, phi);
            g0 = fma(d0, s, g0);
            g1 = fma(b0, s1d, g1);
            g2 = fma(b0, s2d, g2);
        }
        if (act) {
            const size_t o = size_t(e.y + ti);
            pot[o] = double(phi);
            if (grad) {
                grad[o * 3 + 0] = double(g0) * sc;
                grad[o * 3 + 1] = double(g1) * sc;
                grad[o * 3 + 2] = double(g2) * sc;
            }
        }
        __syncwarp();
    }
}

// 3D leaf evaluation as a small GEMM per leaf: one block of 256 threads per target leaf, the
// leaf's P^3 local coefficients a[m0][m1 m2] staged once in shared memory, its targets taken
// 16 at a time.  For a chunk the rows X = [T_m0(x_t); T'_m0(x_t)] (32 rows) multiply the
// coefficients viewed as a P x P^2 matrix:
//     A[r][m1 m2] = sum_m0 X[r][m0] a[m0][m1 m2]                    (2 P^3 multiply-adds per target)
// with a register tile of 8 rows x P^2/64 columns per thread (columns strided by 64, so the
// shared loads of a row are conflict-free and the 8 row values are broadcasts).  Then every
// thread weights its columns by T_m1(y_t) T_m2(z_t) and the derivative tables, and the 64
// threads sharing a target's rows add their partials by a fixed shuffle tree (deterministic).
//     phi  = sum A[T row] Ty Tz,  g_x = sum A[T' row] Ty Tz,
//     g_y  = sum A[T row] Ty' Tz, g_z = sum A[T row] Ty Tz'        (times dt/dx = 2/h)
template <typename T, int P>
constexpr size_t leaf_eval3d_gemm_smem() {
    return sizeof(T) * (size_t(P) * P * P + size_t(P) * 32 + size_t(16) * 4 * (P + 1)) + sizeof(double) * 4 * 2 * 16;
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_leaf_eval3d_gemm(const int4* __restrict__ list, const T* __restrict__ Lc,
                                                          const T* __restrict__ tgt4, double* __restrict__ pot,
                                                          double* __restrict__ grad, double inv_rc) {
    constexpr int PP = P * P, NP = PP * P, CT = PP / 64, RT = 8;
    static_assert(PP % 64 == 0, "columns split over 64 threads");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* La = reinterpret_cast<T*>(smraw);  // [P][PP]
    T* X = La + NP;                       // [P][32]  X[m0][r], r = 2 t + (0: T, 1: T')
    constexpr int PS = P + 1;             // odd row stride: the 16 targets' rows fall in distinct banks
    T* TB = X + P * 32;                   // [16][4][PS]  (Ty, Ty', Tz, Tz') per target
    double* red = reinterpret_cast<double*>(TB + 16 * 4 * PS);  // [4 row groups][2 warps][16]
    const int tid = threadIdx.x, rg = tid >> 6, cg = tid & 63, lane = tid & 31, half = (tid >> 5) & 1;
    const int4 e = list[blockIdx.x];      // (local slot, first target, target count, level)
    const double sc = 2.0 * inv_rc * double(1LL << e.w);  // dt/dx = 2/h
    {
        const T* a = Lc + size_t(e.x) * NP;
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int VW = sizeof(V) / sizeof(T);
        const V* av = reinterpret_cast<const V*>(a);
        V* lv = reinterpret_cast<V*>(La);
        for (int k = tid; k < NP / VW; k += 256) lv[k] = __ldg(av + k);
    }
    for (int t0 = 0; t0 < e.z; t0 += 16) {
        const int nt = min(16, e.z - t0);
        __syncthreads();  // previous chunk done with X, TB, red
        if (tid < 48) {
            const int t = tid / 3, ax = tid - 3 * t;
            T tv = T(0);
            if (t < nt) tv = T(double(tgt4[size_t(e.y + t0 + t) * 4 + ax]) * sc);
            T tm1 = T(1), tm = tv, um1 = T(1), um = T(2) * tv;
            const T live = t < nt ? T(1) : T(0);  // rows of absent targets are zero
            auto put = [&](int m, T b, T d) {
                if (ax == 0) {
                    X[m * 32 + 2 * t] = b * live;
                    X[m * 32 + 2 * t + 1] = d * live;
                } else {
                    TB[(t * 4 + 2 * (ax - 1)) * PS + m] = b;
                    TB[(t * 4 + 2 * (ax - 1) + 1) * PS + m] = d;
                }
            };
            put(0, T(1), T(0));
            put(1, tv, T(1));
#pragma unroll
            for (int m = 2; m < P; ++m) {
                const T tn = fma(T(2) * tv, tm, -tm1);
                put(m, tn, T(m) * um);  // T'_m = m U_{m-1}
                const T un = fma(T(2) * tv, um, -um1);
                tm1 = tm;
                tm = tn;
                um1 = um;
                um = un;
            }
        }
        __syncthreads();
        T acc[RT][CT];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int k = 0; k < CT; ++k) acc[i][k] = T(0);
#pragma unroll 2
        for (int m0 = 0; m0 < P; ++m0) {
            T xr[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) xr[i] = X[m0 * 32 + rg * RT + i];
            const T* lrow = La + m0 * PP + cg;
#pragma unroll
            for (int k = 0; k < CT; ++k) {
                const T l = lrow[64 * k];
#pragma unroll
                for (int i = 0; i < RT; ++i) acc[i][k] = fma(xr[i], l, acc[i][k]);
            }
        }
        // weights of the columns and partial sums for this thread's four targets (the tree
        // over the 64 column threads stays in T: B300's FP64 pipe is a small fraction of FP32)
        T part[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T* tb = TB + (rg * 4 + j) * 4 * PS;
            T sp = T(0), sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
            for (int k = 0; k < CT; ++k) {
                const int col = cg + 64 * k, m1 = col / P, m2 = col - m1 * P;
                const T ty = tb[m1], dy = tb[PS + m1], tz = tb[2 * PS + m2], dz = tb[3 * PS + m2];
                const T a0 = acc[2 * j][k], a1 = acc[2 * j + 1][k];
                const T w = ty * tz;
                sp = fma(a0, w, sp);
                sx = fma(a1, w, sx);
                sy = fma(a0, dy * tz, sy);
                sz = fma(a0, ty * dz, sz);
            }
            part[j][0] = sp;
            part[j][1] = sx;
            part[j][2] = sy;
            part[j][3] = sz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) part[j][q] += __shfl_xor_sync(0xffffffffu, part[j][q], o);
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) red[(rg * 2 + half) * 16 + j * 4 + q] = double(part[j][q]);
        __syncthreads();
        if (tid < 16) {
            const int t = tid;  // target of the chunk: row group t / 4, slot t % 4
            const int g = t >> 2, j = t & 3;
            if (t < nt) {
                double v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = red[(g * 2) * 16 + j * 4 + q] + red[(g * 2 + 1) * 16 + j * 4 + q];
                const size_t o = size_t(e.y + t0 + t);
                pot[o] = v[0];
                if (grad) {
                    grad[o * 3 + 0] = v[1] * sc;
                    grad[o * 3 + 1] = v[2] * sc;
                    grad[o * 3 + 2] = v[3] * sc;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ leaf evaluation
// entry int4 = (local slot, tgt_begin, tgt_count, level)
template <typename T, int D>
__global__ void __launch_bounds__(32) k_leaf_eval(const int4* __restrict__ list, const T* __restrict__ Lc,
                                                   const T* __restrict__ tgt4, double* __restrict__ pot,
                                                   double* __restrict__ grad, PwDims pd, double inv_rc) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int p = pd.p;
    // per-thread T_m and T'_m per dim, interleaved by thread (element k of thread t at
    // k * blockDim + t) so that lanes never share a bank
    T* tb = reinterpret_cast<T*>(sm) + threadIdx.x;
    const int bs = blockDim.x;
    const int4 e = list[blockIdx.x];
    const T* a = Lc + size_t(e.x) * pd.np;
    const double sc = 2.0 * inv_rc * double(1LL << e.w);  // dt/dx = 2/h
    for (int t0 = 0; t0 < e.z; t0 += blockDim.x) {
        const int ti = t0 + threadIdx.x;
        if (ti >= e.z) break;
        const T* x = tgt4 + size_t(e.y + ti) * 4;
        for (int i = 0; i < D; ++i) {
            const T t = T(double(x[i]) * sc);
            T* bt = tb + i * 2 * p * bs;
            T* bd = bt + p * bs;
            // T_m by recurrence; T'_m = m U_{m-1}
            T tm1 = T(1), tm = t, um1 = T(1), um = T(2) * t;
            bt[0] = T(1);
            bd[0] = T(0);
            if (p > 1) { bt[bs] = t; bd[bs] = T(1); }
            for (int m = 2; m < p; ++m) {
                const T tn = fma(T(2) * t, tm, -tm1);
                bt[m * bs] = tn;
                bd[m * bs] = T(m) * um;  // U_{m-1}
                const T un = fma(T(2) * t, um, -um1);
                tm1 = tm; tm = tn;
                um1 = um; um = un;
            }
        }
        T phi = 0, g0 = 0, g1 = 0, g2 = 0;
        const T* b0 = tb;
        const T* d0 = tb + p * bs;
        const T* b1 = tb + 2 * p * bs;
        const T* d1 = tb + 3 * p * bs;
        if (D == 2) {
            for (int m0 = 0; m0 < p; ++m0) {
                T s = 0, sd = 0;
                for (int m1 = 0; m1 < p; ++m1) {
                    const T v = a[m0 * p + m1];
                    s = fma(v, b1[m1 * bs], s);
                    sd = fma(v, d1[m1 * bs], sd);
                }
                phi = fma(b0[m0 * bs], s, phi);
                g0 = fma(d0[m0 * bs], s, g0);
                g1 = fma(b0[m0 * bs], sd, g1);
            }
        } else {
            const T* b2 = tb + 4 * p * bs;
            const T* d2 = tb + 5 * p * bs;
            for (int m0 = 0; m0 < p; ++m0) {
                T s = 0, s1d = 0, s2d = 0;
                for (int m1 = 0; m1 < p; ++m1) {
                    T u = 0, ud = 0;
                    const T* row = a + (m0 * p + m1) * p;
                    for (int m2 = 0; m2 < p; ++m2) {
                        const T v = row[m2];
                        u = fma(v, b2[m2 * bs], u);
                        ud = fma(v, d2[m2 * bs], ud);
                    }
                    s = fma(b1[m1 * bs], u, s);
                    s1d = fma(d1[m1 * bs], u, s1d);
                    s2d = fma(b1[m1 * bs], ud, s2d);
                }
                phi = fma(b0[m0 * bs], s, phi);
                g0 = fma(d0[m0 * bs], s, g0);
                g1 = fma(b0[m0 * bs], s1d, g1);
                g2 = fma(b0[m0 * bs], s2d, g2);
            }
        }
        const size_t o = size_t(e.y + ti);
        pot[o] = double(phi);
        if (grad) {
            grad[o * D + 0] = double(g0) * sc;
            grad[o * D + 1] = double(g1) * sc;
            if (D == 3) grad[o * D + 2] = double(g2) * sc;
        }
    }
}

// ------------------------------------------------------------------ 2D compile-time kernels
// The orders the planner picks by eps, (P, K) = (16, 9), (24, 16), (32, 23), get kernels with
// compile-time loop bounds: fully unrolled contractions, no run-time integer division, lanes
// along the contiguous index of every shared-memory operand.

// Outgoing plane waves of one box from its moments q (shared memory), by the calling block.
// The Chebyshev coefficients of exp(-i a t) are real for even m (the cosine) and imaginary
// for odd m (the sine), even and odd in k respectively:
//   Co[k][2j] = ce[|k|][j],  Co[k][2j+1] = i sgn(k) so[|k|][j].
// Stage 1: A[k0][m1] = sum_m0 Co[k0][m0] Q[m0][m1]      (A.x from even m0, A.y from odd m0)
// Stage 2: E = sum_j ce[k1][j] A[k0][2j],  O = sum_j so[k1][j] A[k0][2j+1]  (k1 >= 0),
//          out[k0][+-k1] = E +- i O.
// Shared scratch (T): ce, so [K+1][P/2] (rows by k), ceT, soT [P/2][K+1] (rows by j), and
// A [K+1][P] complex.  Ends with the block's stores issued.
template <typename T, int P, int K>
__device__ void pw_out_box(const T* q, T* scratch, const C2<T>* __restrict__ Cog, C2<T>* __restrict__ o) {
    constexpr int N1 = 2 * K + 1, H = P / 2, KH = K + 1;
    T* ce = scratch;           // [KH][H]
    T* so = ce + KH * H;       // [KH][H]
    T* ceT = so + KH * H;      // [H][KH]
    T* soT = ceT + H * KH;     // [H][KH]
    C2<T>* A = reinterpret_cast<C2<T>*>(soT + H * KH);  // [KH][P]
    for (int i = threadIdx.x; i < KH * H; i += blockDim.x) {
        const int k = i / H, j = i % H;
        const T e = Cog[(k + K) * P + 2 * j].x, od = Cog[(k + K) * P + 2 * j + 1].y;
        ce[k * H + j] = e;
        so[k * H + j] = od;
        ceT[j * KH + k] = e;
        soT[j * KH + k] = od;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < KH * P; it += blockDim.x) {
        const int k0 = it / P, m1 = it % P;
        T ax = T(0), ay = T(0);
#pragma unroll
        for (int j = 0; j < H; ++j) {
            ax = fma(ce[k0 * H + j], q[(2 * j) * P + m1], ax);
            ay = fma(so[k0 * H + j], q[(2 * j + 1) * P + m1], ay);
        }
        A[k0 * P + m1] = C2<T>{ax, ay};
    }
    __syncthreads();
    for (int it = threadIdx.x; it < KH * KH; it += blockDim.x) {
        const int k0 = it / KH, k1 = it % KH;
        T ex = T(0), ey = T(0), ox = T(0), oy = T(0);
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const C2<T> ae = A[k0 * P + 2 * j], ao = A[k0 * P + 2 * j + 1];
            const T c = ceT[j * KH + k1], s = soT[j * KH + k1];
            ex = fma(c, ae.x, ex);
            ey = fma(c, ae.y, ey);
            ox = fma(s, ao.x, ox);
            oy = fma(s, ao.y, oy);
        }
        // i O = (-oy, ox)
        o[k0 * N1 + K + k1] = C2<T>{ex - oy, ey + ox};
        if (k1 > 0) o[k0 * N1 + K - k1] = C2<T>{ex + oy, ey - ox};
    }
}

// Direct moments of the boxes that send outgoing plane waves:
//   Q_b[m0][m1] = sum_{y in b} q_y T_m0(t0(y)) T_m1(t1(y)),  t = 2 (y - c_b) / h_b,
// the same polynomial projection the merges of the child moments produce (the re-expansions
// S_b are exact), taken straight from the sources so that the upward pass is one launch with
// no level-to-level dependence.  The box coordinate t is the leaf-relative coordinate scaled
// to the box plus the leaf centre's offset, (2 i_leaf + 1) 2^(l_b - l_leaf) - (2 i_b + 1),
// which is exact in T.  One block per (box, segment of at most kDirectSeg sources); eight
// groups of 16 threads split the segment, each thread owns a (P/4) x (P/4) tile; the group
// partials meet in shared memory.  A box of one segment goes straight on to its outgoing
// plane waves; a box of several writes partials to its slots, and the block that completes
// the box sums them in slot order and computes the outgoing waves.
constexpr int kDirectSeg = 1024;
template <typename T>
struct V2;
template <>
struct V2<float> {
    using type = float2;
};
template <>
struct V2<double> {
    using type = double2;
};

template <typename T, int P, int K>
__global__ void __launch_bounds__(128) k_moments_direct2d(const int4* __restrict__ items, const int4* __restrict__ obox,
                                                          const T* __restrict__ src4,
                                                          const int* __restrict__ src_leaf,
                                                          const int4* __restrict__ bcoord, T* __restrict__ part,
                                                          int* __restrict__ seg_done, C2<T>* __restrict__ out,
                                                          const C2<T>* __restrict__ Cog, double inv_rc) {
    using T2 = typename V2<T>::type;
    // row stride: an odd number of pairs (conflict-free row stores), and rows s, s + 1 (the two
    // 16-lane groups of a warp) offset by 2 mod 32 words so their tile loads use disjoint banks
    constexpr int TP = P / 4, S = (P == 24) ? 34 : P + 2, NS = 128, PP = P * P;
    static_assert(P % 8 == 0 && (S / 2) % 2 == 1, "row stride");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* A = reinterpret_cast<T*>(smraw);  // [NS][S]  q T_m(t0)
    T* B = A + NS * S;                   // [NS][S]  T_m(t1)
    const int4 it = items[blockIdx.x];   // (first source, count, partial slot, out slot)
    const int4 ob = obox[it.w];          // (first partial slot, segments, box, -)
    const int4 bc = bcoord[ob.z];        // (i0, i1, level, -)
    const T scale = T(2.0 * inv_rc * double(1LL << bc.z));
    const T ob0 = T(2 * bc.x + 1), ob1 = T(2 * bc.y + 1);
    const int grp = threadIdx.x >> 4, ti = (threadIdx.x >> 2) & 3, tj = threadIdx.x & 3;
    T acc[TP][TP];
#pragma unroll
    for (int r = 0; r < TP; ++r)
#pragma unroll
        for (int c = 0; c < TP; ++c) acc[r][c] = T(0);
    for (int c0 = 0; c0 < it.y; c0 += NS) {
        const int ns = min(NS, it.y - c0);
        __syncthreads();
        if (threadIdx.x < ns) {
            const int j = it.x + c0 + threadIdx.x;
            const T* y = src4 + size_t(j) * 4;
            const int4 lc = bcoord[src_leaf[j]];
            const T sh = T(1) / T(1 << (lc.z - bc.z));  // exact power of two
            const T t0 = fma(y[0], scale, fma(T(2 * lc.x + 1), sh, -ob0));
            const T t1 = fma(y[1], scale, fma(T(2 * lc.y + 1), sh, -ob1));
            const T q = y[3];
            T2* ra = reinterpret_cast<T2*>(A + threadIdx.x * S);
            T2* rb = reinterpret_cast<T2*>(B + threadIdx.x * S);
            T a0 = q, a1 = q * t0, b0 = T(1), b1 = t1;
            const T x0 = t0 + t0, x1 = t1 + t1;
#pragma unroll
            for (int m = 0; m < P; m += 2) {
                ra[m / 2] = T2{a0, a1};
                rb[m / 2] = T2{b0, b1};
                a0 = fma(x0, a1, -a0);
                a1 = fma(x0, a0, -a1);
                b0 = fma(x1, b1, -b0);
                b1 = fma(x1, b0, -b1);
            }
        }
        __syncthreads();
        for (int s = grp; s < ns; s += 8) {
            T a[TP], b[TP];
            const T2* ra = reinterpret_cast<const T2*>(A + s * S + ti * TP);
            const T2* rb = reinterpret_cast<const T2*>(B + s * S + tj * TP);
#pragma unroll
            for (int u = 0; u < TP / 2; ++u) {
                const T2 va = ra[u], vb = rb[u];
                a[2 * u] = va.x;
                a[2 * u + 1] = va.y;
                b[2 * u] = vb.x;
                b[2 * u + 1] = vb.y;
            }
#pragma unroll
            for (int r = 0; r < TP; ++r)
#pragma unroll
                for (int c = 0; c < TP; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
    }
    __syncthreads();
    T* red = A;  // [8][PP] (fits in the staging rows)
#pragma unroll
    for (int r = 0; r < TP; ++r)
#pragma unroll
        for (int c = 0; c < TP; ++c) red[grp * PP + (ti * TP + r) * P + tj * TP + c] = acc[r][c];
    __syncthreads();
    T* q = red + 8 * PP;  // the box's moments [PP]
    T* scr = q + PP;      // outgoing-transform scratch
    for (int i = threadIdx.x; i < PP; i += blockDim.x) {
        T s = T(0);
#pragma unroll
        for (int g = 0; g < 8; ++g) s += red[g * PP + i];
        q[i] = s;
        if (ob.y > 1) part[size_t(it.z) * PP + i] = s;
    }
    if (ob.y > 1) {
        // several segments: the block that completes the box sums the partials in slot order
        // (the counter only decides which block does it) and goes on to the outgoing waves
        __shared__ int s_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(seg_done + it.w, 1) == ob.y - 1;
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        for (int i = threadIdx.x; i < PP; i += blockDim.x) {
            const T* src = part + size_t(ob.x) * PP + i;
            T s = __ldcg(src);
            for (int u = 1; u < ob.y; ++u) s += __ldcg(src + size_t(u) * PP);
            q[i] = s;
        }
    }
    __syncthreads();
    pw_out_box<T, P, K>(q, scr, Cog, out + size_t(it.w) * ((K + 1) * (2 * K + 1)));
}

// translation + incoming, one block per box (list entry: local slot, level, 9 out slots).
// Stage 1 sums the colleagues' outgoing waves with the translation phases for the pair of
// modes (k0, +-k1) at once.  The phases factor by dimension, exp(-i (2 pi/3) k.delta) =
// v^delta0 u^delta1 with u = exp(-i (2 pi/3) k1), v = exp(-i (2 pi/3) k0), and for
// delta in {-1, 0, 1}:  u X_+ + conj(u) X_- = Re(u) (X_+ + X_-) + i Im(u) (X_+ - X_-).
// The mode pair is kept as Sp = I(+k1) + I(-k1), Sm = I(+k1) - I(-k1), which is what the
// parity of Co needs (conj(Co[k][2j]) = ce[|k|][j], conj(Co[k][2j+1]) = -i sgn(k) so[|k|][j]):
// Stage 2: Ap[k0][2j] = sum_k1 ce[k1][j] Sp[k0][k1],  Ap[k0][2j+1] = -i sum_k1 so[k1][j] Sm[k0][k1]
// Stage 3: a[2j][m1] += sum_k0 w ce[k0][j] Re Ap[k0][m1],  a[2j+1][m1] += sum_k0 w so[k0][j] Im Ap[k0][m1]
// (w = 1 for k0 = 0, else 2: the Hermitian half of the k0 axis).
template <typename T, int P, int K>
__global__ void __launch_bounds__(128) k_pw_in2d_p(const int* __restrict__ list, int nbox, const C2<T>* __restrict__ out,
                                                   T* __restrict__ Lc, const C2<T>* __restrict__ Cog,
                                                   const C2<T>* __restrict__ phg, const T* __restrict__ fk) {
    constexpr int N1 = 2 * K + 1, NPW = (K + 1) * N1, H = P / 2, KH = K + 1;
    __shared__ T ce[KH][H], so[KH][H];
    __shared__ C2<T> Sp[KH][KH], Sm[KH][KH];
    __shared__ C2<T> Ap[KH][P];
    __shared__ C2<T> u[KH];
    __shared__ int coll[9];
    for (int i = threadIdx.x; i < KH * H; i += blockDim.x) {
        const int k = i / H, j = i % H;
        ce[k][j] = Cog[(k + K) * P + 2 * j].x;
        so[k][j] = Cog[(k + K) * P + 2 * j + 1].y;
    }
    for (int i = threadIdx.x; i < KH; i += blockDim.x) u[i] = phg[2 * N1 + K + i];  // delta = +1
    const T wlev = T(1.0 / 9.0);
    {
        const int b = blockIdx.x;  // one block per box
        if (b >= nbox) return;
        const int* e = list + size_t(b) * 11;
        __syncthreads();
        if (threadIdx.x < 9) coll[threadIdx.x] = e[2 + threadIdx.x];
        __syncthreads();
        for (int it = threadIdx.x; it < KH * KH; it += blockDim.x) {
            const int k0 = it / KH, k1 = it % KH;
            const T fw = fk[k0 * N1 + K + k1] * wlev;
            C2<T> ip{T(0), T(0)}, im{T(0), T(0)};
            if (fw != T(0)) {
                const C2<T> uu = u[k1], vv = u[k0];
                C2<T> rp[3], rm[3];  // per delta0 row: sums over delta1
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int sm_ = coll[r], s0 = coll[r + 3], sp = coll[r + 6];
                    const size_t op = size_t(k0) * N1 + K + k1, om = size_t(k0) * N1 + K - k1;
                    const C2<T> z{T(0), T(0)};
                    const C2<T> pP = sp >= 0 ? out[size_t(sp) * NPW + op] : z;
                    const C2<T> pM = sm_ >= 0 ? out[size_t(sm_) * NPW + op] : z;
                    const C2<T> p0 = s0 >= 0 ? out[size_t(s0) * NPW + op] : z;
                    const C2<T> mP = sp >= 0 ? out[size_t(sp) * NPW + om] : z;
                    const C2<T> mM = sm_ >= 0 ? out[size_t(sm_) * NPW + om] : z;
                    const C2<T> m0 = s0 >= 0 ? out[size_t(s0) * NPW + om] : z;
                    // +k1: p0 + Re(u) (pP + pM) + i Im(u) (pP - pM)
                    rp[r].x = p0.x + uu.x * (pP.x + pM.x) - uu.y * (pP.y - pM.y);
                    rp[r].y = p0.y + uu.x * (pP.y + pM.y) + uu.y * (pP.x - pM.x);
                    // -k1: u -> conj(u)
                    rm[r].x = m0.x + uu.x * (mP.x + mM.x) + uu.y * (mP.y - mM.y);
                    rm[r].y = m0.y + uu.x * (mP.y + mM.y) - uu.y * (mP.x - mM.x);
                }
                ip.x = fw * (rp[1].x + vv.x * (rp[2].x + rp[0].x) - vv.y * (rp[2].y - rp[0].y));
                ip.y = fw * (rp[1].y + vv.x * (rp[2].y + rp[0].y) + vv.y * (rp[2].x - rp[0].x));
                im.x = fw * (rm[1].x + vv.x * (rm[2].x + rm[0].x) - vv.y * (rm[2].y - rm[0].y));
                im.y = fw * (rm[1].y + vv.x * (rm[2].y + rm[0].y) + vv.y * (rm[2].x - rm[0].x));
            }
            if (k1 == 0) {
                Sp[k0][0] = ip;  // the +-k1 modes coincide
                Sm[k0][0] = C2<T>{T(0), T(0)};
            } else {
                Sp[k0][k1] = C2<T>{ip.x + im.x, ip.y + im.y};
                Sm[k0][k1] = C2<T>{ip.x - im.x, ip.y - im.y};
            }
        }
        __syncthreads();
        for (int it = threadIdx.x; it < KH * H; it += blockDim.x) {
            const int k0 = it / H, j = it % H;
            T ex = T(0), ey = T(0), ox = T(0), oy = T(0);
#pragma unroll
            for (int k1 = 0; k1 < KH; ++k1) {
                const C2<T> sp = Sp[k0][k1], sm_ = Sm[k0][k1];
                const T c = ce[k1][j], s = so[k1][j];
                ex = fma(c, sp.x, ex);
                ey = fma(c, sp.y, ey);
                ox = fma(s, sm_.x, ox);
                oy = fma(s, sm_.y, oy);
            }
            Ap[k0][2 * j] = C2<T>{ex, ey};
            Ap[k0][2 * j + 1] = C2<T>{oy, -ox};  // -i (ox + i oy)
        }
        __syncthreads();
        T* a = Lc + size_t(e[0]) * (P * P);
        for (int it = threadIdx.x; it < H * P; it += blockDim.x) {
            const int j = it / P, m1 = it % P;
            T ae = T(0), ao = T(0);
#pragma unroll
            for (int k0 = 0; k0 < KH; ++k0) {
                const C2<T> v = Ap[k0][m1];
                const T w = k0 == 0 ? T(1) : T(2);
                ae = fma(w * ce[k0][j], v.x, ae);
                ao = fma(w * so[k0][j], v.y, ao);
            }
            a[(2 * j) * P + m1] = ae;  // each in-box has one entry: written, not added
            a[(2 * j + 1) * P + m1] = ao;
        }
    }
}

// ------------------------------------------------------------------ single-launch downward pass
// The per-level downward launches are replaced (2D compile-time orders) by one kernel whose
// blocks take the down items in top-down order from an atomic counter.  An item (parent P,
// its four children) needs P's coefficients complete, i.e. the item that wrote P finished;
// that item has a smaller index, so it was taken earlier by a running block, which never
// waits on a later item: the wait always ends.  It is still bounded (about 1 s of
// %globaltimer); on expiry the block raises the host-visible error flag and skips, and every
// later waiter sees the flag and skips at once.  Children that are target leaves are
// evaluated by the same block right after their coefficients are formed (shared memory),
// so the leaf coefficients never go back to global memory.
struct DownItem {
    int parent;  // local slot of the parent
    int wait;    // item whose completion makes the parent's coefficients final, or -1
    int level;   // level of the children
    int pad;
    int child[4];  // local slots (-1: no child with targets)
    int tb[4];     // child that is a target leaf: first sorted target
    int tc[4];     //   and its target count (0: not a target leaf)
};

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T, int P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_down_persist2d(const DownItem* __restrict__ items, int nitems,
                                                        int* __restrict__ counter, int* __restrict__ flags, int* err,
                                                        int* __restrict__ err_dev,
                                                        T* __restrict__ Lc, const T* __restrict__ Sg,
                                                        const T* __restrict__ tgt4, double* __restrict__ pot,
                                                        double* __restrict__ grad, double inv_rc,
                                                        unsigned long long limit_ns) {
    constexpr int PP = P * P, G = (P + 3) / 4, R = P / 4;
    static_assert(P % 4 == 0, "rows are split four ways");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Sm = reinterpret_cast<T*>(smraw);  // S[b][M][m]   [2 PP]
    T* ap = Sm + 2 * PP;                  // parent       [PP]
    T* U = ap + PP;                       // U_b1[M0][m1] [2 PP]
    T* Lch = U + 2 * PP;                  // children     [4 PP]
    __shared__ DownItem s_it;
    __shared__ int s_item, s_ok;
    for (int i = threadIdx.x; i < 2 * PP; i += blockDim.x) Sm[i] = Sg[i];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int i = atomicAdd(counter, 1);
            if (i < nitems) s_it = items[i];
            s_item = i;
        }
        __syncthreads();
        if (s_item >= nitems) break;
        // the children's own coefficients (written by the incoming kernel) load while the
        // parent may still be pending; a leaf holds no incoming of its own
        for (int idx = threadIdx.x; idx < 4 * PP; idx += blockDim.x) {
            const int c = idx / PP, cs = s_it.child[c];
            Lch[idx] = (cs >= 0 && s_it.tc[c] == 0) ? __ldcg(Lc + size_t(cs) * PP + (idx - c * PP)) : T(0);
        }
        if (threadIdx.x == 0) {
            int ok = 1;
            {
                const int w = s_it.wait;
                if (w >= 0 && ld_relaxed_gpu(flags + w) == 0) {
                    // poll with relaxed loads (an L2 round trip each); one fence once seen
                    const unsigned long long t0 = global_ns();
                    for (;;) {
                        // (the device copy of the error flag: host-mapped memory is far too
                        // slow to poll)
                        if (ld_relaxed_gpu(err_dev) != 0 || global_ns() - t0 > limit_ns) {
                            ok = 0;
                            break;
                        }
                        if (ld_relaxed_gpu(flags + w) != 0) break;
                    }
                    if (!ok) {
                        st_relaxed_gpu(err_dev, 1);
                        *reinterpret_cast<volatile int*>(err) = 1;
                        __threadfence_system();
                    }
                }
                __threadfence();  // order the flag read before the block's reads of the parent
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) continue;
        // parent coefficients (written by another block: read through L2)
        const T* src = Lc + size_t(s_it.parent) * PP;
        for (int i = threadIdx.x; i < PP; i += blockDim.x) ap[i] = __ldcg(src + i);
        __syncthreads();
        // U_b1[M0][m1] = sum_M1 S_b1[M1][m1] a_P[M0][M1]   (lanes along m1)
        for (int it = threadIdx.x; it < 2 * G * P; it += blockDim.x) {
            const int b1 = it / (G * P), rem = it % (G * P), g = rem / P, m1 = rem % P;
            T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int M1 = 0; M1 < P; ++M1) {
                const T s = Sm[(b1 * P + M1) * P + m1];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma(s, ap[(g * 4 + j) * P + M1], acc[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) U[b1 * PP + (g * 4 + j) * P + m1] = acc[j];
        }
        __syncthreads();
        // child (b0, b1): own + sum_M0 S_b0[M0][m0] U_b1[M0][m1]
        for (int it = threadIdx.x; it < 4 * G * P; it += blockDim.x) {
            const int c = it / (G * P), rem = it % (G * P), g = rem / P, m1 = rem % P;
            const int cs = s_it.child[c];
            if (cs < 0) continue;
            const int b0 = c & 1, b1 = c >> 1;
            T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int M0 = 0; M0 < P; ++M0) {
                const T u = U[b1 * PP + M0 * P + m1];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma(Sm[(b0 * P + M0) * P + g * 4 + j], u, acc[j]);
            }
            const bool leaf = s_it.tc[c] > 0;
            T* dst = Lc + size_t(cs) * PP;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = (g * 4 + j) * P + m1;
                const T v = Lch[c * PP + o] + acc[j];
                Lch[c * PP + o] = v;
                if (!leaf) dst[o] = v;
            }
        }
        // the block's stores, then one GPU-scope fence and the flag (the pattern of a grid
        // barrier: the fence after the block barrier covers every thread's stores)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_relaxed_gpu(flags + s_item, 1);
        }
        // leaf evaluation: four lanes per target, lane q takes the rows m0 = 4k + q
        const int tot = s_it.tc[0] + s_it.tc[1] + s_it.tc[2] + s_it.tc[3];
        const double sc = 2.0 * inv_rc * double(1LL << s_it.level);
        const int q = threadIdx.x & 3;
        for (int base = 0; base < tot; base += 64) {
            const int pi = base + (threadIdx.x >> 2);
            const bool act = pi < tot;
            T phi = 0, g0 = 0, g1 = 0;
            int c = 0, t = pi;
            if (act) {
                while (c < 3 && t >= s_it.tc[c]) {
                    t -= s_it.tc[c];
                    ++c;
                }
                const T* x = tgt4 + size_t(s_it.tb[c] + t) * 4;
                const T t0 = T(double(x[0]) * sc), t1 = T(double(x[1]) * sc);
                T b1[P], d1[P];  // T_m(t1), T'_m(t1)
                {
                    T tm1 = T(1), tm = t1, um1 = T(1), um = T(2) * t1;
                    b1[0] = T(1);
                    d1[0] = T(0);
                    b1[1] = t1;
                    d1[1] = T(1);
#pragma unroll
                    for (int m = 2; m < P; ++m) {
                        const T tn = fma(T(2) * t1, tm, -tm1);
                        b1[m] = tn;
                        d1[m] = T(m) * um;
                        const T un = fma(T(2) * t1, um, -um1);
                        tm1 = tm;
                        tm = tn;
                        um1 = um;
                        um = un;
                    }
                }
                // T_m(t0), T'_m(t0) for m < 8, then the stride-4 recurrence
                // T_{m+4} = 2 T_4 T_m - T_{m-4},  T'_{m+4} = 2 T'_4 T_m + 2 T_4 T'_m - T'_{m-4}
                T tv[8], dv[8];
                tv[0] = T(1); dv[0] = T(0);
                tv[1] = t0; dv[1] = T(1);
#pragma unroll
                for (int m = 2; m < 8; ++m) {
                    tv[m] = fma(T(2) * t0, tv[m - 1], -tv[m - 2]);
                    dv[m] = fma(T(2) * t0, dv[m - 1], fma(T(2), tv[m - 1], -dv[m - 2]));
                }
                T A = q == 0 ? tv[0] : q == 1 ? tv[1] : q == 2 ? tv[2] : tv[3];
                T Am = q == 0 ? tv[4] : q == 1 ? tv[3] : q == 2 ? tv[2] : tv[1];
                T Dd = q == 0 ? dv[0] : q == 1 ? dv[1] : q == 2 ? dv[2] : dv[3];
                T Dm = q == 0 ? dv[4] : q == 1 ? dv[3] : q == 2 ? dv[2] : dv[1];  // T_{q-4} = T_{4-q}
                const T T4 = tv[4], D4 = dv[4];
                using T2 = typename V2<T>::type;
                const T* a = Lch + c * PP + q * P;
                // all R rows in one pass over m1: 2 R independent accumulation chains
                T s[R], sd[R];
#pragma unroll
                for (int k = 0; k < R; ++k) s[k] = sd[k] = T(0);
#pragma unroll
                for (int m1 = 0; m1 < P; m1 += 2) {
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const T2 v = reinterpret_cast<const T2*>(a + k * 4 * P)[m1 / 2];
                        s[k] = fma(v.x, b1[m1], s[k]);
                        sd[k] = fma(v.x, d1[m1], sd[k]);
                        s[k] = fma(v.y, b1[m1 + 1], s[k]);
                        sd[k] = fma(v.y, d1[m1 + 1], sd[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    phi = fma(A, s[k], phi);
                    g0 = fma(Dd, s[k], g0);
                    g1 = fma(A, sd[k], g1);
                    const T An = fma(T(2) * T4, A, -Am);
                    const T Dn = fma(T(2) * D4, A, fma(T(2) * T4, Dd, -Dm));
                    Am = A;
                    A = An;
                    Dm = Dd;
                    Dd = Dn;
                }
            }
            phi += __shfl_xor_sync(0xffffffffu, phi, 1);
            g0 += __shfl_xor_sync(0xffffffffu, g0, 1);
            g1 += __shfl_xor_sync(0xffffffffu, g1, 1);
            phi += __shfl_xor_sync(0xffffffffu, phi, 2);
            g0 += __shfl_xor_sync(0xffffffffu, g0, 2);
            g1 += __shfl_xor_sync(0xffffffffu, g1, 2);
            if (act && q == 0) {
                const size_t o = size_t(s_it.tb[c] + t);
                pot[o] = double(phi);
                if (grad) {
                    grad[o * 2 + 0] = double(g0) * sc;
                    grad[o * 2 + 1] = double(g1) * sc;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host side
struct PwImpl {
    PwDims dims{};
    double rc = 1;
    int KC = 1;
    // device tables (precision T as raw bytes)
    void* d_Co = nullptr;  // n1 * p complex
    void* d_S = nullptr;   // 2 p p
    void* d_ph = nullptr;  // 3 n1 complex
    void* d_f = nullptr;   // (K+1) n1^{d-1}
    // 3D compile-time orders: the modes inside the ball |k| <= 3c/pi (where f is nonzero), row
    // by row: for (k0, k1) the modes k2 = -m .. m, row[k0][k1 + K] = (offset of the row's
    // modes k2 = 0 .. m in the half-ball layout, m), m = -1 for an empty row.  The outgoing
    // kernel computes only these modes and stops at the first empty k0 slice.
    int2* d_row = nullptr;
    std::vector<int2> host_row;
    // FP32 compile-time 3D orders: the outgoing waves over the half ball k2 >= 0 only, one pair
    // (E, O) per mode (out(+-k2) = E +- i O), at offset row[k0][k1 + K].x + k2 of the box's nhalf;
    // the per-mode, per-row and per-k0 tables of k_pw_in3d_h
    int nhalf = 0;
    bool half3d = false;
    int nk0 = 0, nrowb = 0, in3d_r1 = 0;
    size_t in3d_smem = 0;
    std::vector<int> host_item;
    std::vector<double> host_fh;
    std::vector<int4> host_rowb;
    std::vector<int2> host_k0rows;
    int* d_item = nullptr;
    void* d_fh = nullptr;
    int4* d_rowb = nullptr;
    int2* d_k0rows = nullptr;
    // lists
    int4* d_leafq = nullptr;
    int nleafq = 0;
    int* d_merge = nullptr;
    std::vector<int> merge_start;  // per level, entry offsets
    int2* d_outl = nullptr;
    int nout = 0;
    int* d_inl = nullptr;
    int nin = 0;
    int* d_down = nullptr;
    std::vector<int> down_start;   // per parent level: entry offsets
    int4* d_eval = nullptr;
    int neval = 0;
    int nlevels = 1;
    // 2D compile-time orders: direct moments of the out boxes (no merges)
    bool direct2d = false;
    int4* d_ditems = nullptr;  // (first source, count, partial slot, box), largest first
    int nditems = 0;
    int* d_src_leaf = nullptr;  // leaf box of every sorted source
    int4* d_bcoord = nullptr;   // (i0, i1, level, 0) per box
    void* d_part = nullptr;     // partial moments [nditems][p p]
    void* d_part3 = nullptr;    // 3D four-way merges: parts [parents of the largest level][4][p^3]
    int* d_done3 = nullptr;     //   and per parent the number of parts written (reset by the last)
    unsigned char* d_ladd = nullptr;  // per local slot: 1 for in-boxes (the downward pass adds), 0 for leaves
    int4* d_obox = nullptr;     // per out slot: (first partial slot, segments, box, 0)
    int* d_seg_done = nullptr;  // per out slot: segments finished in this evaluation
    // single-launch downward pass with folded leaf evaluation (2D compile-time orders)
    DownItem* d_down_items = nullptr;
    int ndown_items = 0;
    int* d_down_flags = nullptr;  // [ndown_items] done flags, [+0] never set, [+1] item counter,
                                  // [+2] device copy of the error flag
    // arrays
    void* d_Q = nullptr;
    void* d_out = nullptr;
    void* d_L = nullptr;
    int64_t nq = 0, nloc = 0;
    int64_t ntgt = 0;
    std::vector<double> host_Co, host_S, host_ph, host_f;  // FP64 masters
};

template <class X>
int pw_alloc(PwPlan* pw, X** p, size_t n) {
    if (n == 0) n = 1;
    void* q = nullptr;
    if (pw->pool) {
        q = pw->pool->get(n * sizeof(X));
        if (!q) return PDMK_ERR_OOM;
    } else if (cudaMalloc(&q, n * sizeof(X)) != cudaSuccess) {
        cudaGetLastError();
        return PDMK_ERR_OOM;
    }
    pw->allocs.push_back({q, n * sizeof(X)});
    pw->device_bytes += int64_t(n * sizeof(X));
    *p = static_cast<X*>(q);
    return PDMK_OK;
}

int pw_upload_typed(PwPlan* pw, void** dst, const std::vector<double>& v, cudaStream_t s) {
    const size_t ts = pw->mixed ? 4 : 8;
    std::vector<unsigned char> buf(std::max<size_t>(v.size(), 1) * ts, 0);
    for (size_t i = 0; i < v.size(); ++i) {
        if (pw->mixed) {
            float f = float(v[i]);
            std::memcpy(&buf[i * 4], &f, 4);
        } else {
            std::memcpy(&buf[i * 8], &v[i], 8);
        }
    }
    unsigned char* p = nullptr;
    int r = pw_alloc(pw, &p, buf.size());
    if (r) return r;
    *dst = p;
    if (cudaMemcpyAsync(p, buf.data(), buf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) return PDMK_ERR_CUDA;
    return PDMK_OK;
}

template <class X>
int pw_upload(PwPlan* pw, X** dst, const std::vector<X>& v, cudaStream_t s) {
    int r = pw_alloc(pw, dst, v.size());
    if (r) return r;
    if (!v.empty() && cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PDMK_ERR_CUDA;
    return PDMK_OK;
}

PwImpl* impl(PwPlan* pw) { return static_cast<PwImpl*>(pw->impl); }

}  // namespace

void pw_plan_create(PwPlan* pw, int d, double eps, double c, const KernelTables& kt, int n_proxy, int n_pw,
                    bool mixed) {
    pw->d = d;
    pw->mixed = mixed;
    PwImpl* I = new PwImpl();
    pw->impl = I;
    // plane-wave half width: xi_max = (pi/3) K / (h/2) >= 2c/h  <=>  K >= 3c/pi
    const int K = n_pw > 0 ? n_pw : int(std::ceil(3.0 * c / kPi - 1e-9));
    // Chebyshev order: the plane waves exp(-i (pi/3) k t), |k| <= K, have frequency <= c
    int p = n_proxy > 0 ? n_proxy : ((int(std::ceil(c)) + 6 + 3) / 4) * 4;
    p = std::max(4, std::min(p, 40));
    pw->p = p;
    pw->K = K;
    PwDims& D = I->dims;
    D.d = d;
    D.p = p;
    D.K = K;
    D.n1 = 2 * K + 1;
    D.pd1 = (d == 3) ? p * p : p;
    D.np = D.pd1 * p;
    D.nk1 = (d == 3) ? D.n1 * D.n1 : D.n1;
    D.npw = (K + 1) * D.nk1;
    (void)eps;
    // Chebyshev nodes of the first kind and the discrete transform T_m(t_g)
    std::vector<double> tg(p);
    for (int g = 0; g < p; ++g) tg[g] = std::cos(kPi * (2.0 * g + 1.0) / (2.0 * p));
    auto Tm = [](int m, double t) { return std::cos(m * std::acos(std::max(-1.0, std::min(1.0, t)))); };
    auto cheb_coef = [&](auto f, int m) {  // coefficient m of the degree-(p-1) interpolant of f
        std::complex<double> s = 0;
        for (int g = 0; g < p; ++g) s += f(tg[g]) * Tm(m, tg[g]);
        return s * ((m == 0 ? 1.0 : 2.0) / p);
    };
    I->host_Co.assign(size_t(D.n1) * p * 2, 0.0);
    for (int kk = 0; kk < D.n1; ++kk) {
        const int k = kk - K;
        for (int m = 0; m < p; ++m) {
            auto f = [&](double t) { return std::exp(std::complex<double>(0.0, -kPi / 3.0 * k * t)); };
            std::complex<double> v = cheb_coef(f, m);
            I->host_Co[(kk * p + m) * 2 + 0] = v.real();
            I->host_Co[(kk * p + m) * 2 + 1] = v.imag();
        }
    }
    I->host_S.assign(size_t(2) * p * p, 0.0);
    for (int b = 0; b < 2; ++b)
        for (int M = 0; M < p; ++M)
            for (int m = 0; m < p; ++m) {
                const double sft = b ? 1.0 : -1.0;
                auto f = [&](double t) { return std::complex<double>(Tm(M, (t + sft) / 2.0), 0.0); };
                double v = (m <= M) ? cheb_coef(f, m).real() : 0.0;
                I->host_S[(b * p + M) * p + m] = v;
            }
    // the register-tiled 3D orders read S from constant memory (the same values for every plan
    // of this order and precision)
    if (d == 3 && ((mixed && (p == 16 || p == 24)) || (!mixed && p == 16))) {
        if (mixed) {
            std::vector<float> sf(I->host_S.begin(), I->host_S.end());
            if (p == 16) cudaMemcpyToSymbol(c_shift_f16, sf.data(), sf.size() * sizeof(float));
            else cudaMemcpyToSymbol(c_shift_f24, sf.data(), sf.size() * sizeof(float));
        } else {
            cudaMemcpyToSymbol(c_shift_d16, I->host_S.data(), I->host_S.size() * sizeof(double));
        }
    }
    I->host_ph.assign(size_t(3) * D.n1 * 2, 0.0);
    for (int dl = 0; dl < 3; ++dl)
        for (int kk = 0; kk < D.n1; ++kk) {
            const int k = kk - K, delta = dl - 1;
            // colleague at c_S = c_T + delta h: phase exp(i xi (c_T - c_S)) = exp(-i (2 pi/3) k delta)
            I->host_ph[(dl * D.n1 + kk) * 2 + 0] = std::cos(-2.0 * kPi / 3.0 * k * delta);
            I->host_ph[(dl * D.n1 + kk) * 2 + 1] = std::sin(-2.0 * kPi / 3.0 * k * delta);
        }
    // f(|k|) on the half grid, zero outside the ball |k| <= 3c/pi (Eq. (2.6) for D_l)
    const double kball = 3.0 * c / kPi;
    I->host_f.assign(size_t(D.npw), 0.0);
    for (int k0 = 0; k0 <= K; ++k0)
        for (int r = 0; r < D.nk1; ++r) {
            const int k1 = ((d == 3) ? r / D.n1 : r) - K;
            const int k2 = (d == 3) ? (r % D.n1) - K : 0;
            const double kk = std::sqrt(double(k0) * k0 + double(k1) * k1 + double(k2) * k2);
            double f = 0;
            if (kk <= kball) {
                if (kk == 0) {
                    f = 3.0 * kt.mu2 / 8.0;
                } else {
                    const double x = 2.0 * kPi * kk / 3.0;
                    f = (kt.what(0.5 * x) - kt.what(x)) / (x * x);
                }
            }
            I->host_f[size_t(k0) * D.nk1 + r] = f;
        }
    if (d == 3) {
        I->host_row.assign(size_t(K + 1) * D.n1, make_int2(0, -1));
        int off = 0;
        for (int k0 = 0; k0 <= K; ++k0)
            for (int kk1 = 0; kk1 < D.n1; ++kk1) {
                const int k1 = kk1 - K;
                int m = -1;
                for (int k2 = 0; k2 <= K; ++k2) {
                    const double kk = std::sqrt(double(k0) * k0 + double(k1) * k1 + double(k2) * k2);
                    if (kk <= kball) m = k2;  // the same test as f: the ball is convex along k2
                }
                I->host_row[size_t(k0) * D.n1 + kk1] = make_int2(off, m);
                off += m + 1;
            }
        I->nhalf = off;
        // the half-ball modes in that order: (k0, k1 + K, k2) and f(|k|), doubled for k2 > 0
        I->host_item.clear();
        I->host_fh.clear();
        for (int k0 = 0; k0 <= K; ++k0)
            for (int kk1 = 0; kk1 < D.n1; ++kk1)
                for (int k2 = 0; k2 <= I->host_row[size_t(k0) * D.n1 + kk1].y; ++k2) {
                    I->host_item.push_back(k0 | (kk1 << 8) | (k2 << 16));
                    const double f = I->host_f[size_t(k0) * D.nk1 + size_t(kk1) * D.n1 + K + k2];
                    I->host_fh.push_back(k2 > 0 ? 2.0 * f : f);
                }
        // rows (k0, k1 >= 0) of the k2 contraction: per k0 the rows k1 = 0, 1, .. that meet the
        // ball (a contiguous range, the ball being convex), as (k0 | k1 << 8 | m << 16, offset of
        // row +k1, offset of row -k1, 0); per k0 (first row, count); nk0 slices meet the ball
        I->host_rowb.clear();
        I->host_k0rows.assign(size_t(K + 1), make_int2(0, 0));
        I->nk0 = 0;
        for (int k0 = 0; k0 <= K; ++k0) {
            I->host_k0rows[k0].x = int(I->host_rowb.size());
            for (int k1 = 0; k1 <= K; ++k1) {
                const int2 rp = I->host_row[size_t(k0) * D.n1 + K + k1];
                const int2 rn = I->host_row[size_t(k0) * D.n1 + K - k1];
                if (rp.y < 0) break;
                I->host_rowb.push_back(make_int4(k0 | (k1 << 8) | (rp.y << 16), rp.x, rn.x, 0));
            }
            I->host_k0rows[k0].y = int(I->host_rowb.size()) - I->host_k0rows[k0].x;
            if (I->host_k0rows[k0].y > 0) I->nk0 = k0 + 1;
        }
        I->nrowb = int(I->host_rowb.size());
        // FP32 plans of the compile-time orders keep the waves over the half ball when the
        // incoming kernel's shared memory fits
        if (mixed && ((p == 16 && K == 9) || (p == 24 && K == 16))) {
            const size_t r1 = std::max(size_t(I->nhalf) * 4, size_t(I->nk0) * p * p * 2);  // floats
            const size_t smem = (r1 + size_t(I->nrowb) * (p + 1) * 4) * sizeof(float);
            int dev = 0, optin = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (smem + 8192 <= size_t(optin)) {
                I->half3d = true;
                I->in3d_r1 = int(r1);
                I->in3d_smem = smem;
            }
        }
    }
    // k0 chunk: the [KC][p^{d-1}] complex slices must fit next to the tables in shared memory
    const size_t ts = mixed ? 4 : 8;
    const size_t per = size_t(D.pd1) * 2 * ts + size_t(D.nk1) * 2 * ts;
    int kc = int(std::max<size_t>(1, (96 * 1024) / std::max<size_t>(per, 1)));
    I->KC = std::max(1, std::min({kc, 16, K + 1}));
}

bool pw_supported(const PwPlan*) { return true; }

// the 2D orders with compile-time kernels (FP64 at P = 32 would exceed the shared memory
// the static layouts assume)
// Parallel stream compaction over [0, n) in index order: count(i) items for index i, emitted
// by fill(i, first position); returns the total.  Static chunks per thread, their offsets by
// a prefix sum, so the result equals the sequential loop's.
template <class Count, class Fill>
static int64_t compact_parallel(int64_t n, Count count, Fill fill) {
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    std::vector<int64_t> part(size_t(nthr) + 1, 0);
#pragma omp parallel num_threads(nthr)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const int64_t i0 = n * tid / nthr, i1 = n * (tid + 1) / nthr;
        int64_t c = 0;
        for (int64_t i = i0; i < i1; ++i) c += count(i);
        part[size_t(tid) + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int k = 0; k < nthr; ++k) part[size_t(k) + 1] += part[size_t(k)];
        int64_t pos = part[size_t(tid)];
        for (int64_t i = i0; i < i1; ++i) {
            const int64_t ci = count(i);
            if (ci) fill(i, pos);
            pos += ci;
        }
    }
    return part[size_t(nthr)];
}

static bool direct2d_orders(const PwDims& pd, bool mixed) {
    return pd.d == 2 && ((pd.p == 16 && pd.K == 9) || (pd.p == 24 && pd.K == 16) || (pd.p == 32 && pd.K == 23 && mixed));
}

// The part of a set-up both layout builders share: the operator tables, the moment,
// outgoing-wave and local arrays, the four-way merge parts and the output arrays.
static int pw_layout_tail(PwPlan* pw, int d, int nlevels, int64_t nq, int64_t nloc, int nout, int64_t ntg,
                          cudaStream_t stream) {
    PwImpl* I = impl(pw);
    const size_t ts = pw->mixed ? 4 : 8;
    int r;
    if ((r = pw_upload_typed(pw, &I->d_Co, I->host_Co, stream))) return r;
    if ((r = pw_upload_typed(pw, &I->d_S, I->host_S, stream))) return r;
    if ((r = pw_upload_typed(pw, &I->d_ph, I->host_ph, stream))) return r;
    if ((r = pw_upload_typed(pw, &I->d_f, I->host_f, stream))) return r;
    unsigned char* p = nullptr;
    const bool leaf_tc = d == 3 && pw->mixed && pw->tensor_cores && (I->dims.p == 16 || I->dims.p == 24);
    if (leaf_tc && !pw->h_err) {
        // the tensor-core leaf evaluation's bounded wait reports through the same flag
        if (cudaHostAlloc(reinterpret_cast<void**>(&pw->h_err), sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&pw->d_err), pw->h_err, 0) != cudaSuccess) {
            cudaGetLastError();
            return PDMK_ERR_CUDA;
        }
        *pw->h_err = 0;
    }
    if ((r = pw_alloc(pw, &p, size_t(std::max<int64_t>(nq, 1)) * I->dims.np * ts))) return r;
    I->d_Q = p;
    const bool fixed3d_sz = d == 3 && ((I->dims.p == 16 && I->dims.K == 9) || (I->dims.p == 24 && I->dims.K == 16));
    const size_t out_modes = I->half3d ? size_t(I->nhalf) * 2 : size_t(I->dims.npw);  // complex values per box
    if ((r = pw_alloc(pw, &p, size_t(std::max(nout, 1)) * out_modes * 2 * ts))) return r;
    I->d_out = p;
    if (fixed3d_sz && (r = pw_upload(pw, &I->d_row, I->host_row, stream))) return r;
    if (I->half3d) {
        if ((r = pw_upload(pw, &I->d_item, I->host_item, stream))) return r;
        if ((r = pw_upload_typed(pw, &I->d_fh, I->host_fh, stream))) return r;
        if ((r = pw_upload(pw, &I->d_rowb, I->host_rowb, stream))) return r;
        if ((r = pw_upload(pw, &I->d_k0rows, I->host_k0rows, stream))) return r;
    }
    if ((r = pw_alloc(pw, &p, size_t(std::max<int64_t>(nloc, 1)) * I->dims.np * ts))) return r;
    I->d_L = p;
    if (d == 3 && (I->dims.p == 16 || I->dims.p == 24)) {
        int maxlev = 1;
        for (int l = 0; l < nlevels; ++l) {
            const int np_l = I->merge_start[l + 1] - I->merge_start[l];
            if (np_l < pw->nsm) maxlev = std::max(maxlev, np_l);  // levels the four-way merge takes
        }
        if ((r = pw_alloc(pw, &p, size_t(maxlev) * 4 * I->dims.np * ts))) return r;
        I->d_part3 = p;
        if ((r = pw_alloc(pw, &I->d_done3, size_t(maxlev)))) return r;
        if (cudaMemsetAsync(I->d_done3, 0, size_t(maxlev) * sizeof(int), stream) != cudaSuccess) return PDMK_ERR_CUDA;
    }
    if ((r = pw_alloc(pw, &pw->d_pot, size_t(std::max<int64_t>(ntg, 1))))) return r;
    if ((r = pw_alloc(pw, &pw->d_grad, size_t(std::max<int64_t>(ntg, 1)) * d))) return r;
    return PDMK_OK;
}


int pw_set_sources(PwPlan* pw, const Tree& t, const SortedSources& /*s*/, const std::vector<int>& leaf_of,
                   const std::vector<int>& /*tgt_leaf*/, const Geometry& g, cudaStream_t stream,
                   const int* d_leaf_of, int64_t nimg) {
    PwImpl* I = impl(pw);
    const int d = t.d;
    const int nb = int(t.level.size());
    const int nc = 1 << d;
    const int ncol = (d == 3) ? 27 : 9;
    I->rc = g.rc;
    I->nlevels = t.nlevels;
    pw->active = t.nlevels > 1;
    if (!pw->active) return PDMK_OK;
    auto has_src = [&](int b) { return t.src_end[b] > t.src_begin[b]; };
    auto has_tgt = [&](int b) { return t.tgt_end[b] > t.tgt_begin[b]; };
    // the slot and list numberings below are ranks in box order, taken by parallel
    // compaction (each equals its sequential loop's)
    // q slots: boxes with sources
    std::vector<int> qslot(nb, -1);
    int nq = int(compact_parallel(
        nb, [&](int64_t b) { return int64_t(has_src(int(b))); }, [&](int64_t b, int64_t k) { qslot[b] = int(k); }));
    // local slots: in-boxes (non-leaf boxes with targets) and boxes below the root with targets
    std::vector<int> lslot(nb, -1);
    const int nloc = int(compact_parallel(
        nb, [&](int64_t b) { return int64_t(has_tgt(int(b)) && (!t.is_leaf(int(b)) || t.level[b] >= 1)); },
        [&](int64_t b, int64_t k) { lslot[b] = int(k); }));
    pw->lslot = lslot;
    pw->local_full.assign(size_t(nb), 0);
    const bool leaves_in_smem = d == 2 && direct2d_orders(I->dims, pw->mixed);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nb; ++b)
        pw->local_full[b] = lslot[b] >= 0 && (!t.is_leaf(b) || !leaves_in_smem);
    // out slots: the colleagues with sources of the in-boxes, in box order
    auto inbox = [&](int b) { return !t.is_leaf(b) && has_tgt(b); };
    std::vector<unsigned char> is_out(size_t(nb), 0);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nb; ++b) {
        if (!inbox(b)) continue;
        for (int o = 0; o < ncol; ++o) {
            const int S = t.colleague[size_t(b) * ncol + o];
            if (S >= 0 && has_src(S)) {
#pragma omp atomic write
                is_out[size_t(S)] = 1;
            }
        }
    }
    std::vector<int> oslot(nb, -1);
    std::vector<int2> outl;
    const int nout = int(compact_parallel(
        nb, [&](int64_t b) { return int64_t(is_out[size_t(b)]); }, [&](int64_t b, int64_t k) { oslot[b] = int(k); }));
    outl.resize(size_t(nout));
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nb; ++b)
        if (oslot[b] >= 0) outl[size_t(oslot[b])] = make_int2(qslot[b], oslot[b]);
    // in-box records: local slot, level, the 27 (9) colleagues' out slots
    std::vector<int> inl;
    {
        std::vector<int> in_rank(nb, -1);
        const int64_t nin = compact_parallel(
            nb, [&](int64_t b) { return int64_t(inbox(int(b))); }, [&](int64_t b, int64_t k) { in_rank[b] = int(k); });
        inl.assign(size_t(nin) * (2 + ncol), -1);
#pragma omp parallel for schedule(static)
        for (int b = 0; b < nb; ++b) {
            if (in_rank[b] < 0) continue;
            int* e = &inl[size_t(in_rank[b]) * (2 + ncol)];
            e[0] = lslot[b];
            e[1] = t.level[b];
            for (int o = 0; o < ncol; ++o) {
                const int S = t.colleague[size_t(b) * ncol + o];
                e[2 + o] = (S >= 0 && has_src(S)) ? oslot[S] : -1;
            }
        }
    }
    I->nin = int(inl.size()) / (2 + ncol);
    I->nout = nout;
    pw->moment_sources = 0;
    // 2D compile-time orders: the out boxes' moments straight from their sources, in
    // segments of at most kDirectSeg; the out list becomes (first partial slot, count)
    I->direct2d = direct2d_orders(I->dims, pw->mixed);
    std::vector<int4> ditems, obox;
    std::vector<int> src_leaf;
    std::vector<int4> bcoord;
    if (I->direct2d) {
        std::vector<int> box_of_out(nout, -1);
        for (int b = 0; b < nb; ++b)
            if (oslot[b] >= 0) box_of_out[oslot[b]] = b;
        int npart = 0;
        obox.resize(nout);
        for (int o = 0; o < nout; ++o) {
            const int b = box_of_out[o];
            const int64_t s0 = t.src_begin[b], ns = t.src_end[b] - t.src_begin[b];
            const int first = npart;
            for (int64_t c = 0; c < ns; c += kDirectSeg)
                ditems.push_back(make_int4(int(s0 + c), int(std::min<int64_t>(kDirectSeg, ns - c)), npart++, o));
            outl[o] = make_int2(first, npart - first);
            obox[o] = make_int4(first, npart - first, b, 0);
        }
        // largest segments first: the long blocks start in the first wave
        std::stable_sort(ditems.begin(), ditems.end(), [](const int4& a, const int4& b) { return a.y > b.y; });
        I->nditems = int(ditems.size());
        src_leaf = leaf_of;
        bcoord.resize(nb);
        for (int b = 0; b < nb; ++b)
            bcoord[b] = make_int4(int(t.coord[size_t(b) * d]), int(t.coord[size_t(b) * d + 1]), t.level[b], 0);
        for (const int4& it : ditems) pw->moment_sources += it.y;
    }
    // leaf moments
    std::vector<int4> leafq;
    if (!I->direct2d) {
        auto is_lq = [&](int64_t b) { return int64_t(t.is_leaf(int(b)) && has_src(int(b))); };
        leafq.resize(size_t(compact_parallel(nb, is_lq, [](int64_t, int64_t) {})));
        compact_parallel(nb, is_lq, [&](int64_t b, int64_t k) {
            leafq[size_t(k)] = make_int4(int(t.src_begin[b]), int(t.src_end[b] - t.src_begin[b]), qslot[b], t.level[b]);
        });
    }
    I->nleafq = int(leafq.size());
    if (!I->direct2d)
        for (const int4& l : leafq) pw->moment_sources += l.y;
    // merges per level (non-leaf boxes with sources), deepest first at eval time;
    // downward lists per parent level: [parent local slot, child local slots]
    std::vector<int> merge, down;
    I->merge_start.assign(t.nlevels + 1, 0);
    I->down_start.assign(t.nlevels + 1, 0);
    auto is_mp = [&](int64_t b) { return int64_t(!I->direct2d && !t.is_leaf(int(b)) && has_src(int(b))); };
    auto is_dp = [&](int64_t b) {
        if (t.is_leaf(int(b)) || lslot[b] < 0) return int64_t(0);
        for (int c = 0; c < nc; ++c)
            if (lslot[t.child0[b] + c] >= 0) return int64_t(1);
        return int64_t(0);
    };
    for (int l = 0; l < t.nlevels; ++l) {
        const int b0 = t.level_start[l], nl = t.level_start[l + 1] - b0;
        I->merge_start[l] = int(merge.size()) / (1 + nc);
        const size_t m0 = merge.size();
        merge.resize(m0 + size_t(compact_parallel(nl, [&](int64_t i) { return is_mp(b0 + i); }, [](int64_t, int64_t) {})) *
                              (1 + nc));
        compact_parallel(nl, [&](int64_t i) { return is_mp(b0 + i); }, [&](int64_t i, int64_t k) {
            const int b = b0 + int(i);
            int* e = &merge[m0 + size_t(k) * (1 + nc)];
            e[0] = qslot[b];
            for (int c = 0; c < nc; ++c) e[1 + c] = qslot[t.child0[b] + c];
        });
        I->down_start[l] = int(down.size()) / (1 + nc);
        const size_t d0 = down.size();
        down.resize(d0 + size_t(compact_parallel(nl, [&](int64_t i) { return is_dp(b0 + i); }, [](int64_t, int64_t) {})) *
                             (1 + nc));
        compact_parallel(nl, [&](int64_t i) { return is_dp(b0 + i); }, [&](int64_t i, int64_t k) {
            const int b = b0 + int(i);
            int* e = &down[d0 + size_t(k) * (1 + nc)];
            e[0] = lslot[b];
            for (int c = 0; c < nc; ++c) e[1 + c] = lslot[t.child0[b] + c];
        });
    }
    I->merge_start[t.nlevels] = int(merge.size()) / (1 + nc);
    pw->merge_parents = I->merge_start[t.nlevels];
    I->down_start[t.nlevels] = int(down.size()) / (1 + nc);
    pw->down_parents = I->down_start[t.nlevels];
    // single-launch downward items (top-down order: the down list is by parent level)
    std::vector<DownItem> ditems_down;
    if (I->direct2d) {
        std::vector<int> box_of_lslot(nloc, -1), writer(nloc, -1);
        for (int b = 0; b < nb; ++b)
            if (lslot[b] >= 0) box_of_lslot[lslot[b]] = b;
        const int ne = I->down_start[t.nlevels];
        ditems_down.resize(ne);
        for (int i = 0; i < ne; ++i) {
            const int* e = &down[size_t(i) * (1 + nc)];
            DownItem& it = ditems_down[i];
            it.parent = e[0];
            it.wait = writer[e[0]];
            it.level = t.level[box_of_lslot[e[0]]] + 1;
            it.pad = 0;
            for (int c = 0; c < 4; ++c) {
                it.child[c] = e[1 + c];
                it.tb[c] = 0;
                it.tc[c] = 0;
                if (e[1 + c] < 0) continue;
                writer[e[1 + c]] = i;
                const int cb = box_of_lslot[e[1 + c]];
                if (t.is_leaf(cb) && has_tgt(cb) && t.level[cb] >= 1) {
                    it.tb[c] = int(t.tgt_begin[cb]);
                    it.tc[c] = int(t.tgt_end[cb] - t.tgt_begin[cb]);
                }
            }
        }
        if (pw->wait_test)  // test hook: the first dependent item waits on the never-set flag
            for (DownItem& it : ditems_down)
                if (it.wait >= 0) {
                    it.wait = ne;
                    break;
                }
        I->ndown_items = ne;
    }
    // leaf evaluation: target leaves below the root level
    std::vector<int4> ev;
    {
        auto is_ev = [&](int64_t b) { return int64_t(t.is_leaf(int(b)) && has_tgt(int(b)) && t.level[b] >= 1); };
        ev.resize(size_t(compact_parallel(nb, is_ev, [](int64_t, int64_t) {})));
        compact_parallel(nb, is_ev, [&](int64_t b, int64_t k) {
            ev[size_t(k)] = make_int4(lslot[b], int(t.tgt_begin[b]), int(t.tgt_end[b] - t.tgt_begin[b]), t.level[b]);
        });
    }
    I->neval = int(ev.size());
    pw->eval_targets = 0;
    for (const int4& e4 : ev) pw->eval_targets += e4.z;
    I->nq = nq;
    I->nloc = nloc;
    int64_t ntg = 0;
    for (int b = 0; b < t.level_start[1]; ++b) ntg += t.tgt_end[b] - t.tgt_begin[b];
    I->ntgt = ntg;
    pw->nout = nout;
    pw->nin = I->nin;
    // device
    const size_t ts = pw->mixed ? 4 : 8;
    int r;
    if ((r = pw_upload(pw, &I->d_leafq, leafq, stream))) return r;
    if ((r = pw_upload(pw, &I->d_merge, merge, stream))) return r;
    if ((r = pw_upload(pw, &I->d_outl, outl, stream))) return r;
    if ((r = pw_upload(pw, &I->d_inl, inl, stream))) return r;
    if ((r = pw_upload(pw, &I->d_down, down, stream))) return r;
    if ((r = pw_upload(pw, &I->d_eval, ev, stream))) return r;
    {
        // per local slot: does the downward pass add (in-boxes, written by the incoming
        // waves) or write (leaves)
        std::vector<unsigned char> ladd(size_t(std::max(nloc, 1)), 0);
#pragma omp parallel for schedule(static)
        for (int b = 0; b < nb; ++b)
            if (lslot[b] >= 0 && !t.is_leaf(b) && has_tgt(b)) ladd[size_t(lslot[b])] = 1;
        if ((r = pw_upload(pw, &I->d_ladd, ladd, stream))) return r;
    }
    unsigned char* p = nullptr;
    if (I->direct2d) {
        if (!pw->h_err) {
            if (cudaHostAlloc(reinterpret_cast<void**>(&pw->h_err), sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
                cudaHostGetDevicePointer(reinterpret_cast<void**>(&pw->d_err), pw->h_err, 0) != cudaSuccess) {
                cudaGetLastError();
                return PDMK_ERR_CUDA;
            }
            *pw->h_err = 0;
        }
        if ((r = pw_upload(pw, &I->d_down_items, ditems_down, stream))) return r;
        if ((r = pw_alloc(pw, &I->d_down_flags, size_t(I->ndown_items) + 3))) return r;
        if ((r = pw_upload(pw, &I->d_ditems, ditems, stream))) return r;
        if ((r = pw_upload(pw, &I->d_obox, obox, stream))) return r;
        if ((r = pw_alloc(pw, &I->d_seg_done, size_t(std::max(nout, 1))))) return r;
        if (!src_leaf.empty() || !d_leaf_of) {
            if ((r = pw_upload(pw, &I->d_src_leaf, src_leaf, stream))) return r;
        } else {
            if ((r = pw_alloc(pw, &I->d_src_leaf, size_t(std::max<int64_t>(nimg, 1))))) return r;
            if (cudaMemcpyAsync(I->d_src_leaf, d_leaf_of, size_t(nimg) * sizeof(int), cudaMemcpyDeviceToDevice,
                                stream) != cudaSuccess)
                return PDMK_ERR_CUDA;
        }
        if ((r = pw_upload(pw, &I->d_bcoord, bcoord, stream))) return r;
        if ((r = pw_alloc(pw, &p, size_t(std::max(I->nditems, 1)) * I->dims.np * ts))) return r;
        I->d_part = p;
        nq = 0;  // no per-box moments
        I->nq = 0;
    }
    return pw_layout_tail(pw, d, t.nlevels, nq, nloc, nout, ntg, stream);
}

// ------------------------------------------------------------------ layout on the device
// The lists of pw_set_sources (3D), built from the device tree: per box the flags of each
// list, exclusive scans for the slots and list positions (ranks in box order, as the host's
// compactions), then one pass that writes every record.
namespace {

__global__ void k_pwl_flags(PwTreeDev t, int* __restrict__ fq, int* __restrict__ fl, int* __restrict__ fin,
                            int* __restrict__ flq, int* __restrict__ fm, int* __restrict__ fev) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nb; b += gridDim.x * blockDim.x) {
        const bool leaf = t.child0[b] < 0, src = t.src_e[b] > t.src_b[b], tgt = t.tgt_e[b] > t.tgt_b[b];
        fq[b] = src;
        fl[b] = tgt && (!leaf || t.level[b] >= 1);
        fin[b] = !leaf && tgt;
        flq[b] = leaf && src;
        fm[b] = !leaf && src;
        fev[b] = leaf && tgt && t.level[b] >= 1;
    }
}

// the colleagues with sources of the in-boxes send outgoing waves
__global__ void k_pwl_mark_out(PwTreeDev t, int* __restrict__ fout) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nb; b += gridDim.x * blockDim.x) {
        if (t.child0[b] < 0 || t.tgt_e[b] <= t.tgt_b[b]) continue;
        for (int o = 0; o < 27; ++o) {
            const int S = t.colleague[size_t(b) * 27 + o];
            if (S >= 0 && t.src_e[S] > t.src_b[S]) fout[S] = 1;  // every writer writes 1
        }
    }
}

// downward parents: non-leaf boxes with a local slot and a child with one
__global__ void k_pwl_down_flag(PwTreeDev t, const int* __restrict__ fl, int* __restrict__ fd) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nb; b += gridDim.x * blockDim.x) {
        int f = 0;
        if (t.child0[b] >= 0 && fl[b])
            for (int c = 0; c < 8; ++c) f |= fl[t.child0[b] + c];
        fd[b] = f;
    }
}

struct PwlRanks {
    const int *fq, *qr, *fl, *lr, *fin, *inr, *fout, *outr, *flq, *lqr, *fm, *mr, *fd, *dr, *fev, *evr;
};
struct PwlOut {
    int4* leafq;
    int* merge;
    int2* outl;
    int* inl;
    int* down;
    int4* ev;
    unsigned char* ladd;
    unsigned long long* sums;  // moment sources, evaluation targets, targets of the root boxes
};

__global__ void k_pwl_fill(PwTreeDev t, int root_end, PwlRanks k, PwlOut o) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < t.nb; b += gridDim.x * blockDim.x) {
        const bool leaf = t.child0[b] < 0;
        const int lslot = k.fl[b] ? k.lr[b] : -1, qslot = k.fq[b] ? k.qr[b] : -1, lev = t.level[b];
        const long long ns = t.src_e[b] - t.src_b[b], nt = t.tgt_e[b] - t.tgt_b[b];
        if (k.fin[b]) {
            int* e = o.inl + size_t(k.inr[b]) * 29;
            e[0] = lslot;
            e[1] = lev;
            for (int c = 0; c < 27; ++c) {
                const int S = t.colleague[size_t(b) * 27 + c];
                e[2 + c] = (S >= 0 && k.fq[S]) ? k.outr[S] : -1;
            }
        }
        if (k.fout[b]) o.outl[k.outr[b]] = make_int2(qslot, k.outr[b]);
        if (k.flq[b]) {
            o.leafq[k.lqr[b]] = make_int4(int(t.src_b[b]), int(ns), qslot, lev);
            atomicAdd(&o.sums[0], static_cast<unsigned long long>(ns));
        }
        if (k.fm[b]) {
            int* e = o.merge + size_t(k.mr[b]) * 9;
            e[0] = qslot;
            for (int c = 0; c < 8; ++c) {
                const int ch = t.child0[b] + c;
                e[1 + c] = k.fq[ch] ? k.qr[ch] : -1;
            }
        }
        if (k.fd[b]) {
            int* e = o.down + size_t(k.dr[b]) * 9;
            e[0] = lslot;
            for (int c = 0; c < 8; ++c) {
                const int ch = t.child0[b] + c;
                e[1 + c] = k.fl[ch] ? k.lr[ch] : -1;
            }
        }
        if (k.fev[b]) {
            o.ev[k.evr[b]] = make_int4(lslot, int(t.tgt_b[b]), int(nt), lev);
            atomicAdd(&o.sums[1], static_cast<unsigned long long>(nt));
        }
        if (lslot >= 0 && !leaf && nt > 0) o.ladd[lslot] = 1;
        if (b < root_end) atomicAdd(&o.sums[2], static_cast<unsigned long long>(nt));
    }
}

// the scan totals and, per level boundary, the merge and downward list positions
__global__ void k_pwl_counts(int nb, const int* __restrict__ ls, int nls, PwlRanks k, int* __restrict__ out) {
    const int i = threadIdx.x;
    if (i == 0) {
        out[0] = k.qr[nb];
        out[1] = k.lr[nb];
        out[2] = k.inr[nb];
        out[3] = k.outr[nb];
        out[4] = k.lqr[nb];
        out[5] = k.mr[nb];
        out[6] = k.dr[nb];
        out[7] = k.evr[nb];
    }
    for (int j = i; j < nls; j += blockDim.x) {
        out[8 + j] = k.mr[ls[j]];
        out[8 + nls + j] = k.dr[ls[j]];
    }
}

}  // namespace

int pw_set_sources_device(PwPlan* pw, const PwTreeDev& dt, const std::vector<int>& level_start, int nlevels,
                          const Geometry& g, cudaStream_t stream) {
    PwImpl* I = impl(pw);
    I->rc = g.rc;
    I->nlevels = nlevels;
    I->direct2d = false;
    pw->active = nlevels > 1;
    pw->lslot.clear();  // filled on demand (pw_host_slots)
    pw->local_full.clear();
    if (!pw->active) return PDMK_OK;
    const int nb = dt.nb;
    const int nt = 256, nblk = int(std::min<int64_t>((int64_t(nb) + nt - 1) / nt, 1 << 16));
    // flags and their exclusive scans, nb + 1 entries each (the total at nb)
    enum { Q, L, IN, OUT, LQ, M, D, EV, NF };
    int* f[NF];
    int* rk[NF];
    int r;
    for (int k = 0; k < NF; ++k) {
        if ((r = pw_alloc(pw, &f[k], size_t(nb) + 1))) return r;
        if ((r = pw_alloc(pw, &rk[k], size_t(nb) + 1))) return r;
        if (cudaMemsetAsync(f[k], 0, (size_t(nb) + 1) * sizeof(int), stream) != cudaSuccess) return PDMK_ERR_CUDA;
    }
    k_pwl_flags<<<nblk, nt, 0, stream>>>(dt, f[Q], f[L], f[IN], f[LQ], f[M], f[EV]);
    k_pwl_mark_out<<<nblk, nt, 0, stream>>>(dt, f[OUT]);
    k_pwl_down_flag<<<nblk, nt, 0, stream>>>(dt, f[L], f[D]);
    size_t tb = 0;
    if (cub::DeviceScan::ExclusiveSum(nullptr, tb, f[Q], rk[Q], nb + 1, stream) != cudaSuccess) return PDMK_ERR_CUDA;
    unsigned char* tmp = nullptr;
    if ((r = pw_alloc(pw, &tmp, tb))) return r;
    for (int k = 0; k < NF; ++k)
        if (cub::DeviceScan::ExclusiveSum(tmp, tb, f[k], rk[k], nb + 1, stream) != cudaSuccess) return PDMK_ERR_CUDA;
    PwlRanks kr{f[Q], rk[Q], f[L], rk[L], f[IN], rk[IN], f[OUT], rk[OUT], f[LQ], rk[LQ], f[M], rk[M], f[D], rk[D],
                f[EV], rk[EV]};
    // counts and the per-level list positions
    const int nls = nlevels + 1;
    std::vector<int> ls(level_start.begin(), level_start.begin() + nls);
    int *d_ls, *d_cnt;
    if ((r = pw_upload(pw, &d_ls, ls, stream))) return r;
    if ((r = pw_alloc(pw, &d_cnt, size_t(8 + 2 * nls)))) return r;
    k_pwl_counts<<<1, 128, 0, stream>>>(nb, d_ls, nls, kr, d_cnt);
    std::vector<int> cnt(size_t(8 + 2 * nls));
    if (cudaMemcpyAsync(cnt.data(), d_cnt, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return PDMK_ERR_CUDA;
    const int nq = cnt[0], nloc = cnt[1], nin = cnt[2], nout = cnt[3], nleafq = cnt[4], nmerge = cnt[5], ndown = cnt[6],
              neval = cnt[7];
    I->merge_start.assign(cnt.begin() + 8, cnt.begin() + 8 + nls);
    I->down_start.assign(cnt.begin() + 8 + nls, cnt.begin() + 8 + 2 * nls);
    // the lists
    PwlOut o;
    if ((r = pw_alloc(pw, &I->d_leafq, size_t(std::max(nleafq, 1))))) return r;
    if ((r = pw_alloc(pw, &I->d_merge, size_t(std::max(nmerge, 1)) * 9))) return r;
    if ((r = pw_alloc(pw, &I->d_outl, size_t(std::max(nout, 1))))) return r;
    if ((r = pw_alloc(pw, &I->d_inl, size_t(std::max(nin, 1)) * 29))) return r;
    if ((r = pw_alloc(pw, &I->d_down, size_t(std::max(ndown, 1)) * 9))) return r;
    if ((r = pw_alloc(pw, &I->d_eval, size_t(std::max(neval, 1))))) return r;
    if ((r = pw_alloc(pw, &I->d_ladd, size_t(std::max(nloc, 1))))) return r;
    unsigned long long* d_sums;
    if ((r = pw_alloc(pw, &d_sums, 3))) return r;
    if (cudaMemsetAsync(I->d_ladd, 0, size_t(std::max(nloc, 1)), stream) != cudaSuccess ||
        cudaMemsetAsync(d_sums, 0, 3 * sizeof(unsigned long long), stream) != cudaSuccess)
        return PDMK_ERR_CUDA;
    o.leafq = I->d_leafq;
    o.merge = I->d_merge;
    o.outl = I->d_outl;
    o.inl = I->d_inl;
    o.down = I->d_down;
    o.ev = I->d_eval;
    o.ladd = I->d_ladd;
    o.sums = d_sums;
    k_pwl_fill<<<nblk, nt, 0, stream>>>(dt, level_start[1], kr, o);
    unsigned long long sums[3] = {0, 0, 0};
    if (cudaMemcpyAsync(sums, d_sums, sizeof(sums), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return PDMK_ERR_CUDA;
    I->nq = nq;
    I->nloc = nloc;
    I->nin = nin;
    I->nout = nout;
    I->nleafq = nleafq;
    I->neval = neval;
    I->ntgt = int64_t(sums[2]);
    pw->moment_sources = int64_t(sums[0]);
    pw->eval_targets = int64_t(sums[1]);
    pw->merge_parents = nmerge;
    pw->down_parents = ndown;
    pw->nout = nout;
    pw->nin = nin;
    return pw_layout_tail(pw, 3, nlevels, nq, nloc, nout, I->ntgt, stream);
}

void pw_host_slots(PwPlan* pw, const Tree& t) {
    if (!pw->active || !pw->lslot.empty()) return;
    const int nb = int(t.level.size());
    auto has_tgt = [&](int b) { return t.tgt_end[b] > t.tgt_begin[b]; };
    std::vector<int> lslot(nb, -1);
    compact_parallel(
        nb, [&](int64_t b) { return int64_t(has_tgt(int(b)) && (!t.is_leaf(int(b)) || t.level[b] >= 1)); },
        [&](int64_t b, int64_t k) { lslot[b] = int(k); });
    PwImpl* I = impl(pw);
    const bool leaves_in_smem = t.d == 2 && direct2d_orders(I->dims, pw->mixed);
    pw->local_full.assign(size_t(nb), 0);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nb; ++b) pw->local_full[b] = lslot[b] >= 0 && (!t.is_leaf(b) || !leaves_in_smem);
    pw->lslot.swap(lslot);
}

void pw_layout_snapshot(PwPlan* pw, std::vector<std::pair<std::string, std::vector<unsigned char>>>* out) {
    PwImpl* I = impl(pw);
    auto dev = [&](const char* name, const void* p, size_t bytes) {
        std::vector<unsigned char> v(bytes);
        if (bytes && p) cudaMemcpy(v.data(), p, bytes, cudaMemcpyDeviceToHost);
        out->push_back({name, std::move(v)});
    };
    int64_t c[12] = {I->nq, I->nloc, I->nin, I->nout, I->nleafq, I->neval, I->ntgt, pw->moment_sources,
                     pw->eval_targets, pw->merge_parents, pw->down_parents, int64_t(pw->active)};
    std::vector<unsigned char> cv(sizeof(c));
    std::memcpy(cv.data(), c, sizeof(c));
    out->push_back({"pw_counts", cv});
    if (!pw->active) return;
    std::vector<unsigned char> st((I->merge_start.size() + I->down_start.size()) * sizeof(int));
    std::memcpy(st.data(), I->merge_start.data(), I->merge_start.size() * sizeof(int));
    std::memcpy(st.data() + I->merge_start.size() * sizeof(int), I->down_start.data(),
                I->down_start.size() * sizeof(int));
    out->push_back({"pw_starts", st});
    const int nc = 1 << pw->d;
    dev("pw_leafq", I->d_leafq, size_t(I->nleafq) * sizeof(int4));
    dev("pw_merge", I->d_merge, size_t(pw->merge_parents) * (1 + nc) * sizeof(int));
    dev("pw_outl", I->d_outl, size_t(I->nout) * sizeof(int2));
    dev("pw_inl", I->d_inl, size_t(I->nin) * (pw->d == 3 ? 29 : 11) * sizeof(int));
    dev("pw_down", I->d_down, size_t(pw->down_parents) * (1 + nc) * sizeof(int));
    dev("pw_eval", I->d_eval, size_t(I->neval) * sizeof(int4));
    dev("pw_ladd", I->d_ladd, size_t(I->nloc));
}

int pw_set_charges(PwPlan*, cudaStream_t) { return PDMK_OK; }

template <typename T, int D>
static int pw_eval_t(PwPlan* pw, cudaStream_t s, int phase) {
    PwImpl* I = impl(pw);
    const PwDims pd = I->dims;
    const size_t ts = sizeof(T);
    const double inv_rc = 1.0 / I->rc;
    // compile-time 2D orders: direct moments, incoming written (not added) per in-box, and the
    // single-launch downward pass; no per-box moment or local arrays to clear
    const bool fixed2d = D == 2 && I->direct2d;
    // 3D register-tiled path (leaf moments, merges and downward pass over the triangular shift
    // matrices): every moment and local slot is written before it is read, so neither array is
    // cleared (the moments and merges write their boxes; the downward pass writes the leaves
    // and adds into the in-boxes, which the incoming waves wrote)
    const bool rpath3d = D == 3 && ((sizeof(T) == 4 && (pd.p == 16 || pd.p == 24)) || (sizeof(T) == 8 && pd.p == 16));
    if (phase == 0) {
    if (!fixed2d && !rpath3d) {
    if (cudaMemsetAsync(I->d_Q, 0, size_t(std::max<int64_t>(I->nq, 1)) * pd.np * ts, s) != cudaSuccess) return PDMK_ERR_CUDA;
    if (cudaMemsetAsync(I->d_L, 0, size_t(std::max<int64_t>(I->nloc, 1)) * pd.np * ts, s) != cudaSuccess) return PDMK_ERR_CUDA;
    }
    if (cudaMemsetAsync(pw->d_pot, 0, size_t(std::max<int64_t>(I->ntgt, 1)) * sizeof(double), s) != cudaSuccess) return PDMK_ERR_CUDA;
    if (cudaMemsetAsync(pw->d_grad, 0, size_t(std::max<int64_t>(I->ntgt, 1)) * D * sizeof(double), s) != cudaSuccess) return PDMK_ERR_CUDA;
    }
    T* Q = static_cast<T*>(I->d_Q);
    T* L = static_cast<T*>(I->d_L);
    C2<T>* out = static_cast<C2<T>*>(I->d_out);
    const C2<T>* Co = static_cast<const C2<T>*>(I->d_Co);
    const T* S = static_cast<const T*>(I->d_S);
    const size_t sm_re = ts * (2 * pd.p * pd.p + pd.pd1 + pd.p * pd.p);
    const size_t sm_m2 = ts * 10 * pd.p * pd.p;
    const size_t sm_d2 = ts * 5 * pd.p * pd.p;
    // 1. moments
    if (phase == 0 && fixed2d && I->nditems > 0) {
        const T* s4 = static_cast<const T*>(pw->d_src4);
        T* part = static_cast<T*>(I->d_part);
        if (cudaMemsetAsync(I->d_seg_done, 0, size_t(std::max(I->nout, 1)) * sizeof(int), s) != cudaSuccess)
            return PDMK_ERR_CUDA;
        C2<T>* outw = static_cast<C2<T>*>(I->d_out);
        const C2<T>* Cot = static_cast<const C2<T>*>(I->d_Co);
        auto direct = [&](auto kern, int P, int K) {
            // staging rows | (group partials, moments, outgoing scratch)
            const size_t smb = ts * std::max(2 * 128 * (P == 24 ? 34 : P + 2), 9 * P * P + 4 * (K + 1) * P);
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
            kern<<<I->nditems, 128, smb, s>>>(I->d_ditems, I->d_obox, s4, I->d_src_leaf, I->d_bcoord, part,
                                              I->d_seg_done, outw, Cot, inv_rc);
        };
        if (pd.p == 16) direct(k_moments_direct2d<T, 16, 9>, 16, 9);
        else if (pd.p == 24) direct(k_moments_direct2d<T, 24, 16>, 24, 16);
        else direct(k_moments_direct2d<T, 32, 23>, 32, 23);
        ++pw->launches;
    }
    if (phase == 0 && I->nleafq > 0) {
        const T* s4 = static_cast<const T*>(pw->d_src4);
        auto gemm = [&](auto kern, size_t smb) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
            kern<<<I->nleafq, 256, smb, s>>>(I->d_leafq, s4, Q, inv_rc);
        };
        bool tiled = false;
        if constexpr (sizeof(T) == 4) {
            const float* s4f = reinterpret_cast<const float*>(s4);
            float* Qf = reinterpret_cast<float*>(Q);
            tiled = D == 3 && (pd.p == 16 || pd.p == 24 || pd.p == 32);
            if (D == 3 && pd.p == 16) k_leaf_moments3d_t<16, 2><<<I->nleafq, 128, 0, s>>>(I->d_leafq, s4f, Qf, inv_rc);
            else if (D == 3 && pd.p == 24) k_leaf_moments3d_t<24, 4><<<I->nleafq, 216, 0, s>>>(I->d_leafq, s4f, Qf, inv_rc);
            else if (D == 3 && pd.p == 32) k_leaf_moments3d_t<32, 4><<<I->nleafq, 512, 0, s>>>(I->d_leafq, s4f, Qf, inv_rc);
        }
        if (tiled) {
        } else if (D == 3 && pd.p == 16) gemm(k_leaf_moments3d_gemm<T, 16>, leaf_moments3d_gemm_smem<T, 16>());
        else if (D == 3 && pd.p == 24) gemm(k_leaf_moments3d_gemm<T, 24>, leaf_moments3d_gemm_smem<T, 24>());
        else {
            const size_t sm = ts * (32 * D * pd.p + 32);
            k_leaf_moments<T, D><<<I->nleafq, 128, sm, s>>>(I->d_leafq, s4, Q, pd, inv_rc);
        }
        ++pw->launches;
    }
    // compile-time-order 2D re-expansion kernels (dynamic shared memory of nel elements)
    int cur_blocks = 0;
    auto launch_p = [&](auto kern, int nel, const int* lst, T* arr) {
        const size_t smb = size_t(nel) * ts;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
        kern<<<cur_blocks, 256, smb, s>>>(lst, arr, S, pd.np);
    };
    // 2. merge, deepest level first
    if (D == 2) {
        cudaFuncSetAttribute(k_merge2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_m2));
        cudaFuncSetAttribute(k_down2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_d2));
    } else {
        cudaFuncSetAttribute(k_merge<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_re));
        cudaFuncSetAttribute(k_down<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_re));
    }
    for (int l = I->nlevels - 1; phase == 1 && l >= 0; --l) {
        const int b = I->merge_start[l], e = I->merge_start[l + 1];
        if (e > b) {
            const int* lst = I->d_merge + size_t(b) * (1 + (1 << D));
            cur_blocks = e - b;
            if (D == 2) {
                switch (pd.p) {
                    case 16: launch_p(k_merge2d_p<T, 16>, 10 * 16 * 16, lst, Q); break;
                    case 20: launch_p(k_merge2d_p<T, 20>, 10 * 20 * 20, lst, Q); break;
                    case 24: launch_p(k_merge2d_p<T, 24>, 10 * 24 * 24, lst, Q); break;
                    case 28: launch_p(k_merge2d_p<T, 28>, 10 * 28 * 28, lst, Q); break;
                    case 32: launch_p(k_merge2d_p<T, 32>, 10 * 32 * 32, lst, Q); break;
                    default: k_merge2d<T><<<e - b, 256, sm_m2, s>>>(lst, Q, S, pd);
                }
            } else if ((sizeof(T) == 4 && (pd.p == 16 || pd.p == 24)) || (sizeof(T) == 8 && pd.p == 16)) {
                // register accumulators over the triangular shift matrices (three P^3
                // shared buffers: FP32 up to P = 24, FP64 P = 16)
                auto mr = [&](auto kern, int P) {
                    const size_t smb = ts * (2 * P * P * P);
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                    kern<<<e - b, P * P, smb, s>>>(lst, Q);
                };
                if (pd.p == 16) mr(k_merge3d_r<T, 16>, 16);
                else if constexpr (sizeof(T) == 4) mr(k_merge3d_r<T, 24>, 24);
            } else if ((pd.p == 16 || pd.p == 24) && e - b < pw->nsm) {
                // a level with fewer parents than SMs: four blocks per parent (k_merge3d_q);
                // larger levels keep one block per parent, which issues fewer shared loads
                auto m3 = [&](auto kern, int P) {
                    const size_t smb = ts * 7 * P * P;
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                    kern<<<4 * (e - b), P * P, smb, s>>>(lst, Q, S, static_cast<T*>(I->d_part3), I->d_done3);
                };
                if (pd.p == 16) m3(k_merge3d_q<T, 16>, 16);
                else m3(k_merge3d_q<T, 24>, 24);
            } else if (pd.p == 16 || pd.p == 24) {
                auto m3 = [&](auto kern, int P) {
                    const size_t smb = ts * 18 * P * P;
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                    kern<<<e - b, P * P, smb, s>>>(lst, Q, S);
                };
                if (pd.p == 16) m3(k_merge3d_p<T, 16>, 16);
                else m3(k_merge3d_p<T, 24>, 24);
            } else {
                k_merge<T, D><<<e - b, 128, sm_re, s>>>(lst, Q, S, pd);
            }
            ++pw->launches;
        }
    }
    // 3. outgoing plane waves (all levels); fused into the moments launch for the compile-time
    //    2D orders
    const bool fixed3d = D == 3 && ((pd.p == 16 && pd.K == 9) || (pd.p == 24 && pd.K == 16));
    if (phase == 2 && I->nout > 0 && fixed3d) {
        if (I->half3d) {
            if constexpr (sizeof(T) == 4) {
                float4* o4 = reinterpret_cast<float4*>(I->d_out);
                auto hout = [&](auto kern, int P) {
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(I->in3d_smem));
                    kern<<<I->nout, P * P, I->in3d_smem, s>>>(I->d_outl, Q, o4, Co, I->d_rowb, I->d_k0rows, I->nhalf,
                                                              I->nk0, I->nrowb, I->in3d_r1);
                };
                if (pd.p == 16) hout(k_pw_out3d_h<16, 9>, 16);
                else hout(k_pw_out3d_h<24, 16>, 24);
            }
        } else {
            if (pd.p == 16) k_pw_out3d_p<T, 16, 9><<<I->nout, 256, 0, s>>>(I->d_outl, Q, out, Co, I->d_row);
            else k_pw_out3d_p<T, 24, 16><<<I->nout, 576, 0, s>>>(I->d_outl, Q, out, Co, I->d_row);
        }
        ++pw->launches;
    } else if (phase == 2 && I->nout > 0 && !fixed2d) {
        size_t sm = ts * 2 * (size_t(pd.n1) * pd.p + size_t(I->KC) * pd.pd1 + 2 * size_t(pd.n1) * pd.p);
        cudaFuncSetAttribute(k_pw_out<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_pw_out<T, D><<<I->nout, 128, sm, s>>>(I->d_outl, Q, out, Co, pd, std::min(I->KC, 16));
        ++pw->launches;
    }
    // 4. translation + incoming (all levels)
    if (phase == 3 && I->nin > 0 && fixed2d) {
        const int g = I->nin;  // one block per box
        const C2<T>* ph = static_cast<const C2<T>*>(I->d_ph);
        const T* fk = static_cast<const T*>(I->d_f);
        if (pd.p == 16) k_pw_in2d_p<T, 16, 9><<<g, 128, 0, s>>>(I->d_inl, I->nin, out, L, Co, ph, fk);
        else if (pd.p == 24) k_pw_in2d_p<T, 24, 16><<<g, 128, 0, s>>>(I->d_inl, I->nin, out, L, Co, ph, fk);
        else k_pw_in2d_p<T, 32, 23><<<g, 128, 0, s>>>(I->d_inl, I->nin, out, L, Co, ph, fk);
        ++pw->launches;
    } else if (phase == 3 && I->nin > 0 && fixed3d && I->half3d) {
        if constexpr (sizeof(T) == 4) {
            const C2<float>* ph = static_cast<const C2<float>*>(I->d_ph);
            const float4* o4 = reinterpret_cast<const float4*>(I->d_out);
            auto hin = [&](auto kern, int P) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(I->in3d_smem));
                kern<<<I->nin, P * P, I->in3d_smem, s>>>(I->d_inl, o4, L, Co, ph, I->d_item,
                                                         static_cast<const float*>(I->d_fh), I->d_rowb, I->d_k0rows,
                                                         I->nhalf, I->nk0, I->nrowb, I->in3d_r1, inv_rc);
            };
            if (pd.p == 16) hin(k_pw_in3d_h<16, 9>, 16);
            else hin(k_pw_in3d_h<24, 16>, 24);
        }
        ++pw->launches;
    } else if (phase == 3 && I->nin > 0 && fixed3d) {
        const C2<T>* ph = static_cast<const C2<T>*>(I->d_ph);
        const T* fk = static_cast<const T*>(I->d_f);
        if (pd.p == 16)
            k_pw_in3d_p<T, 16, 9><<<I->nin, 256, 0, s>>>(I->d_inl, out, L, Co, ph, fk, inv_rc);
        else
            k_pw_in3d_p<T, 24, 16><<<I->nin, 576, 0, s>>>(I->d_inl, out, L, Co, ph, fk, inv_rc);
        ++pw->launches;
    } else if (phase == 3 && I->nin > 0) {
        const int KC = std::min(I->KC, 16);
        size_t sm = ts * 2 * (size_t(pd.n1) * pd.p + 3 * size_t(pd.n1) + size_t(KC) * pd.nk1 + size_t(KC) * pd.pd1 +
                              size_t(pd.n1) * pd.p);
        cudaFuncSetAttribute(k_pw_in<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_pw_in<T, D><<<I->nin, 128, sm, s>>>(I->d_inl, out, L, Co, static_cast<const C2<T>*>(I->d_ph),
                                              static_cast<const T*>(I->d_f), pd, KC, inv_rc);
        ++pw->launches;
    }
    // 5. downward, root first (by parent level); the compile-time 2D orders in one launch
    //    that also evaluates the target leaves
    if (phase == 4 && fixed2d && I->ndown_items > 0) {
        if (cudaMemsetAsync(I->d_down_flags, 0, (size_t(I->ndown_items) + 3) * sizeof(int), s) != cudaSuccess)
            return PDMK_ERR_CUDA;
        const T* t4 = static_cast<const T*>(pw->d_tgt4);
        int* counter = I->d_down_flags + I->ndown_items + 1;
        int* err_dev = I->d_down_flags + I->ndown_items + 2;
        auto persist = [&](auto kern, int P) {
            const size_t smb = ts * 9 * P * P;
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
            int per_sm = 0, nsm = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smb);
            const int grid = std::max(1, std::min(I->ndown_items, std::max(1, per_sm) * nsm));
            kern<<<grid, 256, smb, s>>>(I->d_down_items, I->ndown_items, counter, I->d_down_flags, pw->d_err, err_dev, L, S,
                                        t4, pw->d_pot, pw->d_grad, inv_rc, 1000000000ull);
        };
        if (pd.p == 16) persist(k_down_persist2d<T, 16>, 16);
        else if (pd.p == 24) persist(k_down_persist2d<T, 24>, 24);
        else persist(k_down_persist2d<T, 32>, 32);
        ++pw->launches;
    }
    for (int l = 0; phase == 4 && !fixed2d && l + 1 < I->nlevels; ++l) {
        const int b = I->down_start[l], e = I->down_start[l + 1];
        if (e > b) {
            const int* lst = I->d_down + size_t(b) * (1 + (1 << D));
            cur_blocks = e - b;
            if (D == 2) {
                switch (pd.p) {
                    case 16: launch_p(k_down2d_p<T, 16>, 5 * 16 * 16, lst, L); break;
                    case 20: launch_p(k_down2d_p<T, 20>, 5 * 20 * 20, lst, L); break;
                    case 24: launch_p(k_down2d_p<T, 24>, 5 * 24 * 24, lst, L); break;
                    case 28: launch_p(k_down2d_p<T, 28>, 5 * 28 * 28, lst, L); break;
                    case 32: launch_p(k_down2d_p<T, 32>, 5 * 32 * 32, lst, L); break;
                    default: k_down2d<T><<<e - b, 256, sm_d2, s>>>(lst, L, S, pd);
                }
            } else if ((sizeof(T) == 4 && (pd.p == 16 || pd.p == 24)) || (sizeof(T) == 8 && pd.p == 16)) {
                // two blocks per parent, register accumulators over the triangular shift
                // matrices (two P^3 shared buffers)
                auto dr = [&](auto kern, int P) {
                    const size_t smb = ts * (2 * P * P * P);
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                    kern<<<2 * (e - b), P * P, smb, s>>>(lst, L, I->d_ladd);
                };
                if (pd.p == 16) dr(k_down3d_r<T, 16>, 16);
                else if constexpr (sizeof(T) == 4) dr(k_down3d_r<T, 24>, 24);
            } else if (pd.p == 16 || pd.p == 24) {
                // four blocks per parent (k_down3d_q)
                auto d3 = [&](auto kern, int P) {
                    const size_t smb = ts * (4 * P * P + P * P * P);
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                    kern<<<4 * (e - b), P * P, smb, s>>>(lst, L, S);
                };
                if (pd.p == 16) d3(k_down3d_q<T, 16>, 16);
                else d3(k_down3d_q<T, 24>, 24);
            } else {
                k_down<T, D><<<e - b, 128, sm_re, s>>>(lst, L, S, pd);
            }
            ++pw->launches;
        }
    }
    // 6. leaf evaluation (folded into the downward launch for the compile-time 2D orders)
    const bool leaf_tc = D == 3 && sizeof(T) == 4 && pw->tensor_cores && (pd.p == 16 || pd.p == 24);
    if (phase == 5 && I->neval > 0 && leaf_tc) {
        // tensor cores (tcgen05, 3xTF32): persistent, two CTAs per SM
        if constexpr (sizeof(T) == 4) {
            const float* t4 = static_cast<const float*>(pw->d_tgt4);
            const int grid = std::max(1, std::min(I->neval, 2 * pw->nsm));
            auto tc = [&](auto kern, size_t smb) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                kern<<<grid, 128, smb, s>>>(I->d_eval, I->neval, L, t4, pw->d_pot, pw->d_grad, inv_rc, pw->d_err);
            };
            if (pd.p == 16) tc(k_leaf_eval3d_tc<16>, LeafTcLayout<16>::total);
            else tc(k_leaf_eval3d_tc<24>, LeafTcLayout<24>::total);
        }
        ++pw->launches;
    } else if (phase == 5 && I->neval > 0 && D == 3 && (pd.p == 16 || pd.p == 24 || (pd.p == 32 && sizeof(T) == 4))) {
        const T* t4 = static_cast<const T*>(pw->d_tgt4);
        auto gemm = [&](auto kern, size_t smb) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
            kern<<<I->neval, 256, smb, s>>>(I->d_eval, L, t4, pw->d_pot, pw->d_grad, inv_rc);
        };
        if (pd.p == 16) gemm(k_leaf_eval3d_gemm<T, 16>, leaf_eval3d_gemm_smem<T, 16>());
        else if (pd.p == 24) gemm(k_leaf_eval3d_gemm<T, 24>, leaf_eval3d_gemm_smem<T, 24>());
        else if constexpr (sizeof(T) == 4) gemm(k_leaf_eval3d_gemm<T, 32>, leaf_eval3d_gemm_smem<T, 32>());
        ++pw->launches;
    } else if (phase == 5 && I->neval > 0 && D == 3 && pd.p == 32) {
        // FP64 order 32: the coefficients (256 KB) do not fit in shared memory
        const T* t4 = static_cast<const T*>(pw->d_tgt4);
        k_leaf_eval3d_p<T, 32><<<I->neval, 32, 0, s>>>(I->d_eval, L, t4, pw->d_pot, pw->d_grad, inv_rc);
        ++pw->launches;
    } else if (phase == 5 && I->neval > 0 && !fixed2d) {
        size_t sm = ts * 32 * 2 * D * pd.p;
        cudaFuncSetAttribute(k_leaf_eval<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_leaf_eval<T, D><<<I->neval, 32, sm, s>>>(I->d_eval, L, static_cast<const T*>(pw->d_tgt4), pw->d_pot,
                                                   pw->d_grad, pd, inv_rc);
        ++pw->launches;
    }
    if (cudaGetLastError() != cudaSuccess) return PDMK_ERR_CUDA;
    return PDMK_OK;
}

int pw_eval(PwPlan* pw, cudaStream_t s, int phase) {
    if (phase == 0) pw->launches = 0;
    if (!pw->active) return PDMK_OK;
    if (pw->d == 2) return pw->mixed ? pw_eval_t<float, 2>(pw, s, phase) : pw_eval_t<double, 2>(pw, s, phase);
    return pw->mixed ? pw_eval_t<float, 3>(pw, s, phase) : pw_eval_t<double, 3>(pw, s, phase);
}

int pw_eval_points(PwPlan* pw, cudaStream_t s, const int4* d_list, int nlist, const void* d_pts4, double* pot,
                   double* grad) {
    if (!pw->active || nlist <= 0) return PDMK_OK;
    PwImpl* I = impl(pw);
    const PwDims& pd = I->dims;
    const double inv_rc = 1.0 / I->rc;
    auto run = [&](auto tag, auto dtag) {
        using T = decltype(tag);
        constexpr int D = decltype(dtag)::value;
        const size_t sm = sizeof(T) * 32 * 2 * D * pd.p;
        cudaFuncSetAttribute(k_leaf_eval<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_leaf_eval<T, D><<<nlist, 32, sm, s>>>(d_list, static_cast<const T*>(I->d_L), static_cast<const T*>(d_pts4),
                                                pot, grad, pd, inv_rc);
    };
    if (pw->d == 2) {
        if (pw->mixed) run(float(), std::integral_constant<int, 2>());
        else run(double(), std::integral_constant<int, 2>());
    } else {
        if (pw->mixed) run(float(), std::integral_constant<int, 3>());
        else run(double(), std::integral_constant<int, 3>());
    }
    return cudaGetLastError() == cudaSuccess ? PDMK_OK : PDMK_ERR_CUDA;
}

void pw_free_sources(PwPlan* pw) {
    pw->lslot.clear();
    pw->local_full.clear();
    for (auto& a : pw->allocs) {
        if (pw->pool) pw->pool->put(a.first, a.second);
        else cudaFree(a.first);
    }
    pw->allocs.clear();
    pw->device_bytes = 0;
    pw->active = false;
    pw->d_pot = nullptr;
    pw->d_grad = nullptr;
    PwImpl* I = impl(pw);
    if (I) {
        I->d_Co = I->d_S = I->d_ph = I->d_f = nullptr;
        I->d_row = nullptr;
        I->d_item = nullptr; I->d_fh = nullptr; I->d_rowb = nullptr; I->d_k0rows = nullptr;
        I->d_leafq = nullptr; I->d_merge = nullptr; I->d_outl = nullptr; I->d_inl = nullptr;
        I->d_down = nullptr; I->d_eval = nullptr; I->d_Q = I->d_out = I->d_L = nullptr;
        I->nleafq = I->nout = I->nin = I->neval = 0;
        I->d_ditems = nullptr; I->d_src_leaf = nullptr; I->d_bcoord = nullptr; I->d_part = nullptr;
        I->d_obox = nullptr; I->d_seg_done = nullptr; I->d_part3 = nullptr; I->d_done3 = nullptr;
        I->d_ladd = nullptr;
        I->nditems = 0;
        I->d_down_items = nullptr; I->d_down_flags = nullptr;
        I->ndown_items = 0;
    }
}

void pw_free(PwPlan* pw) {
    pw_free_sources(pw);
    if (pw->h_err) cudaFreeHost(pw->h_err);
    pw->h_err = pw->d_err = nullptr;
    delete impl(pw);
    pw->impl = nullptr;
}

}  // namespace pdmk
