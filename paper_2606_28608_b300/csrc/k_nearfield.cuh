// k_nearfield.cuh -- leaf-level residual-kernel direct sum (Sec. 2.3 and Sec. 3.5; Eq. (2.7)
// for 3D, the radial-transform residual for 2D).
//
// One CTA of 64 threads per target leaf B.  Targets sit in registers (one per thread; the
// threads split into two groups that share the sources when B holds at most 32 targets); the
// sources of every leaf in B's direct list are streamed through shared memory in tiles of
// 64, shifted into B's frame once per tile.  Per target the sum is a plain sum inside a tile and a compensated (Kahan)
// sum across tiles and groups.  R_{L_B} vanishes for r >= h_{L_B}, so pairs beyond the
// cut-off cost one compare.  The self pair (r = 0) is skipped; its W_L(0) is removed later.
//
// Algorithmic bytes: 16 (FP32) / 32 (FP64) per staged source per target leaf, plus the
// target record; flops: ~35 (3D) / ~40 (2D) per pair inside the cut-off.
#pragma once
#include "kernels_common.cuh"

namespace pdmk {

constexpr int kNearThreads = 64;
constexpr int kNearTile = 64;
constexpr int kNearMaxList = 256;

// Clenshaw with a compile-time number of terms (coefficients zero-padded) and coefficients
// in registers: fully unrolled.
template <typename T, int NC>
__device__ __forceinline__ T clenshaw_reg(const T (&c)[NC], T x) {
    T b1 = T(0), b2 = T(0);
    const T x2 = x + x;
#pragma unroll
    for (int k = NC - 1; k >= 1; --k) {
        const T b0 = fma(x2, b1, c[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(x, b1, c[0] - b2);
}

template <typename T>
__device__ __forceinline__ T fast_rcp(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ float fast_rcp<float>(float x) { return __frcp_rn(x); }
template <typename T>
__device__ __forceinline__ T fast_rsqrt(T x) { return T(1) / sqrt(x); }
template <>
__device__ __forceinline__ float fast_rsqrt<float>(float x) { return rsqrtf(x); }

template <typename T, int D, int NC>
__global__ void __launch_bounds__(kNearThreads)
k_nearfield(NearArgs<T> a) {
    __shared__ T sx[kNearTile], sy[kNearTile], sz[kNearTile], sq[kNearTile];
    __shared__ int e_begin[kNearMaxList];
    __shared__ int e_pref[kNearMaxList + 1];
    __shared__ T e_shift[3][kNearMaxList];
    // two-float (hi + lo) copies for the compensated close-pair difference (mixed path)
    constexpr int kLo = (sizeof(T) == 4) ? 1 : 0;
    __shared__ T e_shlo[kLo ? 3 : 1][kLo ? kNearMaxList : 1];
    __shared__ T slx[kLo ? kNearTile : 1], sly[kLo ? kNearTile : 1], slz[kLo ? kNearTile : 1];
    __shared__ double red[4][kNearThreads];

    const TLeaf L = a.tleaf[blockIdx.x];
    const int tid = threadIdx.x;
    T cA[NC], cB[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        cA[k] = k < a.nA ? a.coefA[k] : T(0);
        cB[k] = k < a.nB ? a.coefB[k] : T(0);
    }

    const double hinv_d = a.inv_rc * double(1LL << L.level);
    const T hinv = T(hinv_d);
    const T h2inv = T(hinv_d * hinv_d);
    const double* cB_centre = a.box_center + size_t(L.box) * D;
    const int nt = L.tgt_count;
    // targets per group: the smallest power of two >= nt (so the groups tile the block
    // exactly); the G = 64 / C groups split the source tiles, so small leaves still keep
    // most lanes busy
    int C = 1;
    while (C < nt && C < kNearThreads) C <<= 1;
    const int G = kNearThreads / C;
    const int lt = tid % C;
    const int grp = tid / C;
    const bool ingrp = grp < G;
    const T inv4pi = T(0.07957747154594766788);  // 1/(4 pi)
    unsigned long long nin = 0;

    for (int t0 = 0; t0 < nt; t0 += C) {
        const int ti = t0 + lt;
        const bool act = ingrp && ti < nt;
        T xt = 0, yt = 0, zt = 0;
        T xtl = 0, ytl = 0, ztl = 0;
        if (act) {
            const T* p = a.tgt4 + size_t(L.tgt_begin + ti) * 4;
            xt = p[0];
            yt = p[1];
            if (D == 3) zt = p[2];
            if constexpr (kLo) {
                const T* pl = a.tgt_lo + size_t(L.tgt_begin + ti) * 4;
                xtl = pl[0];
                ytl = pl[1];
                if (D == 3) ztl = pl[2];
            }
        }
        Kahan<T> kp, kx, ky, kz;
        kp.init(); kx.init(); ky.init(); kz.init();

        for (int s0 = 0; s0 < L.list_count; s0 += kNearMaxList) {
            const int ne = min(kNearMaxList, L.list_count - s0);
            __syncthreads();
            for (int e = tid; e < ne; e += kNearThreads) {
                int box = a.list[L.list_begin + s0 + e];
                e_begin[e] = a.box_src_begin[box];
                e_pref[e + 1] = a.box_src_count[box];
                const double* cs = a.box_center + size_t(box) * D;
                for (int k = 0; k < D; ++k) {
                    const double sh = cs[k] - cB_centre[k];
                    e_shift[k][e] = T(sh);
                    if constexpr (kLo) e_shlo[k][e] = T(sh - double(T(sh)));
                }
            }
            __syncthreads();
            if (tid == 0) {
                e_pref[0] = 0;
                for (int e = 0; e < ne; ++e) e_pref[e + 1] += e_pref[e];
            }
            __syncthreads();
            const int total = e_pref[ne];
            for (int ts = 0; ts < total; ts += kNearTile) {
                const int p = ts + tid;
                if (p < total) {
                    int lo = 0, hi = ne - 1;  // entry e with e_pref[e] <= p < e_pref[e+1]
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (e_pref[mid] <= p) lo = mid; else hi = mid - 1;
                    }
                    const int gi = e_begin[lo] + (p - e_pref[lo]);
                    const T* s = a.src4 + size_t(gi) * 4;
                    if constexpr (kLo) {
                        // y' = (y_hi + y_lo) + (sh_hi + sh_lo) as hi + lo: TwoSum of the hi parts
                        const T* sl = a.src_lo + size_t(gi) * 4;
                        T* dh[3] = {sx, sy, sz};
                        T* dl[3] = {slx, sly, slz};
                        for (int k = 0; k < D; ++k) {
                            const T ah = s[k], bh = e_shift[k][lo];
                            const T sum = ah + bh;
                            const T bb = sum - ah;
                            const T err = (ah - (sum - bb)) + (bh - bb);
                            dh[k][tid] = sum;
                            dl[k][tid] = err + sl[k] + e_shlo[k][lo];
                        }
                    } else {
                        sx[tid] = s[0] + e_shift[0][lo];
                        sy[tid] = s[1] + e_shift[1][lo];
                        if (D == 3) sz[tid] = s[2] + e_shift[2][lo];
                    }
                    sq[tid] = s[3];
                }
                __syncthreads();
                const int cnt = min(kNearTile, total - ts);
                T pp = 0, gx = 0, gy = 0, gz = 0;
                if (act) {
                    for (int j = grp; j < cnt; j += G) {
                        T dx = xt - sx[j];
                        T dy = yt - sy[j];
                        T dz = (D == 3) ? zt - sz[j] : T(0);
                        T r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                        T s = r2 * h2inv;
                        if constexpr (kLo) if (s < a.close_s) {
                            // close pair: compensated difference (x_hi - y_hi) + (x_lo - y_lo); the
                            // hi difference is exact for nearby values, so ~48 bits survive
                            dx = (xt - sx[j]) + (xtl - slx[j]);
                            dy = (yt - sy[j]) + (ytl - sly[j]);
                            dz = (D == 3) ? (zt - sz[j]) + (ztl - slz[j]) : T(0);
                            r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                            s = r2 * h2inv;
                        }
                        if (s < T(1) && r2 > T(0)) {
                            if (a.count_in) ++nin;
                            const T q = sq[j];
                            const T xc = fma(T(2), s, T(-1));
                            const T fa = clenshaw_reg<T, NC>(cA, xc);
                            const T fb = clenshaw_reg<T, NC>(cB, xc);
                            if (D == 3) {
                                // R = (1 - t A)/(4 pi r); grad R = -(1 - t A + t B) dr / (4 pi r^3)
                                const T rinv = fast_rsqrt(r2);
                                const T t = r2 * rinv * hinv;
                                const T num = fma(-t, fa, T(1));
                                pp = fma(q * num, rinv, pp);
                                const T gf = -q * fma(t, fb, num) * rinv * rinv * rinv;
                                gx = fma(gf, dx, gx);
                                gy = fma(gf, dy, gy);
                                gz = fma(gf, dz, gz);
                            } else {
                                // R = -log(s)/(4 pi) - A(s); grad R = -sqrt(1-s) S(s) dr/(2 pi r^2)
                                const T lg = log(s);
                                pp = fma(q, fma(-inv4pi, lg, -fa), pp);
                                const T gf = -q * sqrt(T(1) - s) * fb * fast_rcp(r2);
                                gx = fma(gf, dx, gx);
                                gy = fma(gf, dy, gy);
                            }
                        }
                    }
                    kp.add(pp);
                    kx.add(gx);
                    ky.add(gy);
                    if (D == 3) kz.add(gz);
                }
                __syncthreads();
            }
        }
        // combine the groups (FP64), group 0 writes
        red[0][tid] = kp.value();
        red[1][tid] = kx.value();
        red[2][tid] = ky.value();
        red[3][tid] = (D == 3) ? kz.value() : 0.0;
        __syncthreads();
        if (grp == 0 && act) {
            double P = 0, X = 0, Y = 0, Z = 0;
            for (int g = 0; g < G; ++g) {
                P += red[0][g * C + lt];
                X += red[1][g * C + lt];
                Y += red[2][g * C + lt];
                Z += red[3][g * C + lt];
            }
            const double kpot = (D == 3) ? 0.07957747154594766788 : 1.0;
            const double kgrad = (D == 3) ? 0.07957747154594766788 : 0.15915494309189533577;
            const size_t o = size_t(L.tgt_begin + ti);
            a.pot[o] = P * kpot;
            if (a.grad) {
                a.grad[o * D + 0] = X * kgrad;
                a.grad[o * D + 1] = Y * kgrad;
                if (D == 3) a.grad[o * D + 2] = Z * kgrad;
            }
        }
        __syncthreads();
    }
    if (a.count_in) {
        for (int o = 16; o > 0; o >>= 1) nin += __shfl_down_sync(0xffffffffu, nin, o);
        if ((tid & 31) == 0 && nin) atomicAdd(a.count_in, nin);
    }
}

// ---------------------------------------------------------------------------------------
// Warp-per-leaf variant.  One warp owns a target leaf; its targets sit one per lane in
// groups of C = 8, 16 or 32 lanes (the G = 32 / C groups split the sources).  The sources of
// the direct list are streamed as one flat sequence in chunks of 32, shifted into the target
// leaf's frame once per chunk.  Each lane first culls the chunk with the cut-off test r < h
// (a bit per source), then evaluates only its accepted pairs, so the expensive branch runs
// at the density of accepted pairs rather than at the density of any-lane-accepts.  The
// residual series are Horner sums of monomials in x = 2 s - 1 (the host converts the
// Chebyshev fits; both are equally accurate for these well-conditioned series), the
// logarithm, square root and reciprocal use the hardware approximations on the FP32 path.
// Plain sums inside a chunk, compensated (Kahan) sums across chunks, FP64 across groups.
template <typename T>
__device__ __forceinline__ T near_log2(T x) { return log2(x); }
template <>
__device__ __forceinline__ float near_log2<float>(float x) { return __log2f(x); }
template <typename T>
__device__ __forceinline__ T near_sqrt_pos(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float near_sqrt_pos<float>(float x) { return x * rsqrtf(x); }  // x > 0
template <typename T>
__device__ __forceinline__ T near_rcp(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ float near_rcp<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

constexpr int kNearWarps = 4;

template <typename T, int D, int NH>
__global__ void __launch_bounds__(32 * kNearWarps)
k_near_warp(NearArgs<T> a) {
    constexpr int kLo = (sizeof(T) == 4) ? 1 : 0;
    constexpr int ZD = (D == 3) ? 32 : 1, ZL = kLo ? 32 : 1, ZZ = (D == 3 && kLo) ? 32 : 1;
    __shared__ T sx[kNearWarps][32], sy[kNearWarps][32], sz[kNearWarps][ZD], sq[kNearWarps][32];
    __shared__ T lx[kNearWarps][ZL], ly[kNearWarps][ZL], lz[kNearWarps][ZZ];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * kNearWarps + w;
    if (li >= a.ntleaf) return;  // whole warp; the kernel has no block-wide barrier
    const TLeaf L = a.tleaf[li];
    T cA[NH], cB[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) {
        cA[k] = a.monoA[k];
        cB[k] = a.monoB[k];
    }
    const double hinv_d = a.inv_rc * double(1LL << L.level);
    const T hinv = T(hinv_d);
    const T h2inv = T(hinv_d * hinv_d);
    const T clog = T(0.0551589000381629);  // ln(2) / (4 pi): -log(s)/(4 pi) = -clog log2(s)
    const int nt = L.tgt_count;
    const int C = nt > 16 ? 32 : (nt > 8 ? 16 : 8);
    const int G = 32 / C;
    const int lt = lane & (C - 1), g = lane / C;
    unsigned long long nin = 0;
    const int2* ent = a.ent + L.list_begin;
    const T* esh = a.ent_sh + size_t(L.list_begin) * 4;
    const T* eshl = kLo ? a.ent_shlo + size_t(L.list_begin) * 4 : nullptr;
    const int ne = L.list_count;

    for (int t0 = 0; t0 < nt; t0 += C) {
        const int ti = t0 + lt;
        const bool act = ti < nt;
        T xt = 0, yt = 0, zt = 0, xtl = 0, ytl = 0, ztl = 0;
        if (act) {
            const T* p = a.tgt4 + size_t(L.tgt_begin + ti) * 4;
            xt = p[0];
            yt = p[1];
            if (D == 3) zt = p[2];
            if constexpr (kLo) {
                const T* pl = a.tgt_lo + size_t(L.tgt_begin + ti) * 4;
                xtl = pl[0];
                ytl = pl[1];
                if (D == 3) ztl = pl[2];
            }
        }
        Kahan<T> kp, kx, ky, kz;
        kp.init(); kx.init(); ky.init(); kz.init();
        int e = 0, off = 0;  // warp-uniform stream position
        while (e < ne) {
            int filled = 0;
            while (filled < 32 && e < ne) {
                const int2 bc = ent[e];
                const int take = min(32 - filled, bc.y - off);
                if (lane >= filled && lane < filled + take) {
                    const int gi = bc.x + off + (lane - filled);
                    const T* s = a.src4 + size_t(gi) * 4;
                    if constexpr (kLo) {
                        // (y_hi + y_lo) + (sh_hi + sh_lo) as hi + lo: TwoSum of the hi parts
                        const T* sl = a.src_lo + size_t(gi) * 4;
                        T hi[3], lo[3];
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            const T ah = s[k], bh = esh[e * 4 + k];
                            const T sum = ah + bh;
                            const T bb = sum - ah;
                            const T err = (ah - (sum - bb)) + (bh - bb);
                            hi[k] = sum;
                            lo[k] = err + sl[k] + eshl[e * 4 + k];
                        }
                        sx[w][lane] = hi[0];
                        sy[w][lane] = hi[1];
                        lx[w][lane] = lo[0];
                        ly[w][lane] = lo[1];
                        if constexpr (D == 3) {
                            sz[w][lane] = hi[2];
                            lz[w][lane] = lo[2];
                        }
                    } else {
                        sx[w][lane] = s[0] + esh[e * 4 + 0];
                        sy[w][lane] = s[1] + esh[e * 4 + 1];
                        if constexpr (D == 3) sz[w][lane] = s[2] + esh[e * 4 + 2];
                    }
                    sq[w][lane] = s[3];
                }
                filled += take;
                off += take;
                if (off >= bc.y) {
                    ++e;
                    off = 0;
                }
            }
            __syncwarp();
            // cull: bit k <-> source j = g + k G of the chunk
            unsigned mask = 0;
            if (act) {
                int k = 0;
                for (int j = g; j < filled; j += G, ++k) {
                    const T dx = xt - sx[w][j], dy = yt - sy[w][j];
                    const T dz = (D == 3) ? zt - sz[w][j] : T(0);
                    const T r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                    if (r2 * h2inv < T(1)) mask |= 1u << k;
                }
            }
            T pp = 0, gx = 0, gy = 0, gz = 0;
            while (mask) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1;
                const int j = g + k * G;
                T dx = xt - sx[w][j], dy = yt - sy[w][j];
                T dz = (D == 3) ? zt - sz[w][j] : T(0);
                T r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                T s = r2 * h2inv;
                if constexpr (kLo) {
                    if (s < a.close_s) {
                        // close pair: (x_hi - y_hi) + (x_lo - y_lo); the hi difference is exact
                        dx = (xt - sx[w][j]) + (xtl - lx[w][j]);
                        dy = (yt - sy[w][j]) + (ytl - ly[w][j]);
                        if constexpr (D == 3) dz = (zt - sz[w][j]) + (ztl - lz[w][j]);
                        r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                        s = r2 * h2inv;
                    }
                }
                if (r2 > T(0)) {  // the self pair is skipped
                    if (a.count_in) ++nin;
                    const T q = sq[w][j];
                    const T xc = fma(T(2), s, T(-1));
                    T fa = cA[NH - 1], fb = cB[NH - 1];
#pragma unroll
                    for (int m = NH - 2; m >= 0; --m) {
                        fa = fma(fa, xc, cA[m]);
                        fb = fma(fb, xc, cB[m]);
                    }
                    if constexpr (D == 3) {
                        // R = (1 - t A)/(4 pi r); grad R = -(1 - t A + t B) dr / (4 pi r^3)
                        const T rinv = fast_rsqrt(r2);
                        const T t = r2 * rinv * hinv;
                        const T num = fma(-t, fa, T(1));
                        pp = fma(q * num, rinv, pp);
                        const T gf = -q * fma(t, fb, num) * rinv * rinv * rinv;
                        gx = fma(gf, dx, gx);
                        gy = fma(gf, dy, gy);
                        gz = fma(gf, dz, gz);
                    } else {
                        // R = -log(s)/(4 pi) - A(s); grad R = -sqrt(1-s) S(s) dr/(2 pi r^2)
                        pp = fma(q, fma(-clog, near_log2(s), -fa), pp);
                        const T gf = -q * near_sqrt_pos(T(1) - s) * fb * near_rcp(r2);
                        gx = fma(gf, dx, gx);
                        gy = fma(gf, dy, gy);
                    }
                }
            }
            if (act) {
                kp.add(pp);
                kx.add(gx);
                ky.add(gy);
                if (D == 3) kz.add(gz);
            }
            __syncwarp();
        }
        // combine the groups in a fixed order (FP64): lanes lt + g C
        double P = kp.value(), X = kx.value(), Y = ky.value(), Z = (D == 3) ? kz.value() : 0.0;
        for (int o = 16; o >= C; o >>= 1) {
            P += __shfl_down_sync(0xffffffffu, P, o);
            X += __shfl_down_sync(0xffffffffu, X, o);
            Y += __shfl_down_sync(0xffffffffu, Y, o);
            if (D == 3) Z += __shfl_down_sync(0xffffffffu, Z, o);
        }
        if (g == 0 && act) {
            const double kpot = (D == 3) ? 0.07957747154594766788 : 1.0;
            const double kgrad = (D == 3) ? 0.07957747154594766788 : 0.15915494309189533577;
            const size_t o = size_t(L.tgt_begin + ti);
            a.pot[o] = P * kpot;
            if (a.grad) {
                a.grad[o * D + 0] = X * kgrad;
                a.grad[o * D + 1] = Y * kgrad;
                if (D == 3) a.grad[o * D + 2] = Z * kgrad;
            }
        }
    }
    if (a.count_in) {
        for (int o = 16; o > 0; o >>= 1) nin += __shfl_down_sync(0xffffffffu, nin, o);
        if (lane == 0 && nin) atomicAdd(a.count_in, nin);
    }
}

}  // namespace pdmk
