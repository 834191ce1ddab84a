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
// The target groups below must tile the block exactly: a group size C above the block gives
// G = kNearThreads / C = 0 groups, and the source loop (j += G) would never advance; a C that
// does not divide the block leaves threads outside every group.  C is the smallest power of
// two >= the leaf's target count, capped at the block, so a power-of-two block is required.
static_assert(kNearThreads > 0 && (kNearThreads & (kNearThreads - 1)) == 0, "block must be a power of two");
static_assert(kNearTile == kNearThreads, "one staged source per thread");

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
    const int nt = L.tgt_count;
    // targets per group: the smallest power of two >= nt (so the groups tile the block
    // exactly); the G = 64 / C groups split the source tiles, so small leaves still keep
    // most lanes busy
    int C = 1;
    while (C < nt && C < kNearThreads) C <<= 1;
    const int G = kNearThreads / C;  // >= 1, and G * C == kNearThreads (power-of-two C <= block)
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
                // source range and the source leaf centre's shift into this leaf's frame
                // (hi / lo in T), as the host formed them
                const int ei = L.list_begin + s0 + e;
                const int2 bc = a.ent[ei];
                e_begin[e] = bc.x;
                e_pref[e + 1] = bc.y;
                for (int k = 0; k < D; ++k) {
                    e_shift[k][e] = a.ent_sh[size_t(ei) * 4 + k];
                    if constexpr (kLo) e_shlo[k][e] = a.ent_shlo[size_t(ei) * 4 + k];
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
// Warp-per-leaf kernel with a compacted pair queue.  One warp owns a target leaf and takes
// its targets in passes of up to 32 (target t of the pass <-> lane t for the sums).  The
// sources of the direct list stream as one flat sequence in chunks of 32, one per lane,
// shifted into the target leaf's frame.  Per chunk:
//   cull:  for each target t, every lane tests its source against the cut-off r < h; a
//          ballot appends the accepted (t, source) pairs to a per-warp queue, t-major;
//   eval:  lane l takes the l-th of 32 equal contiguous blocks of the queue (every lane
//          busy, whatever the acceptance pattern) and sums in registers while the target
//          stays the same; each run's sum goes to a slot named by where the run starts;
// then lane t adds its target's run sums, in queue order, to its compensated (Kahan)
// accumulators.  The order of every sum is fixed by the queue, so results do not depend
// on scheduling.  The residual
// series are Horner sums of monomials in x = 2 s - 1 (the host converts the Chebyshev fits;
// for these series both are equally accurate); on the FP32 path the logarithm, square root
// and reciprocal use the hardware approximations.
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

// per-warp shared state of the queue kernel; a chunk holds CW sources (CW / 32 per lane)
template <typename T, int D>
struct NearWarpSmem {
    static constexpr int kLo = (sizeof(T) == 4) ? 1 : 0;
    static constexpr int CW = (sizeof(T) == 4) ? 64 : 32;       // sources per chunk
    static constexpr int SH = CW == 64 ? 6 : 5;                 // queue entry: t << SH | source
    T tx[32], ty[32], tz[D == 3 ? 32 : 1];                       // targets of the pass (hi)
    T tlx[kLo ? 32 : 1], tly[kLo ? 32 : 1], tlz[(D == 3 && kLo) ? 32 : 1];  // (lo)
    T sx[CW], sy[CW], sz[D == 3 ? CW : 1], sq[CW];              // chunk sources (hi), charge
    T lx[kLo ? CW : 1], ly[kLo ? CW : 1], lz[(D == 3 && kLo) ? CW : 1];     // (lo)
    // partial sums of the pair runs: [0, 32) a lane's first run, [32, 64) a run that starts
    // at target t's first pair
    T rp[64], rx[64], ry[64], rz[D == 3 ? 64 : 1];
    unsigned short q[32 * CW];                                  // pair queue
};

// NH: padded length of the B series; NA <= NH: of the A series (usually two terms shorter)
template <typename T, int D, int NH, int NA>
__global__ void __launch_bounds__(32 * kNearWarps, sizeof(T) == 4 ? 7 : 1)
k_near_warp(NearArgs<T> a) {
    constexpr int kLo = NearWarpSmem<T, D>::kLo;
    constexpr int CW = NearWarpSmem<T, D>::CW, SH = NearWarpSmem<T, D>::SH, NHALF = CW / 32;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ NearWarpSmem<T, D> smem[kNearWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * kNearWarps + w;
    if (li >= a.ntleaf) return;  // whole warp; the kernel has no block-wide barrier
    static_assert(NH <= kNearMono && NA <= NH, "series lengths");
    NearWarpSmem<T, D>& S = smem[w];
    const TLeaf L = a.tleaf[li];
    const double hinv_d = a.inv_rc * double(1LL << L.level);
    const T hinv = T(hinv_d);
    const T h2inv = T(hinv_d * hinv_d);
    const T clog = T(0.0551589000381629);  // ln(2) / (4 pi): -log(s)/(4 pi) = -clog log2(s)
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long nin = 0;
    const int2* ent = a.ent + L.list_begin;
    const T* esh = a.ent_sh + size_t(L.list_begin) * 4;
    const T* eshl = kLo ? a.ent_shlo + size_t(L.list_begin) * 4 : nullptr;
    const int ne = L.list_count;

    for (int t0 = 0; t0 < L.tgt_count; t0 += 32) {
        const int nt = min(32, L.tgt_count - t0);
        const bool own = lane < nt;  // this lane owns target t0 + lane
        if (own) {
            const T* p = a.tgt4 + size_t(L.tgt_begin + t0 + lane) * 4;
            S.tx[lane] = p[0];
            S.ty[lane] = p[1];
            if constexpr (D == 3) S.tz[lane] = p[2];
            if constexpr (kLo) {
                const T* pl = a.tgt_lo + size_t(L.tgt_begin + t0 + lane) * 4;
                S.tlx[lane] = pl[0];
                S.tly[lane] = pl[1];
                if constexpr (D == 3) S.tlz[lane] = pl[2];
            }
        }
        Kahan<T> kp, kx, ky, kz;
        kp.init(); kx.init(); ky.init(); kz.init();
        int e = 0, off = 0;  // warp-uniform stream position
        while (e < ne) {
            // ---- chunk of up to CW sources, lane l <-> sources l, l + 32, .., in the target
            //      leaf's frame
            int filled = 0;
            while (filled < CW && e < ne) {
                const int2 bc = ent[e];
                const int take = min(CW - filled, bc.y - off);
#pragma unroll
                for (int hh = 0; hh < NHALF; ++hh) {
                const int slot = lane + 32 * hh;
                if (slot >= filled && slot < filled + take) {
                    const int gi = bc.x + off + (slot - filled);
                    T mx, my, mz = T(0);
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
                        mx = hi[0];
                        my = hi[1];
                        S.lx[slot] = lo[0];
                        S.ly[slot] = lo[1];
                        if constexpr (D == 3) {
                            mz = hi[2];
                            S.lz[slot] = lo[2];
                        }
                    } else {
                        mx = s[0] + esh[e * 4 + 0];
                        my = s[1] + esh[e * 4 + 1];
                        if constexpr (D == 3) mz = s[2] + esh[e * 4 + 2];
                    }
                    S.sx[slot] = mx;
                    S.sy[slot] = my;
                    if constexpr (D == 3) S.sz[slot] = mz;
                    S.sq[slot] = s[3];
                }
                }
                filled += take;
                off += take;
                if (off >= bc.y) {
                    ++e;
                    off = 0;
                }
            }
            __syncwarp();
            // ---- cull: every lane tests its sources against target t; accepted pairs queue
            //      in (t, source) order; lane t records where its target's run starts
            T mx[NHALF], my[NHALF], mz[NHALF];
            bool hs[NHALF];
#pragma unroll
            for (int hh = 0; hh < NHALF; ++hh) {
                hs[hh] = lane + 32 * hh < filled;
                mx[hh] = S.sx[lane + 32 * hh];
                my[hh] = S.sy[lane + 32 * hh];
                mz[hh] = (D == 3) ? S.sz[lane + 32 * hh] : T(0);
            }
            int N = 0, my_start = 0;
#pragma unroll 4
            for (int t = 0; t < nt; ++t) {
                const T tx = S.tx[t], ty = S.ty[t];
                const T tz = (D == 3) ? S.tz[t] : T(0);
                int base = N;
#pragma unroll
                for (int hh = 0; hh < NHALF; ++hh) {
                    const T dx = tx - mx[hh], dy = ty - my[hh];
                    const T dz = (D == 3) ? tz - mz[hh] : T(0);
                    const T r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                    const bool acc = hs[hh] && r2 * h2inv < T(1);
                    const unsigned b = __ballot_sync(kFull, acc);
                    if (acc)
                        S.q[base + __popc(b & lt_mask)] = static_cast<unsigned short>((t << SH) | (lane + 32 * hh));
                    base += __popc(b);
                }
                if (lane == t) my_start = N;
                N = base;
            }
            int my_end = __shfl_down_sync(kFull, my_start, 1);
            if (lane == nt - 1) my_end = N;
            __syncwarp();
            // ---- evaluate: lane l takes the queue block [l R, (l + 1) R) and keeps register
            //      sums for the current target; a run is written to its slot when the target
            //      changes (runs start at a block start or at a target's first pair)
            const int R = (N + 31) >> 5;
            const int b0 = min(N, lane * R), b1 = min(N, b0 + R);
            int cur = -1, first = b0;
            T pp = 0, gx = 0, gy = 0, gz = 0;
            for (int i = b0; i < b1; ++i) {
                const int qe = S.q[i];
                const int t = qe >> SH, j = qe & (CW - 1);
                if (t != cur) {
                    if (cur >= 0) {
                        const int sl = (first == b0) ? lane : 32 + cur;
                        S.rp[sl] = pp;
                        S.rx[sl] = gx;
                        S.ry[sl] = gy;
                        if constexpr (D == 3) S.rz[sl] = gz;
                    }
                    cur = t;
                    first = i;
                    pp = gx = gy = gz = T(0);
                }
                const T xt = S.tx[t], yt = S.ty[t];
                const T zt = (D == 3) ? S.tz[t] : T(0);
                T dx = xt - S.sx[j], dy = yt - S.sy[j];
                T dz = (D == 3) ? zt - S.sz[j] : T(0);
                T r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                T s = r2 * h2inv;
                if constexpr (kLo) {
                    if (s < a.close_s) {
                        // close pair: (x_hi - y_hi) + (x_lo - y_lo); the hi difference is exact
                        dx = (xt - S.sx[j]) + (S.tlx[t] - S.lx[j]);
                        dy = (yt - S.sy[j]) + (S.tly[t] - S.ly[j]);
                        if constexpr (D == 3) dz = (zt - S.sz[j]) + (S.tlz[t] - S.lz[j]);
                        r2 = (D == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
                        s = r2 * h2inv;
                    }
                }
                if (r2 > T(0)) {  // the self pair is skipped
                    if (a.count_in) ++nin;
                    const T q = S.sq[j];
                    const T xc = fma(T(2), s, T(-1));
                    T fa = a.cmA[NA - 1], fb = a.cmB[NH - 1];
#pragma unroll
                    for (int m = NH - 2; m >= 0; --m) {
                        if (m < NA - 1) fa = fma(fa, xc, a.cmA[m]);
                        fb = fma(fb, xc, a.cmB[m]);
                    }
                    if constexpr (D == 3) {
                        // R = (1 - t A)/(4 pi r); grad R = -(1 - t A + t B) dr / (4 pi r^3)
                        const T rinv = fast_rsqrt(r2);
                        const T tt = r2 * rinv * hinv;
                        const T num = fma(-tt, fa, T(1));
                        pp = fma(q * num, rinv, pp);
                        const T gf = -q * fma(tt, fb, num) * rinv * rinv * rinv;
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
            if (cur >= 0) {
                const int sl = (first == b0) ? lane : 32 + cur;
                S.rp[sl] = pp;
                S.rx[sl] = gx;
                S.ry[sl] = gy;
                if constexpr (D == 3) S.rz[sl] = gz;
            }
            __syncwarp();
            // ---- lane t adds its target's runs in queue order to the compensated sums
            if (own && my_end > my_start) {
                const int k0 = my_start / R;
                const int s0 = (my_start == k0 * R) ? k0 : 32 + lane;
                T cp = S.rp[s0], cx = S.rx[s0], cy = S.ry[s0], cz = (D == 3) ? S.rz[s0] : T(0);
                for (int k = k0 + 1; k * R < my_end; ++k) {
                    cp += S.rp[k];
                    cx += S.rx[k];
                    cy += S.ry[k];
                    if constexpr (D == 3) cz += S.rz[k];
                }
                kp.add(cp);
                kx.add(cx);
                ky.add(cy);
                if constexpr (D == 3) kz.add(cz);
            }
            __syncwarp();
        }
        if (own) {
            const double kpot = (D == 3) ? 0.07957747154594766788 : 1.0;
            const double kgrad = (D == 3) ? 0.07957747154594766788 : 0.15915494309189533577;
            const size_t o = size_t(L.tgt_begin + t0 + lane);
            a.pot[o] = kp.value() * kpot;
            if (a.grad) {
                a.grad[o * D + 0] = kx.value() * kgrad;
                a.grad[o * D + 1] = ky.value() * kgrad;
                if (D == 3) a.grad[o * D + 2] = kz.value() * kgrad;
            }
        }
        __syncwarp();
    }
    if (a.count_in) {
        for (int o = 16; o > 0; o >>= 1) nin += __shfl_down_sync(kFull, nin, o);
        if (lane == 0 && nin) atomicAdd(a.count_in, nin);
    }
}

}  // namespace pdmk
