// k_farfield.cuh -- the smooth periodic kernel W_0^(p) by the five-step procedure of
// Sec. 3.6 (Eq. (3.14) and the three-step NUFFT realisation): spreading (type-1 half),
// diagonal scaling (Eq. (3.15a) with the m = 0 mode zeroed, window deconvolution folded
// in), interpolation (type-2 half).  The FFTs are cuFFT calls made by the host.
//
// Window: the prolate phi(z) = psi_{c_w}(2z/w)/psi_{c_w}(0), |z| < w/2 grid units, with
// c_w = pi w / 2 (its transform at the grid's band edge equals its own edge value), as a
// Chebyshev series in s = (2z/w)^2 -- smooth up to the support edge, so its derivative is
// well conditioned in FP32 -- on the unpadded M_1 x ... x M_d grid (Remark 3.1).
//
// Spreading is atomics-free by tile ownership.  Sources are sorted by grid bin; a
// subproblem is a bin and at most a few hundred of its sources.  A CTA accumulates one
// subproblem into a shared-memory tile padded by the window (B + w - 1 per dimension);
// each of its 4 warps owns the tile planes whose last index is congruent to its warp id
// mod 4, so no two threads ever update the same cell, and every cell is updated in point
// order: the result is deterministic.  Tiles go to a slab; the fold kernel adds, for every
// grid cell, the slabs of the subproblems whose padded tile covers it, in a fixed order.
#pragma once
#include "kernels_common.cuh"

namespace pdmk {

constexpr int kSpreadThreads = 128;
constexpr int kSpreadWarps = 4;
constexpr int kSpreadChunk = 128;
constexpr int kMaxW = 20;

// Clenshaw with a compile-time number of terms and coefficients in registers
template <typename T, int NC>
__device__ __forceinline__ T clenshaw_reg_w(const T (&c)[NC], T x) {
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
__device__ __forceinline__ T pswf_window(T z, T half_w_inv2, const T* cw, int nw) {
    const T s = z * z * half_w_inv2;
    return s < T(1) ? clenshaw(cw, nw, fma(T(2), s, T(-1))) : T(0);
}
// value and derivative d/dz
template <typename T>
__device__ __forceinline__ void pswf_window_d(T z, T half_w_inv2, const T* cw, int nw, const T* cd, int nd,
                                              T* v, T* dv) {
    const T s = z * z * half_w_inv2;
    if (s < T(1)) {
        const T x = fma(T(2), s, T(-1));
        *v = clenshaw(cw, nw, x);
        *dv = clenshaw(cd, nd, x) * T(2) * z * half_w_inv2;
    } else {
        *v = T(0);
        *dv = T(0);
    }
}

// dynamic shared memory: tile[Ptot] | win[kSpreadChunk][3][w] | q | koff[kSpreadChunk][3] (int)
template <typename T, int D>
__global__ void __launch_bounds__(kSpreadThreads)
k_spread(SpreadArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T cw[kMaxCheb];
    if (threadIdx.x < a.nW) cw[threadIdx.x] = a.coefW[threadIdx.x];
    T* tile = reinterpret_cast<T*>(smem_raw);
    T* win = tile + a.Ptot;
    T* qv = win + kSpreadChunk * 3 * a.w;
    int* koff = reinterpret_cast<int*>(qv + kSpreadChunk);

    const int4 sp = a.sub[blockIdx.x];
    const int begin = sp.y, count = sp.z;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const int w = a.w;
    // bin coordinates and the tile origin (grid index of tile cell 0) per dimension
    for (int i = tid; i < a.Ptot; i += kSpreadThreads) tile[i] = T(0);
    // plane size: 2D planes are rows of P0 (w entries per point), 3D planes are P0*P1
    const int plane_entries = (D == 3) ? w * w : w;
    __syncthreads();
    for (int c0 = 0; c0 < count; c0 += kSpreadChunk) {
        const int np = min(kSpreadChunk, count - c0);
        if (tid < np) {
            const int pi = begin + c0 + tid;
            const int4 g = a.pt_g0[pi];
            const T* dq = a.pt_dq + size_t(pi) * 4;
            // pt_g0 holds the tile offset of the first window node (0 <= k <= B - 1 per
            // dimension; the tile origin is bin*B - floor(w/2)), computed by the host in FP64
            koff[tid * 3 + 0] = g.x;
            koff[tid * 3 + 1] = g.y;
            koff[tid * 3 + 2] = g.z;
            qv[tid] = dq[3];
            for (int k = 0; k < D; ++k) {
                const T del = dq[k];  // M u - g0 (first node's distance), in grid units
                for (int j = 0; j < w; ++j)
                    win[(tid * 3 + k) * w + j] = pswf_window(del - T(j), a.half_w_inv2, cw, a.nW);
            }
        }
        __syncthreads();
        for (int p = 0; p < np; ++p) {
            const T q = qv[p];
            const int kx = koff[p * 3 + 0], ky = koff[p * 3 + 1];
            const int kz = (D == 3) ? koff[p * 3 + 2] : 0;
            const T* wx = win + (p * 3 + 0) * w;
            const T* wy = win + (p * 3 + 1) * w;
            const T* wz = win + (p * 3 + 2) * w;
            const int klast = (D == 3) ? kz : ky;
            // first owned plane j0: (klast + j0) % 4 == wp
            int j0 = (wp - klast) % kSpreadWarps;
            if (j0 < 0) j0 += kSpreadWarps;
            for (int jl = j0; jl < w; jl += kSpreadWarps) {
                if (D == 3) {
                    const T fz = q * wz[jl];
                    T* plane = tile + (kz + jl) * (a.P0 * a.P1);
                    for (int e = lane; e < plane_entries; e += 32) {
                        const int iy = e / w, ix = e - iy * w;
                        plane[(ky + iy) * a.P0 + kx + ix] += fz * wy[iy] * wx[ix];
                    }
                } else {
                    const T fy = q * wy[jl];
                    T* row = tile + (ky + jl) * a.P0;
                    for (int e = lane; e < plane_entries; e += 32) row[kx + e] += fy * wx[e];
                }
            }
        }
        __syncthreads();
    }
    T* out = a.slab + size_t(blockIdx.x) * a.Ptot;
    for (int i = tid; i < a.Ptot; i += kSpreadThreads) out[i] = tile[i];
}

// 3D spreading with the padded tile in registers (cubic tiles, P = B + W - 1 per dimension,
// compile-time W).  Thread t owns the tile columns (X, Y) = (c % P, c / P) for c = t + NT k
// and keeps their P cells along Z in registers.  Per point the host-computed window offset
// places the w window values of each axis inside a zero-padded row of P values (shared
// memory), and every thread adds  q wx[X] wy[Y] wz[Z]  to its cells: P FMAs per owned column,
// skipped where the column lies outside the point's footprint.  A cell is only ever updated by
// its owner, in point order (deterministic, no atomics).  Clustered bins put hundreds of
// thousands of points into a few tiles; with the tile in registers a CTA takes subproblems
// of up to a thousand points, so the fold adds far fewer slabs per grid cell.
// dynamic shared memory: windows [NT][3][PR] | q [NT]
template <typename T, int W, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_spread3d_reg(SpreadArgs<T> a) {
    constexpr int P = 8 + W - 1;                 // B = 8 per dimension
    constexpr int PP = P * P;
    constexpr int NCOL = (PP + NT - 1) / NT;     // columns per thread
    constexpr int PR = (P * int(sizeof(T)) % 16 == 0) ? P : ((P * int(sizeof(T)) + 15) / 16) * 16 / int(sizeof(T));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T cw[kMaxCheb];
    T* win = reinterpret_cast<T*>(smem_raw);     // [NT][3][PR]
    T* qv = win + NT * 3 * PR;                   // [NT]
    const int tid = threadIdx.x;
    if (tid < a.nW) cw[tid] = a.coefW[tid];
    const int4 sp = a.sub[blockIdx.x];
    const int begin = sp.y, count = sp.z;
    int colx[NCOL], coly[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        const int col = tid + c * NT;
        colx[c] = col < PP ? col % P : 0;
        coly[c] = col < PP ? col / P : -1;       // -1: no column (past the tile)
    }
    T acc[NCOL][P];
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int z = 0; z < P; ++z) acc[c][z] = T(0);
    __syncthreads();
    for (int c0 = 0; c0 < count; c0 += NT) {
        const int np = min(NT, count - c0);
        if (tid < np) {
            const int pi = begin + c0 + tid;
            const int4 g = a.pt_g0[pi];           // window start inside the tile, [0, B) per axis
            const T* dq = a.pt_dq + size_t(pi) * 4;
            const int ko[3] = {g.x, g.y, g.z};
            T* row = win + tid * 3 * PR;
            for (int k = 0; k < 3; ++k) {
                const T del = dq[k];             // M u - g0 (first node's distance), grid units
                T* r = row + k * PR;
                for (int x = 0; x < P; ++x) {
                    const int j = x - ko[k];
                    r[x] = (j >= 0 && j < W) ? pswf_window(del - T(j), a.half_w_inv2, cw, a.nW) : T(0);
                }
            }
            qv[tid] = dq[3];
        }
        __syncthreads();
        for (int p = 0; p < np; ++p) {
            const T* row = win + p * 3 * PR;
            const T q = qv[p];
            T wz[P];
#pragma unroll
            for (int z = 0; z < P; ++z) wz[z] = row[2 * PR + z];
#pragma unroll
            for (int c = 0; c < NCOL; ++c) {
                if (coly[c] < 0) continue;
                const T wxy = q * row[colx[c]] * row[PR + coly[c]];
                if (wxy != T(0)) {
#pragma unroll
                    for (int z = 0; z < P; ++z) acc[c][z] = fma(wxy, wz[z], acc[c][z]);
                }
            }
        }
        __syncthreads();
    }
    T* out = a.slab + size_t(blockIdx.x) * (PP * P);
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        if (coly[c] < 0) continue;
        const int col = tid + c * NT;
#pragma unroll
        for (int z = 0; z < P; ++z) out[z * PP + col] = acc[c][z];
    }
}

template <typename T, int W, int NT>
constexpr size_t spread3d_reg_smem() {
    constexpr int P = 8 + W - 1;
    constexpr int PR = (P * int(sizeof(T)) % 16 == 0) ? P : ((P * int(sizeof(T)) + 15) / 16) * 16 / int(sizeof(T));
    return sizeof(T) * (size_t(NT) * 3 * PR + NT);
}

// Small 2D grids: every warp keeps a private copy of the whole periodic grid in shared memory
// and spreads its own contiguous run of points into it (lanes over the w x w footprint, one
// point at a time: no two lanes touch one cell, every cell is updated in point order).  The
// CTA then sums its warps' copies in warp order and writes one slab; k_fold_whole adds the
// slabs in CTA order.  Deterministic, atomics-free, and it needs no sorting by bin.
template <typename T>
__global__ void __launch_bounds__(256)
k_spread_whole(const int4* __restrict__ t_g0, const T* __restrict__ t_dq, const T* __restrict__ q4, int n,
               T* __restrict__ slab, int M0, int M1, int w, T half_w_inv2, const T* __restrict__ coefW, int nW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T cw[kMaxCheb];
    const int ncell = M0 * M1;
    const int nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T* grids = reinterpret_cast<T*>(smem_raw);        // [nwarp][ncell]
    T* wins = grids + nwarp * ncell;                  // [nwarp][2][w]
    if (threadIdx.x < nW) cw[threadIdx.x] = coefW[threadIdx.x];
    for (int i = threadIdx.x; i < nwarp * ncell; i += blockDim.x) grids[i] = T(0);
    __syncthreads();
    T* g = grids + wp * ncell;
    T* wv = wins + wp * 2 * w;
    const int gw = blockIdx.x * nwarp + wp, nw = gridDim.x * nwarp;
    const int per = (n + nw - 1) / nw;
    const int i0 = min(n, gw * per), i1 = min(n, i0 + per);
    const int ww = w * w;
    for (int i = i0; i < i1; ++i) {
        const int4 g0 = t_g0[i];
        const T* dq = t_dq + size_t(i) * 4;
        for (int l = lane; l < 2 * w; l += 32) {
            const int k = l / w, j = l % w;
            wv[l] = pswf_window(dq[k] - T(j), half_w_inv2, cw, nW);
        }
        __syncwarp();
        const T q = q4[size_t(i) * 4 + 3];
        int x0 = g0.x % M0;
        if (x0 < 0) x0 += M0;
        int y0 = g0.y % M1;
        if (y0 < 0) y0 += M1;
        for (int e = lane; e < ww; e += 32) {
            const int iy = e / w, ix = e - iy * w;
            int xx = x0 + ix;
            if (xx >= M0) xx -= M0;
            int yy = y0 + iy;
            if (yy >= M1) yy -= M1;
            g[yy * M0 + xx] += q * wv[w + iy] * wv[ix];
        }
        __syncwarp();
    }
    __syncthreads();
    T* out = slab + size_t(blockIdx.x) * ncell;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        T s = T(0);
        for (int k = 0; k < nwarp; ++k) s += grids[k * ncell + c];
        out[c] = s;
    }
}

// The same with compile-time window width W and window-series length NWC (coefficients in
// registers, footprint index arithmetic folded by the compiler).
template <typename T, int W, int NWC>
__global__ void __launch_bounds__(256)
k_spread_whole_w(const int4* __restrict__ t_g0, const T* __restrict__ t_dq, const T* __restrict__ q4, int n,
                 T* __restrict__ slab, int M0, int M1, T half_w_inv2, const T* __restrict__ coefW, int nW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int WW = W * W, KK = (WW + 31) / 32;
    const int ncell = M0 * M1;
    const int nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T* grids = reinterpret_cast<T*>(smem_raw);  // [nwarp][ncell]
    T* wins = grids + nwarp * ncell;            // [nwarp][2 W]
    T cw[NWC];
#pragma unroll
    for (int k = 0; k < NWC; ++k) cw[k] = k < nW ? coefW[k] : T(0);
    for (int i = threadIdx.x; i < nwarp * ncell; i += blockDim.x) grids[i] = T(0);
    __syncthreads();
    T* g = grids + wp * ncell;
    T* wv = wins + wp * 2 * W;
    int fy[KK], fx[KK];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        const int e = lane + 32 * k;
        fy[k] = e < WW ? e / W : -1;
        fx[k] = e < WW ? e % W : 0;
    }
    const int gw = blockIdx.x * nwarp + wp, nw = gridDim.x * nwarp;
    const int per = (n + nw - 1) / nw;
    const int i0 = min(n, gw * per), i1 = min(n, i0 + per);
    for (int i = i0; i < i1; ++i) {
        const int4 g0 = t_g0[i];
        const T* dq = t_dq + size_t(i) * 4;
#pragma unroll
        for (int l0 = 0; l0 < 2 * W; l0 += 32) {
            const int l = l0 + lane;
            if (l < 2 * W) {
                const int k = l / W, j = l - (l / W) * W;
                const T z = dq[k] - T(j);
                const T s = z * z * half_w_inv2;
                wv[l] = s < T(1) ? clenshaw_reg_w<T, NWC>(cw, fma(T(2), s, T(-1))) : T(0);
            }
        }
        __syncwarp();
        const T q = q4[size_t(i) * 4 + 3];
        int x0 = g0.x % M0;
        if (x0 < 0) x0 += M0;
        int y0 = g0.y % M1;
        if (y0 < 0) y0 += M1;
#pragma unroll
        for (int k = 0; k < KK; ++k) {
            if (fy[k] >= 0) {
                int xx = x0 + fx[k];
                if (xx >= M0) xx -= M0;
                int yy = y0 + fy[k];
                if (yy >= M1) yy -= M1;
                g[yy * M0 + xx] += q * wv[W + fy[k]] * wv[fx[k]];
            }
        }
        __syncwarp();
    }
    __syncthreads();
    T* out = slab + size_t(blockIdx.x) * ncell;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        T s = T(0);
        for (int k = 0; k < nwarp; ++k) s += grids[k * ncell + c];
        out[c] = s;
    }
}

// Sum of the per-CTA slabs: a block takes 32 cells (one per lane); its eight warps split the
// slabs, and warp 0 adds the eight partials in order.
template <typename T, typename G>
__global__ void __launch_bounds__(256) k_fold_whole(const T* __restrict__ slab, int nslab, G* __restrict__ grid,
                                                    int ncell) {
    __shared__ T part[8][32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    T s = T(0);
    if (c < ncell)
        for (int k = wp; k < nslab; k += 8) s += slab[size_t(k) * ncell + c];
    part[wp][lane] = s;
    __syncthreads();
    if (wp == 0 && c < ncell) {
        T t = part[0][lane];
        for (int k = 1; k < 8; ++k) t += part[k][lane];
        grid[c] = G(t);
    }
}

// fold: grid cell g gathers every subproblem tile that covers it (periodic wrap)
template <typename T, int D, typename G>
__global__ void k_fold(FoldArgs<T, G> a) {
    const int64_t ncell = int64_t(a.M0) * a.M1 * (D == 3 ? a.M2 : 1);
    for (int64_t cell = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; cell < ncell;
         cell += int64_t(gridDim.x) * blockDim.x) {
        const int g0 = int(cell % a.M0);
        const int g1 = int((cell / a.M0) % a.M1);
        const int g2 = (D == 3) ? int(cell / (int64_t(a.M0) * a.M1)) : 0;
        // candidate bins per dimension: the tile of bin b starts at b*B - fw and spans P
        int cb0[8], lo0[8], n0 = 0;
        int cb1[8], lo1[8], n1 = 0;
        int cb2[8], lo2[8], n2 = 0;
        auto collect = [&](int g, int M, int B, int P, int nb, int* cb, int* lo, int& n) {
            for (int b = 0; b < nb && n < 8; ++b) {
                int off = g - (b * B - a.fw);
                off %= M;
                if (off < 0) off += M;
                if (off < P) { cb[n] = b; lo[n] = off; ++n; }
            }
        };
        collect(g0, a.M0, a.B0, a.P0, a.nb0, cb0, lo0, n0);
        collect(g1, a.M1, a.B1, a.P1, a.nb1, cb1, lo1, n1);
        if (D == 3) collect(g2, a.M2, a.B2, a.P2, a.nb2, cb2, lo2, n2);
        else { cb2[0] = 0; lo2[0] = 0; n2 = 1; }
        // the slabs are added in the grid's precision (FP64 for the FP64 transforms)
        G acc = G(0);
        for (int i2 = 0; i2 < n2; ++i2)
            for (int i1 = 0; i1 < n1; ++i1)
                for (int i0 = 0; i0 < n0; ++i0) {
                    const int bin = (cb2[i2] * a.nb1 + cb1[i1]) * a.nb0 + cb0[i0];
                    const int idx = (lo2[i2] * a.P1 + lo1[i1]) * a.P0 + lo0[i0];
                    for (int s = a.bin_sub_begin[bin]; s < a.bin_sub_begin[bin + 1]; ++s)
                        acc += G(a.slab[size_t(s) * a.Ptot + idx]);
                }
        a.grid[cell] = acc;
    }
}

// diagonal scaling of the half spectrum by precomputed FP64 weights (zero at m = 0 and on
// the Nyquist planes)
template <typename T>
__global__ void k_scale(T* spec /* interleaved complex */, const double* weight, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double wgt = weight[i];
        spec[2 * i] = T(double(spec[2 * i]) * wgt);
        spec[2 * i + 1] = T(double(spec[2 * i + 1]) * wgt);
    }
}

// grid precision change around the FP64 transforms (grid-stride)
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = B(in[i]);
}

// 3D interpolation with a compile-time window width W, a thread per target: the x-axis
// window values and their derivatives sit in registers, the y and z ones in shared memory
// (one read per grid row).  The block's targets are consecutive in the sorted order and
// usually close together: when the union of their windows fits kInterpTile cells, the block
// copies that part of the grid into shared memory once (coalesced along x, indices wrapped on
// the way in) and every thread reads its window there; otherwise each thread reads the grid
// through the read-only cache with its rows' offsets wrapped once.  Each grid value costs one
// load and two multiply-adds either way.
constexpr int kInterpTile = 8192;  // grid values of the shared tile
template <typename T, int W>
constexpr size_t interp3d_w_smem() {
    return sizeof(T) * (size_t(4) * W * 128 + kInterpTile);
}

template <typename T, int W>
__global__ void __launch_bounds__(128)
k_interp3d_w(InterpArgs<T> a) {
    __shared__ T cw[kMaxCheb], cd[kMaxCheb];
    __shared__ int bmin[3], bmax[3];
    extern __shared__ __align__(16) unsigned char smi[];
    T (*wyz)[W][128] = reinterpret_cast<T (*)[W][128]>(smi);  // [4][W][128]: (value, derivative) x (y, z)
    T* tile = reinterpret_cast<T*>(smi) + 4 * W * 128;
    if (threadIdx.x < a.nW) cw[threadIdx.x] = a.coefW[threadIdx.x];
    if (threadIdx.x < a.nWd) cd[threadIdx.x] = a.coefWd[threadIdx.x];
    if (threadIdx.x < 3) {
        bmin[threadIdx.x] = 0x7fffffff;
        bmax[threadIdx.x] = -1;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < a.nt;
    const int tx = threadIdx.x;
    int4 g = make_int4(0, 0, 0, 0);
    T wx[W], dwx[W];
    if (valid) {
        g = a.t_g0[t];  // window starts wrapped into [0, M)
        const T* dq = a.t_dq + size_t(t) * 4;
#pragma unroll
        for (int j = 0; j < W; ++j) pswf_window_d(dq[0] - T(j), a.half_w_inv2, cw, a.nW, cd, a.nWd, &wx[j], &dwx[j]);
        for (int k = 1; k < 3; ++k) {
            const T del = dq[k];
            for (int j = 0; j < W; ++j) {
                T v, dv;
                pswf_window_d(del - T(j), a.half_w_inv2, cw, a.nW, cd, a.nWd, &v, &dv);
                wyz[2 * (k - 1)][j][tx] = v;
                wyz[2 * (k - 1) + 1][j][tx] = dv;
            }
        }
        atomicMin(&bmin[0], g.x);
        atomicMax(&bmax[0], g.x);
        atomicMin(&bmin[1], g.y);
        atomicMax(&bmax[1], g.y);
        atomicMin(&bmin[2], g.z);
        atomicMax(&bmax[2], g.z);
    }
    __syncthreads();
    const int ex = bmax[0] - bmin[0] + W, ey = bmax[1] - bmin[1] + W, ez = bmax[2] - bmin[2] + W;
    const bool use_tile = bmax[0] >= 0 && ex * ey * ez <= kInterpTile;  // block-uniform
    if (use_tile) {
        for (int i = tx; i < ex * ey * ez; i += 128) {
            const int ix = i % ex, iy = (i / ex) % ey, iz = i / (ex * ey);
            int gx = bmin[0] + ix, gy = bmin[1] + iy, gz = bmin[2] + iz;
            while (gx >= a.M0) gx -= a.M0;
            while (gy >= a.M1) gy -= a.M1;
            while (gz >= a.M2) gz -= a.M2;
            tile[i] = __ldg(a.grid + (size_t(gz) * a.M1 + gy) * a.M0 + gx);
        }
        __syncthreads();
    }
    if (!valid) return;
    T pot = 0, gx = 0, gy = 0, gz = 0;
    if (use_tile) {
        const int ox = g.x - bmin[0], oy = g.y - bmin[1], oz = g.z - bmin[2];
        for (int iz = 0; iz < W; ++iz) {
            const T wz = wyz[2][iz][tx], dwz = wyz[3][iz][tx];
            T py = 0, gxy = 0, gyy = 0;
            for (int iy = 0; iy < W; ++iy) {
                const T* row = tile + ((oz + iz) * ey + (oy + iy)) * ex + ox;
                T sx = 0, sdx = 0;
#pragma unroll
                for (int ix = 0; ix < W; ++ix) {
                    const T v = row[ix];
                    sx = fma(v, wx[ix], sx);
                    sdx = fma(v, dwx[ix], sdx);
                }
                const T wy = wyz[0][iy][tx], dwy = wyz[1][iy][tx];
                py = fma(sx, wy, py);
                gxy = fma(sdx, wy, gxy);
                gyy = fma(sx, dwy, gyy);
            }
            pot = fma(py, wz, pot);
            gx = fma(gxy, wz, gx);
            gy = fma(gyy, wz, gy);
            gz = fma(py, dwz, gz);
        }
    } else {
        int xi[W];
        {
            int xx = g.x;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                xi[j] = xx;
                if (++xx == a.M0) xx = 0;
            }
        }
        int zz = g.z, yy0 = g.y;
        for (int iz = 0; iz < W; ++iz) {
            const T wz = wyz[2][iz][tx], dwz = wyz[3][iz][tx];
            const T* plane = a.grid + size_t(zz) * a.M1 * a.M0;
            int yy = yy0;
            T py = 0, gxy = 0, gyy = 0;
            for (int iy = 0; iy < W; ++iy) {
                const T* row = plane + size_t(yy) * a.M0;
                T sx = 0, sdx = 0;
#pragma unroll
                for (int ix = 0; ix < W; ++ix) {
                    const T v = __ldg(row + xi[ix]);
                    sx = fma(v, wx[ix], sx);
                    sdx = fma(v, dwx[ix], sdx);
                }
                const T wy = wyz[0][iy][tx], dwy = wyz[1][iy][tx];
                py = fma(sx, wy, py);
                gxy = fma(sdx, wy, gxy);
                gyy = fma(sx, dwy, gyy);
                if (++yy == a.M1) yy = 0;
            }
            pot = fma(py, wz, pot);
            gx = fma(gxy, wz, gx);
            gy = fma(gyy, wz, gy);
            gz = fma(py, dwz, gz);
            if (++zz == a.M2) zz = 0;
        }
    }
    a.pot[t] = double(pot);
    a.gradu[size_t(t) * 3 + 0] = double(gx);
    a.gradu[size_t(t) * 3 + 1] = double(gy);
    a.gradu[size_t(t) * 3 + 2] = double(gz);
}

// interpolation at targets: potential and gradient w.r.t. the grid coordinates
template <typename T, int D>
__global__ void __launch_bounds__(128)
k_interp(InterpArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T cw[kMaxCheb], cd[kMaxCheb];
    if (threadIdx.x < a.nW) cw[threadIdx.x] = a.coefW[threadIdx.x];
    if (threadIdx.x < a.nWd) cd[threadIdx.x] = a.coefWd[threadIdx.x];
    __syncthreads();
    // window values and derivatives, interleaved by thread: element k of thread t at
    // k * blockDim + t (lanes never share a bank)
    T* wv = reinterpret_cast<T*>(smem_raw);
    T* wd = wv + blockDim.x * D * a.w;
    const int w = a.w;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nt) return;
    const int4 g = a.t_g0[t];
    const T* dq = a.t_dq + size_t(t) * 4;
    const int bs = blockDim.x;
    T* myv = wv + threadIdx.x;
    T* myd = wd + threadIdx.x;
    for (int k = 0; k < D; ++k) {
        const T del = dq[k];
        for (int j = 0; j < w; ++j) {
            T v, dv;
            pswf_window_d(del - T(j), a.half_w_inv2, cw, a.nW, cd, a.nWd, &v, &dv);
            myv[(k * w + j) * bs] = v;
            myd[(k * w + j) * bs] = dv;
        }
    }
    // the window argument is del - j = M u - (g0 + j), so d/d(M u) phi(del - j) = phi'(del - j)
    T pot = 0, gx = 0, gy = 0, gz = 0;
    const int gx0 = g.x, gy0 = g.y, gz0 = g.z;
    if (D == 2) {
        for (int iy = 0; iy < w; ++iy) {
            int yy = gy0 + iy;
            yy %= a.M1;
            if (yy < 0) yy += a.M1;
            const T* row = a.grid + size_t(yy) * a.M0;
            T sx = 0, sdx = 0;
            int xx = gx0 % a.M0;
            if (xx < 0) xx += a.M0;
            for (int ix = 0; ix < w; ++ix) {
                const T v = __ldg(row + xx);
                sx = fma(v, myv[(ix) * bs], sx);
                sdx = fma(v, myd[(ix) * bs], sdx);
                if (++xx == a.M0) xx = 0;
            }
            pot = fma(sx, myv[(w + iy) * bs], pot);
            gx = fma(sdx, myv[(w + iy) * bs], gx);
            gy = fma(sx, myd[(w + iy) * bs], gy);
        }
    } else {
        for (int iz = 0; iz < w; ++iz) {
            int zz = gz0 + iz;
            zz %= a.M2;
            if (zz < 0) zz += a.M2;
            for (int iy = 0; iy < w; ++iy) {
                int yy = gy0 + iy;
                yy %= a.M1;
                if (yy < 0) yy += a.M1;
                const T* row = a.grid + (size_t(zz) * a.M1 + yy) * a.M0;
                T sx = 0, sdx = 0;
                int xx = gx0 % a.M0;
                if (xx < 0) xx += a.M0;
                for (int ix = 0; ix < w; ++ix) {
                    const T v = __ldg(row + xx);
                    sx = fma(v, myv[(ix) * bs], sx);
                    sdx = fma(v, myd[(ix) * bs], sdx);
                    if (++xx == a.M0) xx = 0;
                }
                const T fyz = myv[(w + iy) * bs] * myv[(2 * w + iz) * bs];
                pot = fma(sx, fyz, pot);
                gx = fma(sdx, fyz, gx);
                gy = fma(sx, myd[(w + iy) * bs] * myv[(2 * w + iz) * bs], gy);
                gz = fma(sx, myv[(w + iy) * bs] * myd[(2 * w + iz) * bs], gz);
            }
        }
    }
    a.pot[t] = double(pot);
    a.gradu[size_t(t) * D + 0] = double(gx);
    a.gradu[size_t(t) * D + 1] = double(gy);
    if (D == 3) a.gradu[size_t(t) * D + 2] = double(gz);
}

// ---------------------------------------------------------------------------------------
// 2D FP32 spreading and interpolation with compile-time window width W and series length NH.
// The window series F (and dF for the gradient) are Horner sums of monomials in
// x = 2 s - 1 (the host converts the Chebyshev fits; for these series Horner is as accurate
// as Clenshaw).  Window starts arrive wrapped into [0, M_i), and the grids carry a halo of
// W - 1 cells on the high side of each axis, so a window never wraps inside the kernel; the
// halo folds back onto the periodic grid (spreading) or is filled from it (interpolation).
// Needs W - 1 <= min(M0, M1).
template <typename T, int NH>
__device__ __forceinline__ T horner(const T (&c)[NH], T x) {
    T r = c[NH - 1];
#pragma unroll
    for (int k = NH - 2; k >= 0; --k) r = fma(r, x, c[k]);
    return r;
}

// Per-warp private halo grids [nwarp][(M0 + W - 1)(M1 + W - 1)]; a warp takes a contiguous
// range of points (sorted order) and adds each point's W x W block (lanes over the cells,
// so one instruction never touches a cell twice).  The block folds the halo and its warps'
// copies in a fixed order into its slab; k_fold_whole sums the slabs.
template <typename T, int W, int NH>
__global__ void __launch_bounds__(256, 2)
k_spread_halo(const int4* __restrict__ t_g0, const T* __restrict__ t_dq, const T* __restrict__ q4, int n,
              T* __restrict__ slab, int M0, int M1, T half_w_inv2, const T* __restrict__ monoW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int WW = W * W, KK = (WW + 31) / 32;
    const int Mp0 = M0 + W - 1, Mp1 = M1 + W - 1, np = Mp0 * Mp1;
    const int nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T* grids = reinterpret_cast<T*>(smem_raw);  // [nwarp][np]
    T* wins = grids + nwarp * np;               // [nwarp][2 W]: x window, q * y window
    T cw[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) cw[k] = monoW[k];
    for (int i = threadIdx.x; i < nwarp * np; i += blockDim.x) grids[i] = T(0);
    __syncthreads();
    T* g = grids + wp * np;
    T* wv = wins + wp * 2 * W;
    int off[KK], fxy[KK];  // cell offset in the halo grid; x | (W + y) << 16 window indices
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        const int e = lane + 32 * k;
        const int fy = e < WW ? e / W : 0, fx = e < WW ? e % W : 0;
        fxy[k] = fx | ((W + fy) << 16);
        off[k] = e < WW ? fy * Mp0 + fx : -1;
    }
    const int gw = blockIdx.x * nwarp + wp, nw = gridDim.x * nwarp;
    const int per = (n + nw - 1) / nw;
    const int i0 = min(n, gw * per), i1 = min(n, i0 + per);
    // points in chunks of 32: one coalesced load per lane, then broadcast point by point
    for (int c0 = i0; c0 < i1; c0 += 32) {
        const int ii = c0 + lane;
        int pb = 0;
        T pdx = T(0), pdy = T(0), pq = T(0);
        if (ii < i1) {
            const int4 g0 = t_g0[ii];
            pb = g0.y * Mp0 + g0.x;
            pdx = t_dq[size_t(ii) * 4 + 0];
            pdy = t_dq[size_t(ii) * 4 + 1];
            pq = q4[size_t(ii) * 4 + 3];
        }
        const int cnt = min(32, i1 - c0);
        for (int j = 0; j < cnt; ++j) {
            const int base = __shfl_sync(0xffffffffu, pb, j);
            const T dx = __shfl_sync(0xffffffffu, pdx, j), dy = __shfl_sync(0xffffffffu, pdy, j);
            const T q = __shfl_sync(0xffffffffu, pq, j);
            if (lane < 2 * W) {
                const bool ky = lane >= W;
                const T z = (ky ? dy : dx) - T(ky ? lane - W : lane);
                const T s = z * z * half_w_inv2;
                const T v = s < T(1) ? horner(cw, fma(T(2), s, T(-1))) : T(0);
                wv[lane] = ky ? v * q : v;
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < KK; ++k)
                if (off[k] >= 0) g[base + off[k]] += wv[fxy[k] >> 16] * wv[fxy[k] & 0xffff];
            __syncwarp();
        }
    }
    __syncthreads();
    T* out = slab + size_t(blockIdx.x) * (size_t(M0) * M1);
    for (int y = wp; y < M1; y += nwarp)
        for (int x = lane; x < M0; x += 32) {
            const bool hx = x + M0 < Mp0, hy = y + M1 < Mp1;
            T s = T(0);
            for (int k = 0; k < nwarp; ++k) {
                const T* gk = grids + k * np;
                s += gk[y * Mp0 + x];
                if (hx) s += gk[y * Mp0 + x + M0];
                if (hy) {
                    s += gk[(y + M1) * Mp0 + x];
                    if (hx) s += gk[(y + M1) * Mp0 + x + M0];
                }
            }
            out[y * M0 + x] = s;
        }
}

// Interpolation of the potential and its grid-coordinate gradient: each block copies the
// periodic grid into a halo grid in shared memory once, then its threads take targets in a
// grid-stride loop (one target per thread).
template <typename T, int W, int NH, int NHD, typename G>
__global__ void __launch_bounds__(256, 2)
k_interp_halo(const G* __restrict__ grid, const int4* __restrict__ t_g0, const T* __restrict__ t_dq, int nt, int M0,
              int M1, T half_w_inv2, const T* __restrict__ monoW, const T* __restrict__ monoWd,
              double* __restrict__ pot, double* __restrict__ gradu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Mp0 = M0 + W - 1, Mp1 = M1 + W - 1;
    T* gs = reinterpret_cast<T*>(smem_raw);  // [Mp1][Mp0]
    for (int y = threadIdx.x / 32; y < Mp1; y += blockDim.x / 32) {
        const int yy = y < M1 ? y : y - M1;
        for (int x = threadIdx.x & 31; x < Mp0; x += 32) gs[y * Mp0 + x] = T(grid[yy * M0 + (x < M0 ? x : x - M0)]);
    }
    T cw[NH], cd[NHD];
#pragma unroll
    for (int k = 0; k < NH; ++k) cw[k] = monoW[k];
#pragma unroll
    for (int k = 0; k < NHD; ++k) cd[k] = monoWd[k];
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const int4 g0 = t_g0[t];
        const T dx = t_dq[size_t(t) * 4 + 0], dy = t_dq[size_t(t) * 4 + 1];
        T wx[W], dwx[W], wy[W], dwy[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            // phi(z) = F(2 s - 1), s = z^2 / (w/2)^2;  phi'(z) = dF(2 s - 1) 2 z / (w/2)^2
            const T zx = dx - T(j), zy = dy - T(j);
            const T sx = zx * zx * half_w_inv2, sy = zy * zy * half_w_inv2;
            const bool ix = sx < T(1), iy = sy < T(1);
            const T xx = fma(T(2), sx, T(-1)), xy = fma(T(2), sy, T(-1));
            wx[j] = ix ? horner(cw, xx) : T(0);
            wy[j] = iy ? horner(cw, xy) : T(0);
            dwx[j] = ix ? horner(cd, xx) * T(2) * zx * half_w_inv2 : T(0);
            dwy[j] = iy ? horner(cd, xy) * T(2) * zy * half_w_inv2 : T(0);
        }
        T p = 0, gx = 0, gy = 0;
        const T* row = gs + g0.y * Mp0 + g0.x;
#pragma unroll
        for (int iy = 0; iy < W; ++iy) {
            T sx = 0, sdx = 0;
#pragma unroll
            for (int ix = 0; ix < W; ++ix) {
                const T v = row[iy * Mp0 + ix];
                sx = fma(v, wx[ix], sx);
                sdx = fma(v, dwx[ix], sdx);
            }
            p = fma(sx, wy[iy], p);
            gx = fma(sdx, wy[iy], gx);
            gy = fma(sx, dwy[iy], gy);
        }
        pot[t] = double(p);
        gradu[size_t(t) * 2 + 0] = double(gx);
        gradu[size_t(t) * 2 + 1] = double(gy);
    }
}

}  // namespace pdmk

namespace pdmk {

// 3D interpolation of the potential and its grid-coordinate gradient, one warp per target
// (small cells have few targets, and a thread per target left most of the GPU idle): lanes
// evaluate the 3 W window values and derivatives (Horner sums of monomials in x = 2 s - 1),
// then take the W^2 (y, z) rows in turn, each row a W-point contraction along x; a warp
// reduction in a fixed order combines the lanes.  Window starts arrive wrapped into
// [0, M_i); needs W - 1 <= min(M0, M1, M2).
template <typename T, int W, int NH, int NHD>
__global__ void __launch_bounds__(256)
k_interp_warp3d(const T* __restrict__ grid, const int4* __restrict__ t_g0, const T* __restrict__ t_dq, int nt, int M0,
                int M1, int M2, T half_w_inv2, const T* __restrict__ monoW, const T* __restrict__ monoWd,
                double* __restrict__ pot, double* __restrict__ gradu) {
    __shared__ T win[8][2][3][W];  // [warp][value, derivative][axis][j]
    T cw[NH], cd[NHD];
#pragma unroll
    for (int k = 0; k < NH; ++k) cw[k] = monoW[k];
#pragma unroll
    for (int k = 0; k < NHD; ++k) cd[k] = monoWd[k];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nt; t += nw) {
        const int4 g0 = t_g0[t];
        for (int l = lane; l < 3 * W; l += 32) {
            const int a = l / W, j = l - a * W;
            const T z = t_dq[size_t(t) * 4 + a] - T(j);
            const T s = z * z * half_w_inv2;
            const bool in = s < T(1);
            const T x = fma(T(2), s, T(-1));
            T v = cw[NH - 1], dv = cd[NHD - 1];
#pragma unroll
            for (int k = NH - 2; k >= 0; --k) v = fma(v, x, cw[k]);
#pragma unroll
            for (int k = NHD - 2; k >= 0; --k) dv = fma(dv, x, cd[k]);
            // phi(z) = F(2 s - 1), phi'(z) = dF(2 s - 1) 2 z / (w/2)^2
            win[wp][0][a][j] = in ? v : T(0);
            win[wp][1][a][j] = in ? dv * T(2) * z * half_w_inv2 : T(0);
        }
        __syncwarp();
        T p = 0, gx = 0, gy = 0, gz = 0;
        for (int r = lane; r < W * W; r += 32) {
            const int iz = r / W, iy = r - iz * W;
            int yy = g0.y + iy;
            if (yy >= M1) yy -= M1;
            int zz = g0.z + iz;
            if (zz >= M2) zz -= M2;
            const T* row = grid + (size_t(zz) * M1 + yy) * M0;
            T sx = 0, sdx = 0;
            int xx = g0.x;
#pragma unroll
            for (int ix = 0; ix < W; ++ix) {
                const T v = __ldg(row + xx);
                sx = fma(v, win[wp][0][0][ix], sx);
                sdx = fma(v, win[wp][1][0][ix], sdx);
                if (++xx == M0) xx = 0;
            }
            const T wy = win[wp][0][1][iy], dwy = win[wp][1][1][iy];
            const T wz = win[wp][0][2][iz], dwz = win[wp][1][2][iz];
            p = fma(sx, wy * wz, p);
            gx = fma(sdx, wy * wz, gx);
            gy = fma(sx, dwy * wz, gy);
            gz = fma(sx, wy * dwz, gz);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_down_sync(0xffffffffu, p, o);
            gx += __shfl_down_sync(0xffffffffu, gx, o);
            gy += __shfl_down_sync(0xffffffffu, gy, o);
            gz += __shfl_down_sync(0xffffffffu, gz, o);
        }
        if (lane == 0) {
            pot[t] = double(p);
            gradu[size_t(t) * 3 + 0] = double(gx);
            gradu[size_t(t) * 3 + 1] = double(gy);
            gradu[size_t(t) * 3 + 2] = double(gz);
        }
        __syncwarp();
    }
}

}  // namespace pdmk
