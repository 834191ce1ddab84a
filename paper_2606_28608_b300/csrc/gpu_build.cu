// gpu_build.cu -- the source set-up on the device (Algorithm 1, steps 1-2; images of Sec. 3.4).
//
// Every point copy gets a 64-bit key: its root cell (axis 0 fastest, as the host's root
// sort), then the interleaved bits of its cell at a fixed deep level K (axis a at bit a of
// each d-bit digit, the coarsest digit first).  Sorted by key, the points of any box at level
// L <= K form one contiguous run: the key prefix of the box.  The tree then follows from runs:
//   * refinement: the boxes with more than n_s points below max_depth are the runs of more
//     than n_s keys at each level (their ancestors are such runs too, so they exist);
//   * level restriction (every colleague of the parent of a non-leaf box is non-leaf): one
//     sweep from the deepest level up, adding the parent's colleagues of every non-leaf box
//     of level L to the non-leaf set of level L - 1.  A forced split only makes leaves (a
//     child with more than n_s points would have split its parent already), so one sweep
//     reaches the closure;
//   * the boxes of level L are the 2^d children of the non-leaf boxes of level L - 1, in key
//     order, which is the host's level order (children of consecutive parents, in order).
// The final order of the sources is by leaf and, within a leaf, by image index (a stable sort
// of the image-ordered copies by their leaf's first position), the order the host's stable
// splits leave.  All FP64 arithmetic is written with explicit round-to-nearest operations so
// that no multiply-add is contracted: every coordinate, bound and record equals the host's.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_select.cuh>

#include <algorithm>
#include <chrono>
#include <cstring>

#include "gpu_build.h"
#include "kernels_common.cuh"
#include "pdmk.h"

namespace pdmk {
namespace {

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

constexpr int kThreads = 256;
inline int blocks_for(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 1 << 20))); }

struct Geo {
    int d;
    int periodic;
    double Q[9], R[9], Rinv[9];
    double lo[3], hi[3], rc;
    double rdiag[3];  // 1 / R[a][a]
    double inv_rc;    // 1 / r_c
    int nroot[3];
};

Geo make_geo(const Geometry& g) {
    Geo o;
    std::memset(&o, 0, sizeof(o));
    o.d = g.d;
    o.periodic = g.periodic_root ? 1 : 0;
    std::memcpy(o.Q, g.Q, sizeof(o.Q));
    std::memcpy(o.R, g.R, sizeof(o.R));
    std::memcpy(o.Rinv, g.Rinv, sizeof(o.Rinv));
    for (int i = 0; i < 3; ++i) {
        o.lo[i] = g.lo[i];
        o.hi[i] = i < g.d ? g.lo[i] + g.nroot[i] * g.rc : 0.0;  // as the host build
        o.nroot[i] = i < g.d ? g.nroot[i] : 1;
    }
    o.rc = g.rc;
    for (int a = 0; a < g.d; ++a) o.rdiag[a] = 1.0 / g.R[a * g.d + a];
    o.inv_rc = 1.0 / g.rc;  // as the host build
    return o;
}

struct ImgTab {
    int ns;
    int Bx[3];
    long long dimx[3];
    const int* sidx;
    const double* trs;
};

// ---------------------------------------------------------------------------------------
// orientation and wrapping; input checks

__global__ void k_orient(Geo g, int64_t n, const double* __restrict__ y, double* __restrict__ u) {
    const int d = g.d;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        double xo[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) xo[i] = dadd(xo[i], dmul(g.Q[i * d + k], y[j * d + k]));
        for (int i = 0; i < d; ++i) {
            double s = 0;
            for (int k = 0; k < d; ++k) s = dadd(s, dmul(g.Rinv[i * d + k], xo[k]));
            s = dsub(s, floor(s));
            if (s >= 1.0) s = 0.0;
            u[j * d + i] = s;
        }
    }
}

__global__ void k_check(int64_t n, int d, const double* __restrict__ y, const double* __restrict__ q,
                        int* __restrict__ nonfinite, double* __restrict__ part) {
    __shared__ double sh[2][kThreads];
    double s = 0, a = 0;
    bool bad = false;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        for (int k = 0; k < d; ++k) bad |= !isfinite(y[j * d + k]);
        const double v = q[j];
        bad |= !isfinite(v);
        s += v;
        a += fabs(v);
    }
    if (bad) atomicOr(nonfinite, 1);
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = a;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh[0][0];
        part[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// ---------------------------------------------------------------------------------------
// images (Sec. 3.4): the host's candidate ranges and in-box test.  The in-box test is the
// host's arithmetic for arithmetic.  The candidate ranges take the reciprocal of the diagonal
// entry instead of dividing by it (FP64 division is slow on this part, and the ranges are
// computed about ten times per point); they carry a slack of 1e-9 (1 + |bound|), far above
// the few ulps this changes, so every shift the in-box test accepts is still a candidate
// and the accepted shifts, in the host's order, are the same.

// D: the dimension (compile-time, so that the loops unroll and the small arrays stay in
// registers)
template <int D>
__device__ __forceinline__ void frac_to_tree(const Geo& g, const double* uj, double* x) {
    constexpr int d = D;
    for (int i = 0; i < d; ++i) {
        double v = 0;
        for (int k = i; k < d; ++k) v = dadd(v, dmul(g.R[i * d + k], uj[k]));
        x[i] = v;
    }
}

template <int D>
__device__ __forceinline__ bool in_domain(const Geo& g, const ImgTab& t, const double* x, int k) {
    bool in = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double p = dadd(x[a], t.trs[k * 3 + a]);
        in &= (p >= g.lo[a] && p < g.hi[a]);
    }
    return in;
}

template <int D>
__device__ __forceinline__ void shift_range(const Geo& g, const ImgTab& t, const double* x, int a, const int* nv,
                                            int* lo_n, int* hi_n) {
    constexpr int d = D;
    double off = 0;
    for (int k = a + 1; k < d; ++k) off = dadd(off, dmul(g.R[a * d + k], double(nv[k])));
    const double l = dmul(dsub(dsub(g.lo[a], x[a]), off), g.rdiag[a]);
    const double h = dmul(dsub(dsub(g.hi[a], x[a]), off), g.rdiag[a]);
    const double sl = dmul(1e-9, dadd(1.0, fabs(l))), sh = dmul(1e-9, dadd(1.0, fabs(h)));
    *lo_n = max(-t.Bx[a], int(ceil(dsub(l, sl))));
    *hi_n = min(t.Bx[a], int(floor(dadd(h, sh))));
}

// calls f(k) for every accepted shift k > 0 in the host's loop order; false if the point
// itself lies outside the extended domain
template <int D, class F>
__device__ __forceinline__ bool for_images(const Geo& g, const ImgTab& t, const double* x, F f) {
    constexpr int d = D;
    if (!in_domain<D>(g, t, x, 0)) return false;
    int nv[3] = {0, 0, 0};
    int l2 = 0, h2 = 0, l1 = 0, h1 = 0, l0 = 0, h0 = 0;
    if (d == 3) shift_range<D>(g, t, x, 2, nv, &l2, &h2);
    for (int v2 = l2; v2 <= h2; ++v2) {
        nv[2] = d == 3 ? v2 : 0;
        shift_range<D>(g, t, x, 1, nv, &l1, &h1);
        for (int v1 = l1; v1 <= h1; ++v1) {
            nv[1] = v1;
            shift_range<D>(g, t, x, 0, nv, &l0, &h0);
            for (int v0 = l0; v0 <= h0; ++v0) {
                nv[0] = v0;
                long long fl = 0;
                for (int a = d - 1; a >= 0; --a) fl = fl * t.dimx[a] + (nv[a] + t.Bx[a]);
                const int k = t.sidx[fl];
                if (k > 0 && in_domain<D>(g, t, x, k)) f(k);
            }
        }
    }
    return true;
}

// per point: the number of images, and the first kImgKeep shifts (in the host's order),
// which spare the write pass a second enumeration for points with at most kImgKeep images
// (in 3D a point near a corner of the extended domain has up to seven)
constexpr int kImgKeep = 8;
template <int D>
__global__ void k_image_count(Geo g, ImgTab t, int64_t n, const double* __restrict__ u, int* __restrict__ cnt,
                              int* __restrict__ kept, int* __restrict__ missing) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        double x[3];
        frac_to_tree<D>(g, u + j * D, x);
        int c = 0;
        int* kj = kept + j * kImgKeep;
        if (!for_images<D>(g, t, x, [&](int k) {
                if (c < kImgKeep) kj[c] = k;
                ++c;
            }))
            atomicOr(missing, 1);
        cnt[j] = c;
    }
}

template <int D>
__global__ void k_image_write(Geo g, ImgTab t, int64_t n, const double* __restrict__ u, const int* __restrict__ off,
                              const int* __restrict__ kept, int* __restrict__ pk, int* __restrict__ pj) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        int w = off[j];
        const int c = off[j + 1] - w;  // off holds n + 1 entries
        if (c == 0) continue;
        if (c <= kImgKeep) {  // the shifts the count pass kept
            for (int i = 0; i < c; ++i) {
                pk[w + i] = kept[j * kImgKeep + i];
                pj[w + i] = int(j);
            }
            continue;
        }
        double x[3];
        frac_to_tree<D>(g, u + j * D, x);
        for_images<D>(g, t, x, [&](int k) {
            pk[w] = k;
            pj[w] = int(j);
            ++w;
        });
    }
}

// ---------------------------------------------------------------------------------------
// keys

// Morton interleave of the per-axis cell bits, and the box key of the level-L cell c (in range)
// and its inverse; D, the dimension, is compile-time (the loops unroll, the arrays stay in
// registers)
template <int D>
__device__ __forceinline__ unsigned long long morton_d(const long long* w, int levels) {
    unsigned long long m = 0;
    for (int b = 0; b < levels; ++b)
#pragma unroll
        for (int a = 0; a < D; ++a) m |= (unsigned long long)((w[a] >> b) & 1) << (D * b + a);
    return m;
}
template <int D>
__device__ __forceinline__ unsigned long long box_key_d(const Geo& g, int L, const long long* c) {
    long long root = 0, w[3] = {0, 0, 0};
#pragma unroll
    for (int a = D - 1; a >= 0; --a) root = root * g.nroot[a] + (c[a] >> L);
#pragma unroll
    for (int a = 0; a < D; ++a) w[a] = c[a] & ((1LL << L) - 1);
    return ((unsigned long long)root << (D * L)) | morton_d<D>(w, L);
}
template <int D>
__device__ __forceinline__ void box_cell_d(const Geo& g, int L, unsigned long long key, long long* c) {
    long long root = (long long)(key >> (D * L));
    long long w[3] = {0, 0, 0};
    const unsigned long long m = key & ((1ULL << (D * L)) - 1);
    for (int b = 0; b < L; ++b)
#pragma unroll
        for (int a = 0; a < D; ++a) w[a] |= (long long)((m >> (D * b + a)) & 1) << b;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const long long rc = root % g.nroot[a];
        root /= g.nroot[a];
        c[a] = (rc << L) | w[a];
    }
}

// positions of the copies in image order, and their keys
template <int D>
__global__ void k_image_pos(Geo g, ImgTab t, int64_t n, int64_t nimg, int K, const double* __restrict__ u,
                            const int* __restrict__ pk, const int* __restrict__ pj, double* __restrict__ pos,
                            unsigned long long* __restrict__ key, int* __restrict__ val) {
    constexpr int d = D;
    const double scale = ldexp(1.0, K);
    for (int64_t im = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; im < nimg; im += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = im < n ? im : pj[im - n];
        const int k = im < n ? 0 : pk[im - n];
        double x[3];
        frac_to_tree<D>(g, u + j * d, x);
        long long root = 0, w[3] = {0, 0, 0};
        long long rcell[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            const double p = dadd(x[a], t.trs[k * 3 + a]);
            pos[im * d + a] = p;
            const double tsc = dmul(dsub(p, g.lo[a]), g.inv_rc);
            long long ci = (long long)floor(tsc);
            ci = min(max(ci, 0LL), (long long)g.nroot[a] - 1);
            rcell[a] = ci;
            long long cK = (long long)floor(dmul(tsc, scale));
            cK = min(max(cK, 0LL), ((long long)g.nroot[a] << K) - 1);
            w[a] = cK & ((1LL << K) - 1);
        }
        for (int a = d - 1; a >= 0; --a) root = root * g.nroot[a] + rcell[a];
        key[im] = ((unsigned long long)root << (d * K)) | morton_d<D>(w, K);
        val[im] = int(im);
    }
}

__device__ __forceinline__ int64_t lower_bound_u64(const unsigned long long* a, int64_t lo, int64_t hi,
                                                   unsigned long long v) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// level-L runs of more than n_s keys (refinement, Algorithm 1 step 2)
__global__ void k_runs(int64_t nimg, const unsigned long long* __restrict__ key, int shift, int n_s,
                       unsigned long long* __restrict__ pref_out, unsigned char* __restrict__ flag) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nimg; i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long p = key[i] >> shift;
        unsigned char f = 0;
        if (i == 0 || (key[i - 1] >> shift) != p) {
            const int64_t e = lower_bound_u64(key, i, nimg, (p + 1) << shift);
            f = (e - i) > n_s;
        }
        pref_out[i] = p;
        flag[i] = f;
    }
}

// the parent's colleagues of every non-leaf box of level L (keys at level L - 1; invalid:
// all ones)
template <int D>
__global__ void k_restrict_cands(Geo g, int L, const unsigned long long* __restrict__ nl, int64_t cnt,
                                 unsigned long long* __restrict__ out) {
    constexpr int d = D;
    constexpr int nn = D == 3 ? 27 : 9;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long P = nl[i] >> d;
        long long c[3];
        box_cell_d<D>(g, L - 1, P, c);
        for (int o = 0; o < nn; ++o) {
            long long c2[3] = {0, 0, 0};
            int r = o;
            bool ok = true;
            for (int a = 0; a < d; ++a) {
                c2[a] = c[a] + (r % 3) - 1;
                r /= 3;
                const long long dim = (long long)g.nroot[a] << (L - 1);
                if (g.periodic) c2[a] = (c2[a] + dim) % dim;
                ok &= (c2[a] >= 0 && c2[a] < dim);
            }
            out[i * nn + o] = ok ? box_key_d<D>(g, L - 1, c2) : ~0ULL;
        }
    }
}

__global__ void k_iota_u64(unsigned long long* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a[i] = (unsigned long long)i;
}
__global__ void k_iota_int(int* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a[i] = int(i);
}
__global__ void k_expand(const unsigned long long* __restrict__ nl, int64_t cnt, int d,
                         unsigned long long* __restrict__ out) {
    const int nc = 1 << d;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cnt * nc; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = (nl[i / nc] << d) | (unsigned long long)(i % nc);
}

struct BoxOut {
    int* level;
    long long* coord;
    int* parent;
    int* child0;
    long long* src_b;
    long long* src_e;
    double* center;
    int* colleague;
};

template <int D>
__global__ void k_boxes(Geo g, int L, int K, const unsigned long long* __restrict__ keys, int64_t nL, int baseL,
                        const unsigned long long* __restrict__ keysUp, int64_t nUp, int baseUp,
                        const unsigned long long* __restrict__ nlUp, const unsigned long long* __restrict__ nlL,
                        int64_t nnlL, int baseDown, const unsigned long long* __restrict__ skey, int64_t nimg,
                        BoxOut o) {
    constexpr int d = D;
    constexpr int nn = D == 3 ? 27 : 9;
    const double h = ddiv(g.rc, double(1LL << L));
    const int shift = d * (K - L);
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nL; i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long key = keys[i];
        const int64_t b = baseL + i;
        long long c[3] = {0, 0, 0};
        box_cell_d<D>(g, L, key, c);
        o.level[b] = L;
        for (int a = 0; a < d; ++a) {
            o.coord[b * d + a] = c[a];
            o.center[b * d + a] = dadd(g.lo[a], dmul(dadd(double(c[a]), 0.5), h));
        }
        if (L == 0) {
            o.parent[b] = -1;
        } else {
            const unsigned long long pk = nlUp[i >> d];
            o.parent[b] = baseUp + int(lower_bound_u64(keysUp, 0, nUp, pk));
        }
        const int64_t ci = lower_bound_u64(nlL, 0, nnlL, key);
        o.child0[b] = (ci < nnlL && nlL[ci] == key) ? int(baseDown + ci * (1 << d)) : -1;
        o.src_b[b] = lower_bound_u64(skey, 0, nimg, key << shift);
        o.src_e[b] = lower_bound_u64(skey, 0, nimg, (key + 1) << shift);
        for (int oo = 0; oo < nn; ++oo) {
            long long c2[3] = {0, 0, 0};
            int r = oo;
            bool ok = true;
            for (int a = 0; a < d; ++a) {
                c2[a] = c[a] + (r % 3) - 1;
                r /= 3;
                const long long dim = (long long)g.nroot[a] << L;
                if (g.periodic) c2[a] = (c2[a] + dim) % dim;
                ok &= (c2[a] >= 0 && c2[a] < dim);
            }
            int X = -1;
            if (ok) {
                const unsigned long long k2 = box_key_d<D>(g, L, c2);
                const int64_t x = lower_bound_u64(keys, 0, nL, k2);
                if (x < nL && keys[x] == k2) X = baseL + int(x);
            }
            o.colleague[b * nn + oo] = X;
        }
    }
}

// leaf of every key-sorted copy, and its leaf's first position per image
__global__ void k_leaf_descent(int d, int K, int64_t nimg, const unsigned long long* __restrict__ skey,
                               const int* __restrict__ sval, const int* __restrict__ child0,
                               const long long* __restrict__ src_b, int* __restrict__ leaf_pos,
                               int* __restrict__ lkey_img) {
    const unsigned long long mask = (1ULL << d) - 1;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nimg; i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long key = skey[i];
        int b = int(key >> (d * K));
        int L = 0;
        while (child0[b] >= 0) {
            ++L;
            b = child0[b] + int((key >> (d * (K - L))) & mask);
        }
        leaf_pos[i] = b;
        lkey_img[sval[i]] = int(src_b[b]);
    }
}

__global__ void k_sorted(int d, int64_t n, int64_t nimg, const int* __restrict__ simg, const int* __restrict__ pj,
                         const double* __restrict__ pos_img, int* __restrict__ orig, double* __restrict__ pos,
                         int* __restrict__ is_tgt) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < nimg; j += int64_t(gridDim.x) * blockDim.x) {
        const int64_t im = simg[j];
        orig[j] = im < n ? int(im) : pj[im - n];
        for (int a = 0; a < d; ++a) pos[j * d + a] = pos_img[im * d + a];
        is_tgt[j] = im < n ? 1 : 0;
    }
}

__global__ void k_targets_of(int64_t nimg, const int* __restrict__ is_tgt, const int* __restrict__ tpos,
                             const int* __restrict__ orig, int* __restrict__ tgt_of, int* __restrict__ tgt_orig) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < nimg; j += int64_t(gridDim.x) * blockDim.x)
        if (is_tgt[j]) {
            tgt_of[tpos[j]] = int(j);
            tgt_orig[tpos[j]] = orig[j];
        }
}

__global__ void k_box_tgt(int64_t nb, const long long* __restrict__ sb, const long long* __restrict__ se,
                          const int* __restrict__ tpos, long long* __restrict__ tb, long long* __restrict__ te) {
    for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nb; b += int64_t(gridDim.x) * blockDim.x) {
        tb[b] = tpos[sb[b]];
        te[b] = tpos[se[b]];
    }
}

// ---------------------------------------------------------------------------------------
// records (the host build's per-point passes)

template <typename T>
__device__ __forceinline__ void put_rec(void* buf, int64_t idx, double v) {
    static_cast<T*>(buf)[idx] = T(v);
}

template <int d>
__device__ __forceinline__ void mat_vec(const double* M, const double* v, double* out, bool transpose) {
#pragma unroll
    for (int i = 0; i < d; ++i) {
        double s = 0;
#pragma unroll
        for (int k = 0; k < d; ++k) s = dadd(s, dmul(transpose ? M[k * d + i] : M[i * d + k], v[k]));
        out[i] = s;
    }
}

// leaf-relative position of sorted source j, in the tree frame, and the caller-frame lattice
// vector of its copy (zero for the point itself)
template <int D>
__device__ __forceinline__ void relative_of(const RecordArgs& a, int64_t j, double* rel, double* disp) {
    constexpr int d = D;
    const int b = a.leaf[j];
    const int64_t o = a.orig[j];
    double yo[3] = {0, 0, 0}, xo[3], m[3], Dv[3], E[3], du[3];
    for (int k = 0; k < d; ++k) yo[k] = a.y[o * d + k];
    mat_vec<d>(a.Q, yo, xo, false);
    bool shifted = false;
    for (int i = 0; i < d; ++i) {
        double f = 0;
        for (int k = 0; k < d; ++k) f = dadd(f, dmul(a.Rinv[i * d + k], dsub(a.pos[j * d + k], xo[k])));
        m[i] = nearbyint(f);
        shifted |= m[i] != 0.0;
    }
    for (int k = 0; k < d; ++k) disp[k] = 0.0;
    if (shifted) {
        double Rm[3];
        for (int i = 0; i < d; ++i) {
            double s = 0;
            for (int k = 0; k < d; ++k) s = dadd(s, dmul(a.R[i * d + k], m[k]));
            Rm[i] = s;
            Dv[i] = dsub(a.center[int64_t(b) * d + i], s);
        }
        mat_vec<d>(a.Q, Dv, E, true);
        mat_vec<d>(a.Q, Rm, disp, true);
    } else {
        for (int i = 0; i < d; ++i) E[i] = a.Cu[int64_t(b) * d + i];
    }
    for (int k = 0; k < d; ++k) du[k] = dsub(yo[k], E[k]);
    mat_vec<d>(a.Q, du, rel, false);
}

template <typename T, int D>
__global__ void k_src_records(RecordArgs a) {
    constexpr int d = D;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < a.nimg; j += int64_t(gridDim.x) * blockDim.x) {
        double rel[3], disp[3];
        relative_of<D>(a, j, rel, disp);
        for (int k = 0; k < d; ++k) {
            put_rec<T>(a.src4, j * 4 + k, rel[k]);
            if (a.mixed) a.src_lo[j * 4 + k] = float(rel[k] - double(float(rel[k])));
            a.src_disp[j * d + k] = disp[k];
        }
        a.src_orig[j] = a.orig[j];
    }
}

template <typename T, int D>
__global__ void k_tgt_records(RecordArgs a) {
    constexpr int d = D;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < a.ntgt; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = a.tgt_of[t];
        const int b = a.leaf[j];
        double rel[3], disp[3];
        relative_of<D>(a, j, rel, disp);
        a.tgt_leaf[t] = b;
        for (int k = 0; k < d; ++k) {
            put_rec<T>(a.tgt4, t * 4 + k, rel[k]);
            if (a.mixed) a.tgt_lo[t * 4 + k] = float(rel[k] - double(float(rel[k])));
        }
        a.tgt_orig_out[t] = a.tgt_orig[t];
        a.self_w[t] = a.self_w_level[a.box_level[b]];
    }
}

__global__ void k_box_cu(int nb, int d, Geo g, const double* __restrict__ center, double* __restrict__ Cu) {
    for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nb; b += int64_t(gridDim.x) * blockDim.x)
        if (d == 3) mat_vec<3>(g.Q, center + b * 3, Cu + b * 3, true);
        else mat_vec<2>(g.Q, center + b * 2, Cu + b * 2, true);
}

// ---------------------------------------------------------------------------------------
// far-field layout (window starts in FP64, as the host build)

__device__ __forceinline__ void grid_coord(double uu, int M, int w, int* g0, double* del) {
    const double Mu = dmul(double(M), uu);
    int gg = int(ceil(dsub(Mu, 0.5 * w)));
    *del = dsub(Mu, double(gg));
    const int fw = w / 2;
    const int key = gg + fw;
    const int wrap = key >= 0 ? key / M : -((-key + M - 1) / M);
    gg -= wrap * M;
    *g0 = gg;
}

__global__ void k_far_bins(FarLayoutArgs a, int* __restrict__ bin, int4* __restrict__ g0o,
                           double* __restrict__ del3, int* __restrict__ vals, int* __restrict__ bin_count) {
    const int fw = a.w / 2;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < a.n; j += int64_t(gridDim.x) * blockDim.x) {
        int64_t bb = 0;
        int off[3] = {0, 0, 0};
        double dl[3] = {0, 0, 0};
        for (int i = a.d - 1; i >= 0; --i) {
            int g0;
            double del;
            grid_coord(a.u[j * a.d + i], a.M[i], a.w, &g0, &del);
            const int key = g0 + fw;
            const int bi = key / a.B[i];
            off[i] = key - bi * a.B[i];
            dl[i] = del;
            bb = bb * a.nbin[i] + bi;
        }
        bin[j] = int(bb);
        g0o[j] = make_int4(off[0], off[1], off[2], 0);
        for (int i = 0; i < 3; ++i) del3[j * 3 + i] = dl[i];
        vals[j] = int(j);
        atomicAdd(&bin_count[bb], 1);
    }
}

template <typename T>
__global__ void k_far_points(FarLayoutArgs a, const int* __restrict__ order, const int4* __restrict__ g0o,
                             const double* __restrict__ del3) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < a.n; k += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = order[k];
        a.pt_g0[k] = g0o[j];
        for (int i = 0; i < 3; ++i) put_rec<T>(a.pt_dq, k * 4 + i, del3[j * 3 + i]);
        put_rec<T>(a.pt_dq, k * 4 + 3, 0.0);
        a.sp_orig[k] = int(j);
    }
}

template <typename T>
__global__ void k_far_targets(FarLayoutArgs a) {
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < a.ntgt; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = a.tgt_orig[t];
        int gg[3] = {0, 0, 0};
        double dl[4] = {0, 0, 0, 0};
        for (int i = 0; i < a.d; ++i) grid_coord(a.u[j * a.d + i], a.M[i], a.w, &gg[i], &dl[i]);
        for (int i = 0; i < 4; ++i) put_rec<T>(a.t_dq, t * 4 + i, dl[i]);
        for (int i = 0; i < a.d; ++i) gg[i] = ((gg[i] % a.M[i]) + a.M[i]) % a.M[i];
        a.t_g0[t] = make_int4(gg[0], gg[1], gg[2], 0);
    }
}

// ---------------------------------------------------------------------------------------
// near-field entries

template <typename T>
__global__ void k_entries(EntryArgs a) {
    const int d = a.d;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < a.nlist; e += int64_t(gridDim.x) * blockDim.x) {
        // target leaf k of entry e: the last k with list_begin[k] <= e
        int lo = 0, hi = a.ntleaf;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.list_begin[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int tb = a.tleaf[lo];
        const int sb = a.list[e];
        a.ent[e] = make_int2(a.bsb[sb], a.bsc[sb]);
        const double* Ln = a.Ln + a.shift[e] * 3;
        double du[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) du[k] = dsub(dadd(a.Cu[int64_t(sb) * d + k], Ln[k]), a.Cu[int64_t(tb) * d + k]);
        for (int i = 0; i < d; ++i) {
            double sh = 0;
            for (int k = 0; k < d; ++k) sh = dadd(sh, dmul(a.Q[i * d + k], du[k]));
            put_rec<T>(a.ent_sh, e * 4 + i, sh);
            if (a.mixed) a.ent_shlo[e * 4 + i] = float(sh - double(float(sh)));
        }
    }
}

// ---------------------------------------------------------------------------------------
// host helpers

// temporary buffers of one call: from the plan's pool when there is one (the caller returns
// them once the stream has drained), else cudaMalloc'd and freed on return
struct Scratch {
    DevicePool* pool = nullptr;
    std::vector<std::pair<void*, size_t>>* keep = nullptr;
    std::vector<void*> ptrs;
    Scratch(DevicePool* p, std::vector<std::pair<void*, size_t>>* k) : pool(p && k ? p : nullptr), keep(k) {}
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class X>
    X* get(size_t count) {
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(X);
        void* p = nullptr;
        if (pool) {
            p = pool->get(bytes);
            if (!p) return nullptr;
            keep->push_back({p, bytes});
            return static_cast<X*>(p);
        }
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<X*>(p);
    }
};

int bits_for(uint64_t v) {  // bits to hold values < v
    int b = 0;
    while (b < 64 && (uint64_t(1) << b) < v) ++b;
    return b;
}

#define GB_CK(call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) {                                 \
            if (msg) *msg = cudaGetErrorString(e_);              \
            return PDMK_ERR_CUDA;                                \
        }                                                        \
    } while (0)
#define GB_ALLOC(ptr, X, count)                                  \
    do {                                                         \
        ptr = scr.get<X>(count);                                 \
        if (!ptr) {                                              \
            if (msg) *msg = "device allocation failed (set-up)"; \
            return PDMK_ERR_CUDA;                                \
        }                                                        \
    } while (0)

template <class X>
int own(GpuBuild* b, X** out, size_t count, std::string* msg) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(X);
    void* p = nullptr;
    if (b->pool) {
        p = b->pool->get(bytes);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) {
        if (msg) *msg = "device allocation failed (set-up)";
        return PDMK_ERR_CUDA;
    }
    b->allocs.push_back({p, bytes});
    *out = static_cast<X*>(p);
    return PDMK_OK;
}

}  // namespace

void gpu_build_free(GpuBuild* b) {
    for (auto& a : b->allocs) {
        if (b->pool)
            b->pool->put(a.first, a.second);
        else
            cudaFree(a.first);
    }
    b->allocs.clear();
    b->nb = 0;
    b->d_level = b->d_parent = b->d_child0 = b->d_colleague = nullptr;
    b->d_center = nullptr;
    b->d_coord = b->d_src_b = b->d_src_e = b->d_tgt_b = b->d_tgt_e = nullptr;
    b->d_u = nullptr;
    b->d_orig = nullptr;
    b->d_pos = nullptr;
    b->d_leaf = nullptr;
    b->d_tgt_of = nullptr;
    b->d_tgt_orig = nullptr;
}

void gpu_orient(const Geometry& g, int64_t n, const double* y, double* u, cudaStream_t s) {
    if (n > 0) k_orient<<<blocks_for(n), kThreads, 0, s>>>(make_geo(g), n, y, u);
}

void gpu_check_inputs(int64_t n, int d, const double* y, const double* q, int* d_nonfinite, double* d_part, int nblk,
                      cudaStream_t s) {
    k_check<<<nblk, kThreads, 0, s>>>(n, d, y, q, d_nonfinite, d_part);
}

int gpu_build_tree(const Geometry& g, int64_t n, int n_s, int max_depth, cudaStream_t s, GpuBuild* bo, Tree* t,
                   BuildStats* st, std::string* msg) {
    const int d = g.d;
    const Geo geo = make_geo(g);
    Scratch scr(bo->pool, bo->scratch);
    // host wall clock of the phases (kDeviceBuildPhases), the stream drained at each boundary
    auto clk = std::chrono::steady_clock::now();
    auto lap = [&](int k) -> int {
        if (cudaStreamSynchronize(s) != cudaSuccess) return PDMK_ERR_CUDA;
        const auto now = std::chrono::steady_clock::now();
        if (st) st->phase_ms[k] = std::chrono::duration<double, std::milli>(now - clk).count();
        clk = now;
        return PDMK_OK;
    };
    // ---- images ----
    ImageShifts tab;
    image_shifts(g, &tab);
    ImgTab it;
    it.ns = tab.ns;
    for (int a = 0; a < 3; ++a) {
        it.Bx[a] = tab.Bx[a];
        it.dimx[a] = tab.dimx[a];
    }
    int* d_sidx;
    double* d_trs;
    GB_ALLOC(d_sidx, int, tab.sidx.size());
    GB_ALLOC(d_trs, double, tab.trs.size());
    GB_CK(cudaMemcpyAsync(d_sidx, tab.sidx.data(), tab.sidx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    GB_CK(cudaMemcpyAsync(d_trs, tab.trs.data(), tab.trs.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    it.sidx = d_sidx;
    it.trs = d_trs;
    int *d_cnt, *d_off, *d_flag;
    int* d_kept;
    GB_ALLOC(d_cnt, int, n + 1);
    GB_ALLOC(d_kept, int, size_t(n) * kImgKeep);
    GB_ALLOC(d_off, int, n + 1);
    GB_ALLOC(d_flag, int, 1);
    GB_CK(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
    GB_CK(cudaMemsetAsync(d_cnt + n, 0, sizeof(int), s));
    if (d == 3) k_image_count<3><<<blocks_for(n), kThreads, 0, s>>>(geo, it, n, bo->d_u, d_cnt, d_kept, d_flag);
    else k_image_count<2><<<blocks_for(n), kThreads, 0, s>>>(geo, it, n, bo->d_u, d_cnt, d_kept, d_flag);
    size_t tb = 0;
    GB_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, d_cnt, d_off, int(n + 1), s));
    void* d_tmp = nullptr;
    size_t tmp_bytes = 0;
    auto tmp = [&](size_t need) -> void* {
        if (need > tmp_bytes) {
            d_tmp = scr.get<unsigned char>(need);
            tmp_bytes = d_tmp ? need : 0;
        }
        return d_tmp;
    };
    if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceScan::ExclusiveSum(d_tmp, tb, d_cnt, d_off, int(n + 1), s));
    int h_flag = 0, h_nextra = 0;
    GB_CK(cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemcpyAsync(&h_nextra, d_off + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaStreamSynchronize(s));
    if (h_flag) {
        if (msg) *msg = "a point lies outside the extended domain";
        return PDMK_ERR_INTERNAL;
    }
    const int64_t nx = h_nextra;
    const int64_t nimg = n + nx;
    if (nimg >= (int64_t(1) << 30)) return kGpuBuildUnsupported;
    int *d_pk, *d_pj, *d_pk2, *d_pj2;
    GB_ALLOC(d_pk, int, nx);
    GB_ALLOC(d_pj, int, nx);
    GB_ALLOC(d_pk2, int, nx);
    GB_ALLOC(d_pj2, int, nx);
    if (nx > 0) {
        if (d == 3) k_image_write<3><<<blocks_for(n), kThreads, 0, s>>>(geo, it, n, bo->d_u, d_off, d_kept, d_pk, d_pj);
        else k_image_write<2><<<blocks_for(n), kThreads, 0, s>>>(geo, it, n, bo->d_u, d_off, d_kept, d_pk, d_pj);
        const int kb = std::max(1, bits_for(uint64_t(tab.ns)));
        GB_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, d_pk, d_pk2, d_pj, d_pj2, int(nx), 0, kb, s));
        if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
        GB_CK(cub::DeviceRadixSort::SortPairs(d_tmp, tb, d_pk, d_pk2, d_pj, d_pj2, int(nx), 0, kb, s));
    }
    if (lap(0)) return PDMK_ERR_CUDA;
    // ---- keys ----
    int64_t nroot_tot = 1;
    for (int a = 0; a < d; ++a) nroot_tot *= g.nroot[a];
    const int rbits = bits_for(uint64_t(nroot_tot));
    const int K = std::min((63 - rbits) / d, 30);
    if (K < 1) return kGpuBuildUnsupported;
    double* d_posimg;
    unsigned long long *d_key, *d_key2;
    int *d_val, *d_val2;
    GB_ALLOC(d_posimg, double, size_t(nimg) * d);
    GB_ALLOC(d_key, unsigned long long, nimg);
    GB_ALLOC(d_key2, unsigned long long, nimg);
    GB_ALLOC(d_val, int, nimg);
    GB_ALLOC(d_val2, int, nimg);
    if (d == 3)
        k_image_pos<3><<<blocks_for(nimg), kThreads, 0, s>>>(geo, it, n, nimg, K, bo->d_u, d_pk2, d_pj2, d_posimg, d_key,
                                                      d_val);
    else
        k_image_pos<2><<<blocks_for(nimg), kThreads, 0, s>>>(geo, it, n, nimg, K, bo->d_u, d_pk2, d_pj2, d_posimg, d_key,
                                                      d_val);
    const int keybits = rbits + d * K;
    GB_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, d_key, d_key2, d_val, d_val2, int(nimg), 0, keybits, s));
    if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceRadixSort::SortPairs(d_tmp, tb, d_key, d_key2, d_val, d_val2, int(nimg), 0, keybits, s));
    const unsigned long long* skey = d_key2;
    const int* sval = d_val2;
    if (lap(1)) return PDMK_ERR_CUDA;
    // ---- refinement: non-leaf boxes per level ----
    std::vector<unsigned long long*> nl;  // device arrays per level
    std::vector<int64_t> nnl;
    unsigned long long* d_pref;
    unsigned char* d_rflag;
    int64_t* d_nsel;
    GB_ALLOC(d_pref, unsigned long long, nimg);
    GB_ALLOC(d_rflag, unsigned char, nimg);
    GB_ALLOC(d_nsel, int64_t, 1);
    for (int L = 0;; ++L) {
        if (L >= max_depth) break;
        if (L > K) return kGpuBuildUnsupported;
        k_runs<<<blocks_for(nimg), kThreads, 0, s>>>(nimg, skey, d * (K - L), n_s, d_pref, d_rflag);
        unsigned long long* out;
        GB_ALLOC(out, unsigned long long, nimg);
        GB_CK(cub::DeviceSelect::Flagged(nullptr, tb, d_pref, d_rflag, out, d_nsel, nimg, s));
        if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
        GB_CK(cub::DeviceSelect::Flagged(d_tmp, tb, d_pref, d_rflag, out, d_nsel, nimg, s));
        int64_t h_n = 0;
        GB_CK(cudaMemcpyAsync(&h_n, d_nsel, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GB_CK(cudaStreamSynchronize(s));
        if (h_n == 0) break;
        if (L == K) return kGpuBuildUnsupported;  // a box of the deepest key level would split
        nl.push_back(out);
        nnl.push_back(h_n);
    }
    if (lap(2)) return PDMK_ERR_CUDA;
    // ---- level restriction, deepest level first ----
    int nn = 1;
    for (int a = 0; a < d; ++a) nn *= 3;
    for (int L = int(nl.size()) - 1; L >= 1; --L) {
        const int64_t nc = nnl[L] * nn, tot = nnl[L - 1] + nc;
        unsigned long long *cat, *cat2, *uq;
        GB_ALLOC(cat, unsigned long long, tot);
        GB_ALLOC(cat2, unsigned long long, tot);
        GB_ALLOC(uq, unsigned long long, tot);
        GB_CK(cudaMemcpyAsync(cat, nl[L - 1], nnl[L - 1] * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
        (d == 3 ? k_restrict_cands<3> : k_restrict_cands<2>)<<<blocks_for(nnl[L]), kThreads, 0, s>>>(
            geo, L, nl[L], nnl[L], cat + nnl[L - 1]);
        GB_CK(cub::DeviceRadixSort::SortKeys(nullptr, tb, cat, cat2, int(tot), 0, 64, s));
        if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
        GB_CK(cub::DeviceRadixSort::SortKeys(d_tmp, tb, cat, cat2, int(tot), 0, 64, s));
        GB_CK(cub::DeviceSelect::Unique(nullptr, tb, cat2, uq, d_nsel, tot, s));
        if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
        GB_CK(cub::DeviceSelect::Unique(d_tmp, tb, cat2, uq, d_nsel, tot, s));
        int64_t h_n = 0;
        unsigned long long last = 0;
        GB_CK(cudaMemcpyAsync(&h_n, d_nsel, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GB_CK(cudaStreamSynchronize(s));
        GB_CK(cudaMemcpy(&last, uq + (h_n - 1), sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        if (last == ~0ULL) --h_n;
        nl[L - 1] = uq;
        nnl[L - 1] = h_n;
    }
    if (lap(3)) return PDMK_ERR_CUDA;
    // ---- boxes per level ----
    const int nlev = int(nl.size()) + 1;
    std::vector<unsigned long long*> lk(nlev);
    std::vector<int64_t> nlk(nlev);
    GB_ALLOC(lk[0], unsigned long long, nroot_tot);
    nlk[0] = nroot_tot;
    k_iota_u64<<<blocks_for(nroot_tot), kThreads, 0, s>>>(lk[0], nroot_tot);
    for (int L = 1; L < nlev; ++L) {
        nlk[L] = nnl[L - 1] << d;
        GB_ALLOC(lk[L], unsigned long long, nlk[L]);
        k_expand<<<blocks_for(nlk[L]), kThreads, 0, s>>>(nl[L - 1], nnl[L - 1], d, lk[L]);
    }
    std::vector<int> lstart(nlev + 1, 0);
    for (int L = 0; L < nlev; ++L) {
        if (int64_t(lstart[L]) + nlk[L] >= (int64_t(1) << 31)) return kGpuBuildUnsupported;
        lstart[L + 1] = lstart[L] + int(nlk[L]);
    }
    const int nb = lstart[nlev];
    BoxOut bx;
    // the box arrays the near-field lists read stay on the device (freed by gpu_build_free)
    {
        int r0;
        if ((r0 = own(bo, &bx.level, nb, msg))) return r0;
        if ((r0 = own(bo, &bx.coord, size_t(nb) * d, msg))) return r0;
        if ((r0 = own(bo, &bx.parent, nb, msg))) return r0;
        if ((r0 = own(bo, &bx.child0, nb, msg))) return r0;
        if ((r0 = own(bo, &bx.src_b, nb, msg))) return r0;
        if ((r0 = own(bo, &bx.src_e, nb, msg))) return r0;
        if ((r0 = own(bo, &bx.colleague, size_t(nb) * nn, msg))) return r0;
        if ((r0 = own(bo, &bx.center, size_t(nb) * d, msg))) return r0;
    }
    for (int L = 0; L < nlev; ++L) {
        const bool has_down = L < int(nl.size());
        (d == 3 ? k_boxes<3> : k_boxes<2>)<<<blocks_for(nlk[L]), kThreads, 0, s>>>(
            geo, L, K, lk[L], nlk[L], lstart[L], L > 0 ? lk[L - 1] : nullptr, L > 0 ? nlk[L - 1] : 0,
            L > 0 ? lstart[L - 1] : 0, L > 0 ? nl[L - 1] : nullptr, has_down ? nl[L] : nullptr,
            has_down ? nnl[L] : 0, L + 1 <= nlev ? lstart[std::min(L + 1, nlev)] : 0, skey, nimg, bx);
    }
    // ---- final order: by leaf, then by image index ----
    int *d_leafpos, *d_lkey, *d_lkey2, *d_iota, *d_simg;
    GB_ALLOC(d_leafpos, int, nimg);
    GB_ALLOC(d_lkey, int, nimg);
    GB_ALLOC(d_lkey2, int, nimg);
    GB_ALLOC(d_iota, int, nimg);
    GB_ALLOC(d_simg, int, nimg);
    k_leaf_descent<<<blocks_for(nimg), kThreads, 0, s>>>(d, K, nimg, skey, sval, bx.child0, bx.src_b, d_leafpos,
                                                         d_lkey);
    k_iota_int<<<blocks_for(nimg), kThreads, 0, s>>>(d_iota, nimg);
    const int lb = std::max(1, bits_for(uint64_t(nimg)));
    GB_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, d_lkey, d_lkey2, d_iota, d_simg, int(nimg), 0, lb, s));
    if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceRadixSort::SortPairs(d_tmp, tb, d_lkey, d_lkey2, d_iota, d_simg, int(nimg), 0, lb, s));
    // ---- sorted outputs ----
    int r;
    if ((r = own(bo, &bo->d_orig, nimg, msg))) return r;
    if ((r = own(bo, &bo->d_pos, size_t(nimg) * d, msg))) return r;
    if ((r = own(bo, &bo->d_tgt_of, n, msg))) return r;
    if ((r = own(bo, &bo->d_tgt_orig, n, msg))) return r;
    if ((r = own(bo, &bo->d_leaf, nimg, msg))) return r;
    int *d_istgt, *d_tpos;
    GB_ALLOC(d_istgt, int, nimg + 1);
    GB_ALLOC(d_tpos, int, nimg + 1);
    GB_CK(cudaMemsetAsync(d_istgt + nimg, 0, sizeof(int), s));
    k_sorted<<<blocks_for(nimg), kThreads, 0, s>>>(d, n, nimg, d_simg, d_pj2, d_posimg, bo->d_orig, bo->d_pos,
                                                   d_istgt);
    GB_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, d_istgt, d_tpos, int(nimg + 1), s));
    if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceScan::ExclusiveSum(d_tmp, tb, d_istgt, d_tpos, int(nimg + 1), s));
    k_targets_of<<<blocks_for(nimg), kThreads, 0, s>>>(nimg, d_istgt, d_tpos, bo->d_orig, bo->d_tgt_of,
                                                       bo->d_tgt_orig);
    long long *d_tb, *d_te;
    if ((r = own(bo, &d_tb, nb, msg))) return r;
    if ((r = own(bo, &d_te, nb, msg))) return r;
    k_box_tgt<<<blocks_for(nb), kThreads, 0, s>>>(nb, bx.src_b, bx.src_e, d_tpos, d_tb, d_te);
    // the key-sorted and the final order share every leaf's range
    GB_CK(cudaMemcpyAsync(bo->d_leaf, d_leafpos, size_t(nimg) * sizeof(int), cudaMemcpyDeviceToDevice, s));
    int h_ntgt = 0;
    GB_CK(cudaMemcpyAsync(&h_ntgt, d_tpos + nimg, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (lap(4)) return PDMK_ERR_CUDA;
    // ---- the host tree ----
    t->d = d;
    for (int a = 0; a < 3; ++a) t->nroot[a] = a < d ? g.nroot[a] : 1;
    t->periodic = g.periodic_root;
    t->nlevels = nlev;
    t->level_start = lstart;
    bo->nb = nb;
    bo->d_level = bx.level;
    bo->d_coord = bx.coord;
    bo->d_parent = bx.parent;
    bo->d_child0 = bx.child0;
    bo->d_src_b = bx.src_b;
    bo->d_src_e = bx.src_e;
    bo->d_tgt_b = d_tb;
    bo->d_tgt_e = d_te;
    bo->d_colleague = bx.colleague;
    bo->d_center = bx.center;
    if (bo->download_tree) {
        GB_CK(cudaStreamSynchronize(s));
        if ((r = gpu_tree_download(*bo, t, s, msg))) return r;
    }
    GB_CK(cudaStreamSynchronize(s));
    if (lap(5)) return PDMK_ERR_CUDA;
    bo->n = n;
    bo->nimg = nimg;
    bo->ntgt = h_ntgt;
    bo->key_levels = K;
    if (st) {
        st->n = n;
        st->n_images = nimg;
        st->nboxes = nb;
        // every non-leaf box has 2^d children, and every box below the root is a child
        st->nleaves = nb - (nb - lstart[1]) / (1 << d);
        st->depth = nlev - 1;
    }
    return PDMK_OK;
}

// the per-box arrays of the device tree into the host tree t (resized): through the page-locked
// staging buffer when it has one, its two halves taking alternate chunks so that the copy of
// one chunk into the host arrays (on the host's threads) overlaps the transfer of the next;
// else straight into the host arrays
int gpu_tree_download(const GpuBuild& b, Tree* t, cudaStream_t s, std::string* msg) {
    const int nb = b.nb, d = t->d, nn = d == 3 ? 27 : 9;
    const GpuBuild* bo = &b;
    struct BoxPtrs {
        int* level;
        long long* coord;
        int* parent;
        int* child0;
        long long* src_b;
        long long* src_e;
        double* center;
        int* colleague;
    } bx{b.d_level, b.d_coord, b.d_parent, b.d_child0, b.d_src_b, b.d_src_e, b.d_center, b.d_colleague};
    const long long* d_tb = b.d_tgt_b;
    const long long* d_te = b.d_tgt_e;
    t->level.resize(nb);
    t->coord.resize(size_t(nb) * d);
    t->parent.resize(nb);
    t->child0.resize(nb);
    t->src_begin.resize(nb);
    t->src_end.resize(nb);
    t->tgt_begin.resize(nb);
    t->tgt_end.resize(nb);
    t->center.resize(size_t(nb) * d);
    t->colleague.resize(size_t(nb) * nn);
    static_assert(sizeof(long long) == sizeof(int64_t), "64-bit box arrays");
    struct Piece {
        void* dst;
        const void* src;
        size_t bytes;
    };
    std::vector<Piece> pieces;
    auto download = [&](void* dst, const void* src, size_t bytes) { pieces.push_back({dst, src, bytes}); };
    download(t->level.data(), bx.level, size_t(nb) * sizeof(int));
    download(t->coord.data(), bx.coord, size_t(nb) * d * sizeof(int64_t));
    download(t->parent.data(), bx.parent, size_t(nb) * sizeof(int));
    download(t->child0.data(), bx.child0, size_t(nb) * sizeof(int));
    download(t->src_begin.data(), bx.src_b, size_t(nb) * sizeof(int64_t));
    download(t->src_end.data(), bx.src_e, size_t(nb) * sizeof(int64_t));
    download(t->tgt_begin.data(), d_tb, size_t(nb) * sizeof(int64_t));
    download(t->tgt_end.data(), d_te, size_t(nb) * sizeof(int64_t));
    download(t->center.data(), bx.center, size_t(nb) * d * sizeof(double));
    download(t->colleague.data(), bx.colleague, size_t(nb) * nn * sizeof(int));
    const size_t half = bo->stage_cap / 2;
    if (!bo->h_stage || half < (size_t(1) << 20)) {
        for (const Piece& pc : pieces)
            GB_CK(cudaMemcpyAsync(pc.dst, pc.src, pc.bytes, cudaMemcpyDeviceToHost, s));
    } else {
        struct Chunk {
            unsigned char* dst;
            const unsigned char* src;
            size_t len;
        };
        std::vector<Chunk> chunks;
        for (const Piece& pc : pieces)
            for (size_t off = 0; off < pc.bytes; off += half)
                chunks.push_back({static_cast<unsigned char*>(pc.dst) + off, static_cast<const unsigned char*>(pc.src) + off,
                                  std::min(half, pc.bytes - off)});
        cudaEvent_t ev[2];
        GB_CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        if (cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaEventDestroy(ev[0]);
            if (msg) *msg = "event creation failed (set-up)";
            return PDMK_ERR_CUDA;
        }
        auto drain = [&](size_t i) {  // chunk i from its half into the host array
            const unsigned char* from = bo->h_stage + (i & 1) * half;
            const size_t len = chunks[i].len;
            const int64_t npiece = int64_t((len + (size_t(1) << 20) - 1) >> 20);
#pragma omp parallel for schedule(static)
            for (int64_t k = 0; k < npiece; ++k) {
                const size_t o = size_t(k) << 20, l = std::min(size_t(1) << 20, len - o);
                std::memcpy(chunks[i].dst + o, from + o, l);
            }
        };
        int rc = PDMK_OK;
        for (size_t i = 0; i < chunks.size() && rc == PDMK_OK; ++i) {
            if (cudaMemcpyAsync(bo->h_stage + (i & 1) * half, chunks[i].src, chunks[i].len, cudaMemcpyDeviceToHost,
                                s) != cudaSuccess ||
                cudaEventRecord(ev[i & 1], s) != cudaSuccess) {
                rc = PDMK_ERR_CUDA;
                break;
            }
            if (i > 0) {
                if (cudaEventSynchronize(ev[(i - 1) & 1]) != cudaSuccess) {
                    rc = PDMK_ERR_CUDA;
                    break;
                }
                drain(i - 1);
            }
        }
        if (rc == PDMK_OK && !chunks.empty()) {
            if (cudaEventSynchronize(ev[(chunks.size() - 1) & 1]) != cudaSuccess) rc = PDMK_ERR_CUDA;
            else drain(chunks.size() - 1);
        }
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        if (rc != PDMK_OK) {
            if (msg) *msg = cudaGetErrorString(cudaGetLastError());
            return rc;
        }
    }
    GB_CK(cudaStreamSynchronize(s));
    return PDMK_OK;
}

void gpu_box_cu(int nb, int d, const double* Q, const double* center, double* Cu, cudaStream_t s) {
    Geo g;
    std::memset(&g, 0, sizeof(g));
    g.d = d;
    std::memcpy(g.Q, Q, sizeof(g.Q));
    if (nb > 0) k_box_cu<<<blocks_for(nb), kThreads, 0, s>>>(nb, d, g, center, Cu);
}

void gpu_records(const RecordArgs& a, cudaStream_t s) {
    if (a.nimg > 0) {
        const int nb = blocks_for(a.nimg);
        if (a.mixed) (a.d == 3 ? k_src_records<float, 3> : k_src_records<float, 2>)<<<nb, kThreads, 0, s>>>(a);
        else (a.d == 3 ? k_src_records<double, 3> : k_src_records<double, 2>)<<<nb, kThreads, 0, s>>>(a);
    }
    if (a.ntgt > 0) {
        const int nb = blocks_for(a.ntgt);
        if (a.mixed) (a.d == 3 ? k_tgt_records<float, 3> : k_tgt_records<float, 2>)<<<nb, kThreads, 0, s>>>(a);
        else (a.d == 3 ? k_tgt_records<double, 3> : k_tgt_records<double, 2>)<<<nb, kThreads, 0, s>>>(a);
    }
}

void gpu_near_entries(const EntryArgs& a, cudaStream_t s) {
    if (a.nlist <= 0) return;
    if (a.mixed) k_entries<float><<<blocks_for(a.nlist), kThreads, 0, s>>>(a);
    else k_entries<double><<<blocks_for(a.nlist), kThreads, 0, s>>>(a);
}

int gpu_far_layout(const FarLayoutArgs& a, cudaStream_t s, std::string* msg) {
    Scratch scr(a.pool, a.scratch);
    int *d_bin, *d_bin2, *d_vals, *d_order;
    int4* d_g0;
    double* d_del;
    GB_ALLOC(d_bin, int, a.n);
    GB_ALLOC(d_bin2, int, a.n);
    GB_ALLOC(d_vals, int, a.n);
    GB_ALLOC(d_order, int, a.n);
    GB_ALLOC(d_g0, int4, a.n);
    GB_ALLOC(d_del, double, size_t(a.n) * 3);
    GB_CK(cudaMemsetAsync(a.bin_count, 0, size_t(a.nbins_tot) * sizeof(int), s));
    if (a.n > 0) {
        k_far_bins<<<blocks_for(a.n), kThreads, 0, s>>>(a, d_bin, d_g0, d_del, d_vals, a.bin_count);
        size_t tb = 0;
        const int kb = std::max(1, bits_for(uint64_t(a.nbins_tot)));
        GB_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, d_bin, d_bin2, d_vals, d_order, int(a.n), 0, kb, s));
        void* d_tmp;
        GB_ALLOC(d_tmp, unsigned char, tb);
        GB_CK(cub::DeviceRadixSort::SortPairs(d_tmp, tb, d_bin, d_bin2, d_vals, d_order, int(a.n), 0, kb, s));
        if (a.mixed) k_far_points<float><<<blocks_for(a.n), kThreads, 0, s>>>(a, d_order, d_g0, d_del);
        else k_far_points<double><<<blocks_for(a.n), kThreads, 0, s>>>(a, d_order, d_g0, d_del);
    }
    if (a.ntgt > 0) {
        if (a.mixed) k_far_targets<float><<<blocks_for(a.ntgt), kThreads, 0, s>>>(a);
        else k_far_targets<double><<<blocks_for(a.ntgt), kThreads, 0, s>>>(a);
    }
    GB_CK(cudaGetLastError());
    GB_CK(cudaStreamSynchronize(s));  // the scratch is freed on return
    return PDMK_OK;
}


// ------------------------------------------------------------------ near-field lists
namespace {

constexpr int kMaxNear = 27 * 8 + 27;  // children of 27 colleagues, or 27 coarser leaves

struct BoxView {
    int d, nn;
    const int* level;
    const long long* coord;
    const int* parent;
    const int* child0;
    const long long* src_b;
    const long long* src_e;
    const int* colleague;
};

// the shift code of the lattice vector that brings the level-L cell c into the root grid
// (periodic roots; c is wrapped), 13 otherwise (as the host tree's wrap)
__device__ int wrap_code(const Geo& g, int d, int L, long long* c) {
    if (!g.periodic) return 13;
    int code = 0, mul = 1;
    for (int a = 0; a < d; ++a) {
        const long long dim = static_cast<long long>(g.nroot[a]) << L;
        int n = 0;
        while (c[a] < 0) { c[a] += dim; --n; }
        while (c[a] >= dim) { c[a] -= dim; ++n; }
        code += (n + 1) * mul;
        mul *= 3;
    }
    for (int a = d; a < 3; ++a) {
        code += mul;
        mul *= 3;
    }
    return code;
}

// the sorted, unique (source leaf, shift code) pairs of target leaf b; -1 when the list
// outgrows kMaxNear or a colleague's child is refined (neither happens under the level
// restriction; the host build then serves the inputs)
__device__ int near_list_of(const BoxView& v, const Geo& g, int b, int2* lst) {
    const int d = v.d, nn = v.nn, L = v.level[b];
    int n = 0;
    for (int o = 0; o < nn; ++o) {
        long long c[3] = {0, 0, 0};
        int r = o;
        for (int a = 0; a < d; ++a) {
            c[a] = v.coord[size_t(b) * d + a] + (r % 3) - 1;
            r /= 3;
        }
        const int code = wrap_code(g, d, L, c);
        const int X = v.colleague[size_t(b) * nn + o];
        if (X >= 0) {
            if (v.child0[X] < 0) {
                if (v.src_e[X] > v.src_b[X]) {
                    if (n >= kMaxNear) return -1;
                    lst[n++] = make_int2(X, code);
                }
            } else {
                for (int cc = 0; cc < (1 << d); ++cc) {
                    const int Y = v.child0[X] + cc;
                    if (v.child0[Y] >= 0) return -1;
                    if (v.src_e[Y] > v.src_b[Y]) {
                        if (n >= kMaxNear) return -1;
                        lst[n++] = make_int2(Y, code);
                    }
                }
            }
            continue;
        }
        // no same-level box: the colleague of b's parent at the parent-level cell
        if (L == 0) continue;
        const int pb = v.parent[b];
        int oi = 0, mul = 1, rr = o;
        for (int a = 0; a < d; ++a) {
            const long long cc = v.coord[size_t(b) * d + a] + (rr % 3) - 1;
            rr /= 3;
            oi += int((cc >> 1) - v.coord[size_t(pb) * d + a] + 1) * mul;
            mul *= 3;
        }
        const int F = v.colleague[size_t(pb) * nn + oi];
        if (F >= 0 && v.child0[F] < 0 && v.src_e[F] > v.src_b[F]) {
            if (n >= kMaxNear) return -1;
            lst[n++] = make_int2(F, code);
        }
    }
    for (int i = 1; i < n; ++i) {
        const int2 k = lst[i];
        int j = i - 1;
        while (j >= 0 && (lst[j].x > k.x || (lst[j].x == k.x && lst[j].y > k.y))) {
            lst[j + 1] = lst[j];
            --j;
        }
        lst[j + 1] = k;
    }
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (m == 0 || lst[i].x != lst[m - 1].x || lst[i].y != lst[m - 1].y) lst[m++] = lst[i];
    return m;
}

__global__ void k_tleaf_flags(int nb, const int* __restrict__ child0, const long long* __restrict__ tb,
                              const long long* __restrict__ te, unsigned char* __restrict__ flag) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        flag[b] = child0[b] < 0 && te[b] > tb[b];
}

__global__ void k_near_count(BoxView v, Geo g, int ntleaf, const int* __restrict__ tleaf,
                             const long long* __restrict__ tb, const long long* __restrict__ te, int split32,
                             long long* __restrict__ cnt, long long* __restrict__ nsrc, long long* __restrict__ pairs,
                             long long* __restrict__ ndesc, int* __restrict__ err) {
    int2 lst[kMaxNear];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ntleaf; k += gridDim.x * blockDim.x) {
        const int b = tleaf[k];
        int m = near_list_of(v, g, b, lst);
        if (m < 0) {
            atomicExch(err, 1);
            m = 0;
        }
        long long ns = 0;
        for (int i = 0; i < m; ++i) ns += v.src_e[lst[i].x] - v.src_b[lst[i].x];
        const long long nt = te[b] - tb[b];
        cnt[k] = m;
        nsrc[k] = ns;
        pairs[k] = ns * nt;
        ndesc[k] = split32 ? (nt > 32 ? (nt + 31) / 32 : 1) : 1;
    }
}

__global__ void k_near_fill(BoxView v, Geo g, int ntleaf, const int* __restrict__ tleaf,
                            const long long* __restrict__ tb, const long long* __restrict__ te,
                            const long long* __restrict__ lbeg, const long long* __restrict__ dbeg,
                            const long long* __restrict__ nsrc, int split32, int* __restrict__ list,
                            int* __restrict__ shift, TLeaf* __restrict__ desc, unsigned long long* __restrict__ key) {
    int2 lst[kMaxNear];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ntleaf; k += gridDim.x * blockDim.x) {
        const int b = tleaf[k];
        const int m = max(near_list_of(v, g, b, lst), 0);
        const long long e0 = lbeg[k];
        for (int i = 0; i < m; ++i) {
            list[e0 + i] = lst[i].x;
            shift[e0 + i] = lst[i].y;
        }
        const int nt = int(te[b] - tb[b]);
        TLeaf base;
        base.tgt_begin = int(tb[b]);
        base.tgt_count = nt;
        base.list_begin = int(e0);
        base.list_count = m;
        base.level = v.level[b];
        base.box = b;
        base.pad0 = base.pad1 = 0;
        long long j = dbeg[k];
        if (split32) {
            for (int t0 = 0; t0 < max(nt, 1); t0 += 32, ++j) {
                TLeaf c = base;
                c.tgt_begin = base.tgt_begin + t0;
                c.tgt_count = min(32, nt - t0);
                desc[j] = c;
                key[j] = ~static_cast<unsigned long long>(nsrc[k] * c.tgt_count);  // decreasing cost
            }
        } else {
            desc[j] = base;
            key[j] = ~static_cast<unsigned long long>(nsrc[k] * nt);
        }
    }
}

__global__ void k_gather_desc(int64_t n, const int* __restrict__ idx, const TLeaf* __restrict__ in,
                              TLeaf* __restrict__ out) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x)
        out[j] = in[idx[j]];
}

__global__ void k_box_src(int nb, const long long* __restrict__ sb, const long long* __restrict__ se,
                          int* __restrict__ bsb, int* __restrict__ bsc) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        bsb[b] = int(sb[b]);
        bsc[b] = int(se[b] - sb[b]);
    }
}

BoxView box_view(const GpuBuild& b, int d) {
    BoxView v;
    v.d = d;
    v.nn = d == 3 ? 27 : 9;
    v.level = b.d_level;
    v.coord = b.d_coord;
    v.parent = b.d_parent;
    v.child0 = b.d_child0;
    v.src_b = b.d_src_b;
    v.src_e = b.d_src_e;
    v.colleague = b.d_colleague;
    return v;
}

}  // namespace

int gpu_near_count(GpuBuild* b, const Geometry& g, bool split32, NearLists* nl, cudaStream_t s, std::string* msg) {
    Scratch scr(b->pool, b->scratch);
    const int nb = b->nb, d = g.d;
    const Geo geo = make_geo(g);
    unsigned char* flag;
    int *iota, *nsel, *err;
    GB_ALLOC(flag, unsigned char, nb);
    GB_ALLOC(iota, int, nb);
    GB_ALLOC(nsel, int, 1);
    GB_ALLOC(err, int, 1);
    int r;
    if ((r = own(b, &nl->d_tleaf, nb, msg))) return r;
    k_tleaf_flags<<<blocks_for(nb), kThreads, 0, s>>>(nb, b->d_child0, b->d_tgt_b, b->d_tgt_e, flag);
    k_iota_int<<<blocks_for(nb), kThreads, 0, s>>>(iota, nb);
    size_t tb = 0;
    unsigned char* d_tmp = nullptr;
    size_t have = 0;
    auto tmp = [&](size_t need) -> bool {
        if (need <= have) return true;
        d_tmp = scr.get<unsigned char>(need);
        have = d_tmp ? need : 0;
        return d_tmp != nullptr;
    };
    GB_CK(cub::DeviceSelect::Flagged(nullptr, tb, iota, flag, nl->d_tleaf, nsel, nb, s));
    if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceSelect::Flagged(d_tmp, tb, iota, flag, nl->d_tleaf, nsel, nb, s));
    int ntl = 0;
    GB_CK(cudaMemcpyAsync(&ntl, nsel, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    GB_CK(cudaStreamSynchronize(s));
    nl->ntleaf = ntl;
    long long *cnt, *pairs, *ndesc, *psum;
    GB_ALLOC(cnt, long long, size_t(ntl) + 1);
    GB_ALLOC(pairs, long long, std::max(ntl, 1));
    GB_ALLOC(ndesc, long long, size_t(ntl) + 1);
    GB_ALLOC(psum, long long, 1);
    if ((r = own(b, &nl->d_nsrc, std::max(ntl, 1), msg))) return r;
    if ((r = own(b, &nl->d_list_begin, size_t(ntl) + 1, msg))) return r;
    if ((r = own(b, &nl->d_desc_begin, size_t(ntl) + 1, msg))) return r;
    GB_CK(cudaMemsetAsync(cnt + ntl, 0, sizeof(long long), s));
    GB_CK(cudaMemsetAsync(ndesc + ntl, 0, sizeof(long long), s));
    GB_CK(cudaMemsetAsync(psum, 0, sizeof(long long), s));
    if (ntl > 0) {
        k_near_count<<<blocks_for(ntl), 128, 0, s>>>(box_view(*b, d), geo, ntl, nl->d_tleaf, b->d_tgt_b, b->d_tgt_e,
                                                      split32 ? 1 : 0, cnt, nl->d_nsrc, pairs, ndesc, err);
        GB_CK(cudaGetLastError());
        GB_CK(cub::DeviceReduce::Sum(nullptr, tb, pairs, psum, ntl, s));
        if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
        GB_CK(cub::DeviceReduce::Sum(d_tmp, tb, pairs, psum, ntl, s));
    }
    GB_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, nl->d_list_begin, ntl + 1, s));
    if (!tmp(tb)) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceScan::ExclusiveSum(d_tmp, tb, cnt, nl->d_list_begin, ntl + 1, s));
    GB_CK(cub::DeviceScan::ExclusiveSum(d_tmp, tb, ndesc, nl->d_desc_begin, ntl + 1, s));
    long long h[3] = {0, 0, 0};
    int herr = 0;
    GB_CK(cudaMemcpyAsync(&h[0], nl->d_list_begin + ntl, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemcpyAsync(&h[1], nl->d_desc_begin + ntl, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemcpyAsync(&h[2], psum, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaStreamSynchronize(s));  // the scratch is freed on return
    if (herr) {
        if (msg) *msg = "a near-field list outgrew its bound (host lists used)";
        return PDMK_ERR_INTERNAL;
    }
    nl->nlist = h[0];
    nl->ndesc = h[1];
    nl->pairs = h[2];
    if ((r = own(b, &nl->d_shift, std::max<int64_t>(nl->nlist, 1), msg))) return r;
    return PDMK_OK;
}

int gpu_near_fill(GpuBuild* b, const Geometry& g, bool split32, NearLists* nl, int* d_list, TLeaf* d_desc,
                  int* d_bsb, int* d_bsc, cudaStream_t s, std::string* msg) {
    Scratch scr(b->pool, b->scratch);
    const int d = g.d, ntl = nl->ntleaf;
    const int64_t nd = nl->ndesc;
    k_box_src<<<blocks_for(b->nb), kThreads, 0, s>>>(b->nb, b->d_src_b, b->d_src_e, d_bsb, d_bsc);
    if (ntl == 0 || nd == 0) {
        GB_CK(cudaGetLastError());
        return PDMK_OK;
    }
    TLeaf* dtmp;
    unsigned long long *key, *key2;
    int *idx, *idx2;
    GB_ALLOC(dtmp, TLeaf, nd);
    GB_ALLOC(key, unsigned long long, nd);
    GB_ALLOC(key2, unsigned long long, nd);
    GB_ALLOC(idx, int, nd);
    GB_ALLOC(idx2, int, nd);
    k_near_fill<<<blocks_for(ntl), 128, 0, s>>>(box_view(*b, d), make_geo(g), ntl, nl->d_tleaf, b->d_tgt_b, b->d_tgt_e,
                                                 nl->d_list_begin, nl->d_desc_begin, nl->d_nsrc, split32 ? 1 : 0, d_list,
                                                 nl->d_shift, dtmp, key);
    GB_CK(cudaGetLastError());
    k_iota_int<<<blocks_for(nd), kThreads, 0, s>>>(idx, nd);
    size_t tb = 0;
    GB_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, key, key2, idx, idx2, int(nd), 0, 64, s));
    unsigned char* d_tmp = scr.get<unsigned char>(tb);
    if (!d_tmp) { if (msg) *msg = "device allocation failed (set-up)"; return PDMK_ERR_CUDA; }
    GB_CK(cub::DeviceRadixSort::SortPairs(d_tmp, tb, key, key2, idx, idx2, int(nd), 0, 64, s));
    k_gather_desc<<<blocks_for(nd), kThreads, 0, s>>>(nd, idx2, dtmp, d_desc);
    GB_CK(cudaGetLastError());
    GB_CK(cudaStreamSynchronize(s));  // the scratch is freed on return
    return PDMK_OK;
}

}  // namespace pdmk
