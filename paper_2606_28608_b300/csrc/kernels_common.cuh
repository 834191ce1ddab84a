// kernels_common.cuh -- shared device helpers: series evaluation, compensated sums,
// launch-time argument structs.  Templated on the arithmetic type T (double for the
// FP64 path, float for the mixed path).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pdmk {

constexpr int kMaxCheb = 40;  // Chebyshev terms held per kernel function
constexpr int kNearMono = 24;  // monomial terms of the warp near-field kernel's series (its longest instance)

// Chebyshev series in x in [-1, 1] by Clenshaw's recurrence (stable in FP32).
template <typename T>
__device__ __forceinline__ T clenshaw(const T* __restrict__ c, int n, T x) {
    T b1 = T(0), b2 = T(0);
    const T x2 = x + x;
    for (int k = n - 1; k >= 1; --k) {
        T b0 = fma(x2, b1, c[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(x, b1, c[0] - b2);
}

// Compensated (Kahan) accumulation of partial sums.  In FP64 the correction term stays ~0.
template <typename T>
struct Kahan {
    T s, c;
    __device__ __forceinline__ void init() { s = T(0); c = T(0); }
    __device__ __forceinline__ void add(T v) {
        T y = v - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

// -------- near field ----------------------------------------------------------------
struct TLeaf {
    int tgt_begin, tgt_count;  // sorted-target range
    int list_begin, list_count;
    int level, box;
    int pad0, pad1;
};

template <typename T>
struct NearArgs {
    const TLeaf* tleaf;
    int ntleaf;
    const int* list;            // source leaf box ids
    const int* box_src_begin;   // per box
    const int* box_src_count;   // per box
    const double* box_center;   // d per box
    const T* src4;              // per sorted source: (x, y, z, q), relative to its leaf centre
    const T* tgt4;              // per sorted target: (x, y, z, q), relative to its leaf centre
    double* pot;                // per sorted target
    double* grad;               // d per sorted target, or nullptr
    double inv_rc;              // 1 / r_c
    const T* coefA;             // kMaxCheb
    const T* coefB;
    int nA, nB;
    unsigned long long* count_in;  // if not null: adds the number of pairs inside the support
    // mixed path: pairs with (r/h)^2 < close_s take their difference in two-float
    // arithmetic from hi + lo coordinates (plain FP32 cancels for r << h)
    const T* src_lo;            // 4 per sorted source: lo parts of the leaf-relative coordinates
    const T* tgt_lo;            // 4 per sorted target
    T close_s;
    // warp kernel: per direct-list entry the source range and the shift of the source leaf's
    // centre into the target leaf's frame (hi, and lo on the mixed path), 4 T per entry
    const int2* ent;
    const T* ent_sh;
    const T* ent_shlo;
    // warp kernel: A and B as monomials in x = 2 s - 1 (zero-padded), by value: the kernel's
    // Horner steps take them as constant operands instead of holding them in registers
    T cmA[kNearMono];
    T cmB[kNearMono];
};

// -------- far field -----------------------------------------------------------------
template <typename T>
struct SpreadArgs {
    const int4* pt_g0;      // per spread point: grid index of the first window node per dim
    const T* pt_dq;         // per spread point: 4 values (delta_x, delta_y, delta_z, q)
    const int4* sub;        // per subproblem: (bin, begin, count, 0)
    int nsub;
    T* slab;                // nsub * Ptot
    int P0, P1, P2, Ptot;   // padded tile dims
    int B0, B1, B2;         // bin dims
    int w;
    T half_w_inv2;          // (2/w)^2
    const T* coefW;         // window F(s), s = (2z/w)^2, Chebyshev in 2s - 1
    int nW;
};

template <typename T, typename G>
struct FoldArgs {
    const T* slab;
    const int* bin_sub_begin;  // per bin: first subproblem (nbin + 1 entries)
    G* grid;                   // M0*M1*M2, in the precision of the transforms
    int M0, M1, M2;
    int nb0, nb1, nb2;
    int B0, B1, B2;
    int P0, P1, P2, Ptot;
    int fw;                    // floor(w/2)
};

template <typename T>
struct InterpArgs {
    const T* grid;
    const int4* t_g0;     // per target
    const T* t_dq;        // per target: (delta_x, delta_y, delta_z, unused)
    int nt;
    int M0, M1, M2;
    int w;
    T half_w_inv2;
    const T* coefW;       // window F(s)
    const T* coefWd;      // dF/ds
    int nW, nWd;
    double* pot;          // per target
    double* gradu;        // d per target: gradient w.r.t. grid coordinates (M_i u_i)
};

}  // namespace pdmk
