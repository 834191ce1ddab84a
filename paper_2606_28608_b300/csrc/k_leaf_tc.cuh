// k_leaf_tc.cuh -- 3D leaf evaluation (Sec. 3.5) on the fifth-generation tensor cores.
//
// For a target leaf with local coefficients a[m0][m1][m2] (P per axis) and targets t at leaf
// coordinates (x, y, z) in [-1, 1]^3,
//     phi_t = sum_m a[m] T_m0(x) T_m1(y) T_m2(z),   grad_t from T'_m = m U_{m-1},
// the x contraction is a dense product: rows X = [T_m0(x_t) (64 targets); T'_m0(x_t) (the same
// 64)] (128 x P) times the coefficients viewed as P x P^2, in chunks of 8 P columns (8 values
// of m1 by P of m2):
//     C[r][n] = sum_m0 X[r][m0] a[m0][n]          (tcgen05.mma kind::tf32, M = 128, N = 8 P)
// accumulated in tensor memory.  TF32 keeps 10 mantissa bits, so every operand is split as
// x = hi + lo (hi: x rounded to TF32, lo: the remainder rounded to TF32, |x - hi - lo| <=
// 2^-24 |x|) and the product is hi*hi + hi*lo + lo*hi with FP32 accumulation, which holds the
// FP32 result's accuracy (the dropped lo*lo term is below 2^-22 relative).  The epilogue reads each row of C from
// tensor memory (a thread per row: the T rows give the potential and the y, z derivatives,
// the T' rows the x derivative) and weights the columns by T_m1(y) T_m2(z) and the derivative
// tables in FP32.  Every sum has a fixed order: results do not depend on scheduling.
//
// Operands sit in shared memory in the canonical K-major layout without swizzling: 8-row by
// 16-byte core matrices, core matrices adjacent along K 128 bytes apart, 8-row groups 32 P
// bytes apart.  One CTA of 128 threads per SM pair slot (two resident per SM), persistent over
// the leaves; thread 0 issues the MMAs and commits them to an mbarrier, on which every thread
// waits with an iteration limit (on expiry: the plan's error flag, one more bounded wait, the
// tensor memory freed, return).
#pragma once
#include <cstdint>

namespace pdmk {
namespace tcg {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor (start address, leading- and stride-dimension byte offsets,
// descriptor version 1, no swizzle)
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((addr & 0x3FFFFu) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// instruction descriptor: D in FP32, A and B in TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ uint32_t try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok;
}
// bounded wait on the mbarrier phase of the given parity
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// x rounded to the nearest TF32 value (10 mantissa bits; the low 13 bits of the result are zero)
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// x = hi + lo with hi and lo TF32 values: |x - hi - lo| <= 2^-24 |x|
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = tf32_rn(x);
    lo = tf32_rn(x - hi);
}

}  // namespace tcg

template <int P>
struct LeafTcLayout {
    static constexpr int NC = 8 * P;                            // columns per chunk
    static constexpr uint32_t SBO = 32 * P;                     // bytes between 8-row groups
    static constexpr size_t b_bytes = size_t(NC) * P * 4;       // one chunk, hi or lo
    static constexpr size_t a_bytes = size_t(128) * P * 4;      // 128 rows, hi or lo
    static constexpr size_t tb_bytes = size_t(4) * P * 64 * 4;  // Ty, Ty', Tz, Tz' of 64 targets
    static constexpr size_t off_bl = b_bytes, off_ah = 2 * b_bytes, off_al = off_ah + a_bytes,
                            off_tb = off_al + a_bytes, off_bar = off_tb + tb_bytes, total = off_bar + 16;
};

// byte offset of element (row r, k) in a K-major operand with 8-row groups SBO bytes apart
template <int P>
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
    return uint32_t(r >> 3) * LeafTcLayout<P>::SBO + uint32_t(k >> 2) * 128u + uint32_t(r & 7) * 16u + uint32_t(k & 3) * 4u;
}

// Chebyshev values T_m(v) and derivatives T'_m(v) = m U_{m-1}(v), m < P
template <int P>
__device__ __forceinline__ void cheb_rows(float v, float* tr, float* dr) {
    float tm1 = 1.f, tm = v, um1 = 1.f, um = 2.f * v;
    tr[0] = 1.f;
    dr[0] = 0.f;
    tr[1] = v;
    dr[1] = 1.f;
#pragma unroll
    for (int m = 2; m < P; ++m) {
        const float tn = fmaf(2.f * v, tm, -tm1);
        tr[m] = tn;
        dr[m] = float(m) * um;
        const float un = fmaf(2.f * v, um, -um1);
        tm1 = tm;
        tm = tn;
        um1 = um;
        um = un;
    }
}

// list entry int4 = (local slot, first target, target count, level); persistent over entries
template <int P>
__global__ void __launch_bounds__(128, 2)
    k_leaf_eval3d_tc(const int4* __restrict__ list, int nlist, const float* __restrict__ Lc,
                     const float* __restrict__ tgt4, double* __restrict__ pot, double* __restrict__ grad,
                     double inv_rc, int* __restrict__ err) {
    using Lay = LeafTcLayout<P>;
    constexpr int NC = Lay::NC, NCH = P / 8, KS = P / 8, PP = P * P;
    constexpr uint32_t IDESC = tcg::idesc_tf32(128, NC);
    static_assert(P % 8 == 0 && NC % 32 == 0 && NC <= 256, "tile shape");
    extern __shared__ __align__(1024) unsigned char smtc[];
    unsigned char* Bh = smtc;
    unsigned char* Bl = smtc + Lay::off_bl;
    unsigned char* Ah = smtc + Lay::off_ah;
    unsigned char* Al = smtc + Lay::off_al;
    float* TB = reinterpret_cast<float*>(smtc + Lay::off_tb);  // [4][P][64]: Ty, Ty', Tz, Tz'
    uint64_t* bar = reinterpret_cast<uint64_t*>(smtc + Lay::off_bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smtc + Lay::off_bar + 8);
    const int tid = threadIdx.x, warp = tid >> 5, t = tid & 63;
    const bool vrow = tid < 64;  // T rows (potential, y and z derivatives); else T' rows (x derivative)
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcg::smem_addr(bar)) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(tcg::smem_addr(slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tcg::fence_before();
    __syncthreads();
    tcg::fence_after();
    const uint32_t tmem = *slot;
    const uint32_t taddr = tmem + (uint32_t(32 * warp) << 16);
    uint32_t phase = 0;
    bool failed = false;
    for (int li = blockIdx.x; li < nlist && !failed; li += gridDim.x) {
        const int4 e = list[li];
        const double sc = 2.0 * inv_rc * double(1LL << e.w);  // dt/dx = 2/h
        const float* a = Lc + size_t(e.x) * (PP * P);
        for (int t0 = 0; t0 < e.z && !failed; t0 += 64) {
            const int nt = min(64, e.z - t0);
            const bool live = t < nt;
            // ---- rows of the tile's targets (thread t: x axis; thread 64 + t: y and z tables)
            if (vrow) {
                float tr[P], dr[P];
                const float xv = live ? float(double(tgt4[size_t(e.y + t0 + t) * 4]) * sc) : 0.f;
                cheb_rows<P>(xv, tr, dr);
                const float s0 = live ? 1.f : 0.f;  // rows of absent targets are zero
#pragma unroll
                for (int g = 0; g < P / 4; ++g) {
                    float th[4], tl[4], dh[4], dl[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        tcg::split_tf32(tr[4 * g + j] * s0, th[j], tl[j]);
                        tcg::split_tf32(dr[4 * g + j] * s0, dh[j], dl[j]);
                    }
                    *reinterpret_cast<float4*>(Ah + kmajor_off<P>(t, 4 * g)) = make_float4(th[0], th[1], th[2], th[3]);
                    *reinterpret_cast<float4*>(Al + kmajor_off<P>(t, 4 * g)) = make_float4(tl[0], tl[1], tl[2], tl[3]);
                    *reinterpret_cast<float4*>(Ah + kmajor_off<P>(64 + t, 4 * g)) = make_float4(dh[0], dh[1], dh[2], dh[3]);
                    *reinterpret_cast<float4*>(Al + kmajor_off<P>(64 + t, 4 * g)) = make_float4(dl[0], dl[1], dl[2], dl[3]);
                }
            } else {
                float tr[P], dr[P];
#pragma unroll
                for (int ax = 1; ax <= 2; ++ax) {
                    const float v = live ? float(double(tgt4[size_t(e.y + t0 + t) * 4 + ax]) * sc) : 0.f;
                    cheb_rows<P>(v, tr, dr);
#pragma unroll
                    for (int m = 0; m < P; ++m) {
                        TB[((2 * (ax - 1)) * P + m) * 64 + t] = tr[m];
                        TB[((2 * (ax - 1) + 1) * P + m) * 64 + t] = dr[m];
                    }
                }
            }
            float accP = 0.f, accX = 0.f, accY = 0.f, accZ = 0.f;
#pragma unroll 1
            for (int c = 0; c < NCH; ++c) {
                // ---- the chunk's coefficients: column n <-> (m1 = 8 c + n / P, m2 = n % P); task
                //      (n, g) moves a[4g .. 4g+3][NC c + n] as one K-group of hi and of lo.  Every
                //      thread's loads are issued before the first is used.
                constexpr int TASKS = NC * (P / 4) / 128;
                static_assert(TASKS * 128 == NC * (P / 4), "tasks split evenly over the block");
                float xs[TASKS][4];
#pragma unroll
                for (int i = 0; i < TASKS; ++i) {
                    const int task = tid + 128 * i, n = task % NC, g = task / NC;
                    const float* src = a + size_t(4 * g) * PP + NC * c + n;
#pragma unroll
                    for (int j = 0; j < 4; ++j) xs[i][j] = __ldg(src + j * PP);
                }
#pragma unroll
                for (int i = 0; i < TASKS; ++i) {
                    const int task = tid + 128 * i, n = task % NC, g = task / NC;
                    float h[4], l[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) tcg::split_tf32(xs[i][j], h[j], l[j]);
                    const uint32_t off = kmajor_off<P>(n, 4 * g);
                    *reinterpret_cast<float4*>(Bh + off) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(Bl + off) = make_float4(l[0], l[1], l[2], l[3]);
                }
                tcg::fence_async_smem();
                tcg::fence_before();
                __syncthreads();
                tcg::fence_after();
                if (tid == 0) {
                    const uint32_t ah = tcg::smem_addr(Ah), al = tcg::smem_addr(Al);
                    const uint32_t bh = tcg::smem_addr(Bh), bl = tcg::smem_addr(Bl);
#pragma unroll
                    for (int s = 0; s < KS; ++s) {
                        const uint32_t ko = uint32_t(s) * 256u;  // 8 K values = two core matrices
                        tcg::mma_tf32(tmem, tcg::desc_kmajor(ah + ko, 128, Lay::SBO), tcg::desc_kmajor(bh + ko, 128, Lay::SBO),
                                      IDESC, s > 0 ? 1u : 0u);
                        tcg::mma_tf32(tmem, tcg::desc_kmajor(ah + ko, 128, Lay::SBO), tcg::desc_kmajor(bl + ko, 128, Lay::SBO),
                                      IDESC, 1u);
                        tcg::mma_tf32(tmem, tcg::desc_kmajor(al + ko, 128, Lay::SBO), tcg::desc_kmajor(bh + ko, 128, Lay::SBO),
                                      IDESC, 1u);
                    }
                    tcg::commit(bar);
                }
                const bool ok = tcg::wait_bounded(bar, phase & 1u);
                ++phase;
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
                tcg::fence_after();
                // ---- this thread's row of the chunk: sums over m2 per m1, then over m1
                float tz[P], tzd[P];
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    tz[m] = TB[(2 * P + m) * 64 + t];
                    tzd[m] = vrow ? TB[(3 * P + m) * 64 + t] : 0.f;
                }
                float u[8], v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) u[j] = v[j] = 0.f;
#pragma unroll
                for (int q = 0; q < NC / 32; ++q) {
                    uint32_t r[32];
                    tcg::ld32(taddr + uint32_t(32 * q), r);
                    tcg::wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int n = 32 * q + i, j = n / P, m2 = n - (n / P) * P;
                        const float cv = __uint_as_float(r[i]);
                        u[j] = fmaf(cv, tz[m2], u[j]);
                        if (vrow) v[j] = fmaf(cv, tzd[m2], v[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int m1 = 8 * c + j;
                    const float ty = TB[m1 * 64 + t];
                    if (vrow) {
                        const float tyd = TB[(P + m1) * 64 + t];
                        accP = fmaf(ty, u[j], accP);
                        accY = fmaf(tyd, u[j], accY);
                        accZ = fmaf(ty, v[j], accZ);
                    } else {
                        accX = fmaf(ty, u[j], accX);
                    }
                }
                // the next chunk rewrites the operands and tensor memory: every read is done
                tcg::fence_before();
                __syncthreads();
            }
            if (!failed && live) {
                const size_t o = size_t(e.y + t0 + t);
                if (vrow) {
                    pot[o] = double(accP);
                    if (grad) {
                        grad[o * 3 + 1] = double(accY) * sc;
                        grad[o * 3 + 2] = double(accZ) * sc;
                    }
                } else if (grad) {
                    grad[o * 3 + 0] = double(accX) * sc;
                }
            }
            __syncthreads();  // the tables of the next tile
        }
    }
    if (failed) {
        // the wait expired: report, wait once more (bounded) for the MMAs in flight, then free
        if (tid == 0 && err) *reinterpret_cast<volatile int*>(err) = 1;
        tcg::wait_bounded(bar, (phase - 1u) & 1u);
    }
    tcg::fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}


}  // namespace pdmk
