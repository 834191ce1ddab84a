// capi.cu -- the C ABI of include/pdmk.h: plan creation (FP64 host planning), source set-up
// (images, tree, device layouts) and the evaluation launch sequence on one CUDA stream.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "dev_pool.h"
#include "gpu_build.h"
#include "host_plan.h"
#include "k_assemble.cuh"
#include "k_bloch.cuh"
#include "k_farfield.cuh"
#include "k_nearfield.cuh"
#include "k_pw.cuh"
#include "kernels_common.cuh"
#include "pdmk.h"

using namespace pdmk;

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) {                             \
            plan_set_msg(plan, cudaGetErrorString(e_));      \
            return PDMK_ERR_CUDA;                            \
        }                                                    \
    } while (0)
#define CKFFT(call)                                          \
    do {                                                     \
        cufftResult r_ = (call);                             \
        if (r_ != CUFFT_SUCCESS) {                           \
            plan_set_msg(plan, "cufft failure");             \
            return PDMK_ERR_CUDA;                            \
        }                                                    \
    } while (0)

// streaming multiprocessors of the current device (grid sizing)
static int device_sms() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        return 1;
    }
    return nsm;
}

struct pdmk_plan_s {
    int d = 3;
    double eps = 1e-6;
    double Lc[9] = {0};  // the caller's lattice (column-major), kept for autotuning
    pdmk_opts opts{};
    double c = 0, kappa = 0, beta = 0;
    int n_s = 0, w = 0, max_depth = 0;
    Geometry g;
    KernelTables kt;
    WindowTables wt;
    std::vector<double> cA, cB, cW, cWd;  // near-field Chebyshev coefficients (FP64 master copy)
    std::vector<double> mA, mB;  // A and B as monomials in x = 2 s - 1 (warp near-field kernel)
    int near_nh = 0;             // > 0: warp near-field kernel with this many monomial terms
    std::vector<double> mW, mWd; // window F, dF as monomials in x = 2 s - 1
    bool far_halo = false;       // 2D FP32 halo-grid spreading / interpolation kernels
    bool far_warp3d = false;     // 3D warp-per-target interpolation
    bool spread_reg3d = false;   // 3D spreading with the padded tile in registers (k_spread3d_reg)
    int B[3] = {1, 1, 1}, nbin[3] = {1, 1, 1}, P[3] = {1, 1, 1}, Ptot = 1;
    int whole_ctas = 0;  // > 0: 2D whole-grid spreading with this many CTAs (small grids)
    int64_t ncell = 1, nhalf = 1;
    cudaStream_t stream = nullptr;  // the caller's stream
    cudaStream_t ws = nullptr;      // the plan's own work stream (graph capture needs a non-default stream)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // branches of one evaluation: the plane-wave chain (highest priority: many small
    // latency-bound launches) and the near-field sum run beside the far field on ws
    cudaStream_t ws_pw = nullptr, ws_near = nullptr;
    cudaEvent_t ev_s = nullptr, ev_pw = nullptr, ev_near = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double* g_pot = nullptr;
    double* g_grad = nullptr;
    int evals_since_setup = 0;
    bool ready = false;
    std::string msg;
    // plan-lifetime device buffers
    std::vector<std::pair<void*, size_t>> plan_allocs, src_allocs;  // (buffer, bytes)
    DevicePool pool;  // the previous set-up's buffers, offered to the next (dev_pool.h)
    void* d_coefA = nullptr;
    void* d_coefB = nullptr;
    void* d_coefW = nullptr;
    void* d_coefWd = nullptr;
    void* d_monoW = nullptr;
    void* d_monoWd = nullptr;
    double* d_weight = nullptr;
    void* d_grid = nullptr;
    void* d_grid64 = nullptr;  // grid of the transforms (the grid itself unless FP64 transforms of a mixed plan)
    bool fft32 = false;        // FP32 transforms (2D mixed plans)
    void* d_spec = nullptr;
    double* d_qsums = nullptr;
    double* d_qsum_part = nullptr;  // [sum_blocks][3] partial charge sums
    int nsm = 1;                    // SMs of the plan's device
    int sum_blocks = 2;             // blocks of the two-stage charge sums (2 per SM)
    unsigned long long* d_count = nullptr;
    bool count_pending = false;
    cufftHandle fft_fwd = 0, fft_inv = 0;
    bool have_fft = false;
    // source-dependent device buffers
    int64_t n = 0, nimg = 0, ntgt = 0, nspread = 0;
    int nbox = 0, ntleaf = 0, nsub = 0, nbins_tot = 1;
    int nnear = 0;  // near-field descriptors (target leaves cut into groups of 32 targets)
    void* d_src4 = nullptr;
    int* d_src_orig = nullptr;
    void* d_tgt4 = nullptr;
    void* d_src_lo = nullptr;
    void* d_tgt_lo = nullptr;
    int* d_tgt_orig = nullptr;
    double* d_q_tgt = nullptr;
    double* d_self_w = nullptr;
    TLeaf* d_tleaf = nullptr;
    int* d_list = nullptr;
    int2* d_ent = nullptr;      // per direct-list entry: source range
    void* d_ent_sh = nullptr;   // per entry: shift into the target leaf's frame (4 T)
    void* d_ent_shlo = nullptr; // per entry: lo part of the shift (mixed)
    int* d_box_src_begin = nullptr;
    int* d_box_src_count = nullptr;
    double* d_box_center = nullptr;
    int4* d_pt_g0 = nullptr;
    void* d_pt_dq = nullptr;
    int* d_spread_orig = nullptr;
    int4* d_sub = nullptr;
    int* d_bin_sub_begin = nullptr;
    void* d_slab = nullptr;
    void* slab_override = nullptr;  // set only for the duration of pdmk_eval_noalloc
    double* d_adj = nullptr;        // adjoint scratch (n (4 + 2 d) doubles), allocated on first use
    int64_t n_src = 0;              // the caller's sources (n = n_src + separate targets)
    int64_t out_first = 0;          // first caller-order point written by pdmk_eval
    int64_t n_out = 0;              // points written by pdmk_eval
    int4* d_t_g0 = nullptr;
    void* d_t_dq = nullptr;
    double* d_pot_near = nullptr;
    double* d_grad_near = nullptr;
    double* d_pot_far = nullptr;
    double* d_gradu_far = nullptr;
    double* d_q_user = nullptr;
    double* d_pot_out = nullptr;
    double* d_grad_out = nullptr;
    PwPlan pw;  // plane-wave (difference-kernel) passes
    // host copies kept after set_sources for evaluations at new targets (pdmk_eval_targets)
    Tree h_tree;
    std::vector<double> h_u;                   // fractional coordinates of the plan's points (n x d)
    std::vector<int64_t> h_src_orig;           // sorted source -> point index
    std::vector<unsigned char> h_src_is_orig;  // the sorted source is the point itself, not an image
    std::vector<double> h_Cu;                  // caller-frame centre of every box (d per box)
    // after a 3D device set-up the per-box arrays of h_tree (and h_Cu) are read back from the
    // device tree only when a host path needs them (host_tree false until then)
    bool host_tree = true;
    GpuBuild tree_dev;                                      // its device arrays (pointers)
    std::vector<std::pair<void*, size_t>> tree_keep;        // the same, owned by the plan
    std::vector<double> h_y;                   // the caller's positions (n x d)
    std::vector<double> h_src_disp;            // per sorted source: caller-frame lattice vector from
                                               // its point's given position to this copy (d each)
    // quasi-periodic evaluation (pdmk_eval_bloch): buffers made on first use
    bool bl_ready = false;
    double* bl_buf = nullptr;     // device block: displacements, positions, grids, weights, results
    cufftHandle bl_fft = 0;       // complex-to-complex transform of the full grid (FP64)
    bool bl_have_fft = false;
    double* bl_tab = nullptr;     // device: quadrature of the smoothing transform and window tables
    // per-call target scratch of pdmk_eval_targets (grown on demand, kept until set_sources)
    void* tq_buf = nullptr;
    size_t tq_cap = 0;
    // profiling
    std::vector<cudaEvent_t> ev;
    std::vector<std::string> stage_names;
    std::vector<double> stage_ms;
    // page-locked staging of the device set-up's downloads (kept for the plan's next set-up)
    unsigned char* h_stage = nullptr;
    size_t stage_cap = 0;
    // device set-up (gpu_build.cu): the per-point host copies are downloaded on first use
    bool setup_device = false;
    bool host_copies = true;
    double* d_u_keep = nullptr;     // fractional coordinates (n x d)
    double* d_y_keep = nullptr;     // the caller's positions (n x d)
    double* d_src_disp = nullptr;   // per sorted source: caller-frame lattice vector (d)
    int* d_tgt_of_keep = nullptr;   // per sorted target: sorted source index
    int64_t nlist = 0;              // direct-list entries
    // host phases of the last pdmk_set_sources (milliseconds, wall clock)
    std::vector<const char*> setup_names;
    std::vector<double> setup_ms;
    pdmk_info info{};
    int64_t device_bytes = 0;
    int launches = 0;  // kernels launched by the last eval (this library's own)
};

static void plan_set_msg(pdmk_plan plan, const char* m) {
    if (plan) plan->msg = m ? m : "";
}

template <class X>
static int dalloc(pdmk_plan plan, std::vector<std::pair<void*, size_t>>& list, X** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* p = plan->pool.get(count * sizeof(X));
    if (!p) {
        plan_set_msg(plan, "device allocation failed");
        return PDMK_ERR_OOM;
    }
    list.push_back({p, count * sizeof(X)});
    plan->device_bytes += int64_t(count * sizeof(X));
    *out = static_cast<X*>(p);
    return PDMK_OK;
}
#define DALLOC(list, ptr, type, count)                                          \
    do {                                                                        \
        type* tmp_ = nullptr;                                                   \
        int rc_ = dalloc<type>(plan, list, &tmp_, size_t(count));               \
        if (rc_ != PDMK_OK) return rc_;                                         \
        ptr = reinterpret_cast<decltype(ptr)>(tmp_);                            \
    } while (0)

template <class X>
static int upload(pdmk_plan plan, void* dst, const std::vector<X>& v) {
    if (v.empty()) return PDMK_OK;
    CK(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, plan->ws));
    return PDMK_OK;
}

static void free_list(std::vector<std::pair<void*, size_t>>& l, int64_t* bytes) {
    for (auto& a : l) cudaFree(a.first);
    l.clear();
    (void)bytes;
}

static size_t tsize(const pdmk_plan plan) { return plan->opts.precision == PDMK_MIXED ? 4 : 8; }

// spreading scratch: per-subproblem padded tiles, or one whole-grid slab per CTA
static size_t slab_bytes(const pdmk_plan plan) {
    const size_t tiles = size_t(std::max(plan->nsub, 1)) * size_t(plan->Ptot);
    const size_t whole = size_t(plan->whole_ctas) * size_t(plan->ncell);
    return std::max(tiles, whole) * tsize(plan);
}

extern "C" void pdmk_default_opts(pdmk_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->kappa = 0;
    o->n_s = 0;
    o->precision = PDMK_FP64;
    o->window_w = 0;
    o->n_proxy = 0;
    o->n_pw = 0;
    o->max_depth = -1;
    o->neutrality = 1;
    o->profile = 0;
    o->stream = nullptr;
    o->wait_test = 0;
    o->autotune = 0;
    o->root_mode = 0;
    o->build_mode = 0;
    o->tensor_cores = 0;
}

extern "C" const char* pdmk_strerror(int code) {
    switch (code) {
        case PDMK_OK: return "ok";
        case PDMK_ERR_BAD_ARG: return "bad argument";
        case PDMK_ERR_SINGULAR_LATTICE: return "singular lattice";
        case PDMK_ERR_NON_NEUTRAL: return "charges are not neutral";
        case PDMK_ERR_BAD_EPS: return "eps outside [1e-12, 1e-2]";
        case PDMK_ERR_NONFINITE: return "non-finite input";
        case PDMK_ERR_OOM: return "out of memory";
        case PDMK_ERR_CUDA: return "CUDA error";
        case PDMK_ERR_TIMEOUT: return "device wait timed out";
        case PDMK_ERR_NOT_READY: return "sources not set";
        case PDMK_ERR_INTERNAL: return "internal consistency check failed";
        case PDMK_ERR_TOO_LARGE: return "size exceeds the documented maximum";
        default: return "unknown error";
    }
}

// spreading bins: per dimension B <= M - w + 1 (a padded tile never wraps onto itself) and
// B >= ceil((w - 1)/6) (at most 8 tiles cover a grid cell per dimension); M grows if needed
static void size_bins(pdmk_plan plan) {
    const int d = plan->d, w = plan->w;
    const int Bdef = (d == 2) ? 32 : 8;
    const int Bmin = std::max(1, (w - 1 + 5) / 6);
    plan->Ptot = 1;
    plan->ncell = 1;
    for (int i = 0; i < 3; ++i) {
        if (i >= d) {
            plan->B[i] = 1; plan->nbin[i] = 1; plan->P[i] = 1; plan->g.M[i] = 1;
            continue;
        }
        int M = plan->g.M[i];
        if (M < Bmin + w - 1) {
            M = Bmin + w - 1;
            M += (M & 1);
            plan->g.M[i] = M;
        }
        int B = std::min(Bdef, M - w + 1);
        B = std::max(B, Bmin);
        plan->B[i] = B;
        plan->nbin[i] = (M + B - 1) / B;
        plan->P[i] = B + w - 1;
        plan->Ptot *= plan->P[i];
        plan->ncell *= M;
    }
    plan->nhalf = int64_t(plan->g.M[0] / 2 + 1) * plan->g.M[1] * (d == 3 ? plan->g.M[2] : 1);
    plan->nbins_tot = plan->nbin[0] * plan->nbin[1] * plan->nbin[2];
    // 2D grids whose 8 per-warp copies fit in ~96 KB of shared memory use whole-grid spreading
    const size_t ts = plan->opts.precision == PDMK_MIXED ? 4 : 8;
    plan->whole_ctas = (d == 2 && size_t(plan->ncell) * ts * 8 <= size_t(96) * 1024) ? 2 * plan->nsm : 0;
}

// Largest far-field weight over the one of the lowest nonzero mode.  Eq. (3.15) puts the
// band edge of axis i at its Nyquist index; where the band's ellipse in index space reaches
// the corners of the index box (strongly skewed cells), the window deconvolution of several
// axes multiplies, and rounding in the spread grid is amplified by this ratio.
static double far_amplification(pdmk_plan plan) {
    const int d = plan->d;
    const Geometry& g = plan->g;
    std::vector<double> ph[3];
    for (int i = 0; i < d; ++i) {
        ph[i].resize(g.M[i] / 2 + 1);
        for (int m = 0; m <= g.M[i] / 2; ++m) ph[i][m] = plan->wt.ft(double(m) / g.M[i]);
    }
    double wmax = 0, kmin = 1e300, wlow = 0;
    const int h0 = g.M[0] / 2, h1 = g.M[1] / 2, h2 = d == 3 ? g.M[2] / 2 : 0;
    for (int m2 = -h2 + (d == 3 ? 1 : 0); m2 < std::max(h2, 1); ++m2)
        for (int m1 = -h1 + 1; m1 < h1; ++m1)
            for (int m0 = 0; m0 < h0; ++m0) {
                if (m0 == 0 && m1 == 0 && m2 == 0) continue;
                const int m[3] = {m0, m1, m2};
                double k2 = 0;
                for (int b = 0; b < d; ++b) {
                    double s = 0;
                    for (int a = 0; a < d; ++a) s += g.Rinv[a * d + b] * m[a];
                    s *= 2.0 * kPi;
                    k2 += s * s;
                }
                const double kk = std::sqrt(k2);
                if (kk * g.rc > plan->c) continue;
                double den = 1;
                for (int i = 0; i < d; ++i) {
                    const double f = ph[i][std::abs(m[i])];
                    den *= f * f;
                }
                const double wv = plan->kt.what(kk * g.rc) / k2 / den;
                wmax = std::max(wmax, wv);
                if (kk < kmin) { kmin = kk; wlow = wv; }
            }
    return wlow > 0 ? wmax / wlow : 1.0;
}

// FP64 far-field weights for the half spectrum (Eq. (3.14)-(3.15a) with the window
// deconvolution of both NUFFT halves folded in); zero at m = 0 and on Nyquist planes
static std::vector<double> far_weights(pdmk_plan plan) {
    const int d = plan->d;
    const Geometry& g = plan->g;
    std::vector<double> ph[3];
    for (int i = 0; i < d; ++i) {
        ph[i].resize(g.M[i]);
        for (int j = 0; j < g.M[i]; ++j) {
            int m = j <= g.M[i] / 2 ? j : j - g.M[i];
            ph[i][j] = plan->wt.ft(double(m) / g.M[i]);
        }
    }
    const int Mh0 = g.M[0] / 2 + 1;
    std::vector<double> wt(size_t(plan->nhalf), 0.0);
    const int M2 = d == 3 ? g.M[2] : 1;
    for (int j2 = 0; j2 < M2; ++j2)
        for (int j1 = 0; j1 < g.M[1]; ++j1)
            for (int j0 = 0; j0 < Mh0; ++j0) {
                int jj[3] = {j0, j1, j2};
                int m[3] = {0, 0, 0};
                bool nyq = false, zero = true;
                for (int i = 0; i < d; ++i) {
                    int Mi = g.M[i];
                    if (jj[i] == Mi / 2) nyq = true;
                    m[i] = jj[i] < Mi / 2 ? jj[i] : jj[i] - Mi;
                    if (i == 0) m[i] = jj[i];
                    zero &= (m[i] == 0);
                }
                double val = 0;
                if (!nyq && !zero) {
                    double k2 = 0;
                    for (int b = 0; b < d; ++b) {
                        double s = 0;
                        for (int a = 0; a < d; ++a) s += g.Rinv[a * d + b] * m[a];
                        s *= 2.0 * kPi;
                        k2 += s * s;
                    }
                    double kk = std::sqrt(k2);
                    // only modes inside the active ball |k| <= c / r_c carry weight (Sec. 3.6);
                    // beyond it hat-w is below eps while the window deconvolution grows
                    double W0 = (kk * g.rc <= plan->c) ? plan->kt.what(kk * g.rc) / k2 : 0.0;
                    double den = g.V;
                    for (int i = 0; i < d; ++i) {
                        double f = ph[i][jj[i]];
                        den *= f * f;
                    }
                    val = W0 / den;
                }
                wt[(size_t(j2) * g.M[1] + j1) * Mh0 + j0] = val;
            }
    return wt;
}

// ---------------------------------------------------------------------------------------
// Work estimate of one cell and the partition of independent cells over ranks (host only).
// Cells of a batch share nothing, so the ranks of a multi-GPU run split the cells and
// exchange nothing on the data path.  The estimate counts flops per source of the three
// parts of an evaluation from the plan's parameters (no tree needed): near-field pairs
// ~ 3^d n_s per target at ~10 flops each, the plane-wave moments and leaf evaluation 4 p^d,
// spreading and interpolation 6 w^d, and the two transforms 10 prod(M) log2 prod(M).
extern "C" int pdmk_cell_work(int d, const double* L, double eps, const pdmk_opts* opts, int64_t n, double* work) {
    if (!L || !work || (d != 2 && d != 3) || n < 0) return PDMK_ERR_BAD_ARG;
    if (!(eps >= 1e-12 && eps <= 1e-2)) return PDMK_ERR_BAD_EPS;
    for (int i = 0; i < d * d; ++i)
        if (!std::isfinite(L[i])) return PDMK_ERR_NONFINITE;
    pdmk_opts o;
    if (opts) o = *opts; else pdmk_default_opts(&o);
    static std::mutex mu;
    static std::map<double, double> ccache;  // bandwidth c per eps (a root search)
    double c;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = ccache.find(eps);
        if (it == ccache.end()) it = ccache.emplace(eps, pswf_calibrate(eps)).first;
        c = it->second;
    }
    Geometry tmp, g;
    int rc = make_geometry(d, L, 1.0, c, &tmp);
    if (rc != PDMK_OK) return rc;
    double kappa;
    int ns;
    table1_defaults(d, eps, &tmp, L, &kappa, &ns);
    if (o.kappa > 0) kappa = o.kappa;
    if (o.n_s > 0) ns = o.n_s;
    rc = make_geometry(d, L, kappa, c, &g);
    if (rc != PDMK_OK) return rc;
    const int p = o.n_proxy > 0 ? o.n_proxy : ((int(std::ceil(c)) + 6 + 3) / 4) * 4;
    const int w = o.window_w > 0 ? o.window_w : int(std::ceil(2.0 * c / kPi - 1e-9)) + 2;
    double ncell = 1;
    for (int i = 0; i < d; ++i) ncell *= g.M[i];
    const double per_src = 10.0 * std::pow(3.0, d) * ns + 4.0 * std::pow(double(p), d) + 6.0 * std::pow(double(w), d);
    *work = double(n) * per_src + 10.0 * ncell * std::log2(std::max(ncell, 2.0));
    return PDMK_OK;
}

// Longest-processing-time assignment: cells in order of decreasing work (ties by index) go
// to the rank with the least work so far (ties to the lowest rank).  Deterministic, so every
// rank computes the same partition without communicating.
extern "C" int pdmk_partition_cells(int ncells, const double* work, int nranks, int* rank_of_cell) {
    if (ncells < 0 || nranks < 1 || (ncells > 0 && (!work || !rank_of_cell))) return PDMK_ERR_BAD_ARG;
    for (int c = 0; c < ncells; ++c)
        if (!std::isfinite(work[c]) || work[c] < 0) return PDMK_ERR_BAD_ARG;
    std::vector<int> ord(static_cast<size_t>(ncells));
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<double> load(static_cast<size_t>(nranks), 0.0);
    for (int c : ord) {
        int best = 0;
        for (int r = 1; r < nranks; ++r)
            if (load[r] < load[best]) best = r;
        rank_of_cell[c] = best;
        load[best] += work[c];
    }
    return PDMK_OK;
}

extern "C" int pdmk_kernel_table_eval(int d, double eps, int kind, double x, double* value) {
    if ((d != 2 && d != 3) || !value) return PDMK_ERR_BAD_ARG;
    if (!(eps >= 1e-12 && eps <= 1e-2)) return PDMK_ERR_BAD_EPS;
    // tables are cached per (d, eps): building one takes a few hundred milliseconds
    static std::mutex mu;
    static std::map<std::pair<int, double>, KernelTables> cache;
    KernelTables kt;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({d, eps});
        if (it == cache.end()) it = cache.emplace(std::make_pair(d, eps), make_kernel_tables(d, eps, 1e-15)).first;
        kt = it->second;
    }
    switch (kind) {
        case 0: {
            double t = x, s = t * t;
            if (!(t > 0 && t <= 1)) return PDMK_ERR_BAD_ARG;
            *value = (d == 3) ? (1.0 - t * kt.A.eval(s)) / (4 * kPi * t) : -std::log(s) / (4 * kPi) - kt.A.eval(s);
            return PDMK_OK;
        }
        case 1: {
            double t = x, s = t * t;
            if (!(t > 0 && t <= 1)) return PDMK_ERR_BAD_ARG;
            // dR/dt (scale-free): 3D -(1 - tA + tB)/(4 pi t^2); 2D -sqrt(1-s) B/(2 pi t)
            *value = (d == 3) ? -(1.0 - t * kt.A.eval(s) + t * kt.B.eval(s)) / (4 * kPi * s)
                              : -std::sqrt(std::max(1.0 - s, 0.0)) * kt.B.eval(s) / (2 * kPi * t);
            return PDMK_OK;
        }
        case 2: *value = kt.what(x); return PDMK_OK;
        case 3: *value = kt.psi.c; return PDMK_OK;
        case 4: *value = kt.self_coef; return PDMK_OK;
        case 5: *value = kt.rhat0; return PDMK_OK;
        case 6:
        case 7: {
            const int w = std::max(2, std::min(int(std::ceil(2.0 * kt.psi.c / kPi - 1e-9)) + 2, kMaxW));
            const WindowTables wt = make_window(w, kPi * w / 2.0, std::max(eps * 1e-5, 1e-15));
            if (kind == 6) {
                if (!(x >= 0 && x <= 1)) return PDMK_ERR_BAD_ARG;
                *value = wt.F.eval(x);
            } else {
                *value = wt.ft(x);
            }
            return PDMK_OK;
        }
        default: return PDMK_ERR_BAD_ARG;
    }
}

extern "C" // Chebyshev series sum_k c_k T_k(x) on [-1, 1] as monomials sum_k a_k x^k (long double
// recurrence T_{k+1} = 2 x T_k - T_{k-1}).  Returns sum |a_k| / max |f| on a grid: the factor
// by which Horner's rounding error can exceed Clenshaw's.
static double cheb_to_mono(const std::vector<double>& c, std::vector<double>* a) {
    const size_t n = c.size();
    std::vector<long double> tm1(n + 1, 0.0L), t0(n + 1, 0.0L), acc(n + 1, 0.0L);
    tm1[0] = 1.0L;  // T_0
    if (n > 0) for (size_t i = 0; i <= n; ++i) acc[i] += c[0] * tm1[i];
    if (n > 1) {
        t0[1] = 1.0L;  // T_1
        for (size_t i = 0; i <= n; ++i) acc[i] += c[1] * t0[i];
    }
    for (size_t k = 2; k < n; ++k) {
        std::vector<long double> t1(n + 1, 0.0L);
        for (size_t i = 0; i + 1 <= n; ++i) t1[i + 1] += 2.0L * t0[i];
        for (size_t i = 0; i <= n; ++i) t1[i] -= tm1[i];
        for (size_t i = 0; i <= n; ++i) acc[i] += c[k] * t1[i];
        tm1.swap(t0);
        t0.swap(t1);
    }
    a->assign(n, 0.0);
    double sa = 0;
    for (size_t i = 0; i < n; ++i) {
        (*a)[i] = double(acc[i]);
        sa += std::fabs((*a)[i]);
    }
    double fmax = 0;
    for (int g = 0; g <= 2000; ++g) {
        const double x = -1.0 + g / 1000.0;
        long double v = 0;
        for (size_t i = n; i-- > 0;) v = v * x + acc[i];
        fmax = std::max(fmax, std::fabs(double(v)));
    }
    return fmax > 0 ? sa / fmax : 1.0;
}

int pdmk_plan_create(int d, const double* L, double eps, const pdmk_opts* opts, pdmk_plan* out) {
    if (!out) return PDMK_ERR_BAD_ARG;
    *out = nullptr;
    if (!L || (d != 2 && d != 3)) return PDMK_ERR_BAD_ARG;
    if (!(eps >= 1e-12 && eps <= 1e-2)) return PDMK_ERR_BAD_EPS;
    for (int i = 0; i < d * d; ++i)
        if (!std::isfinite(L[i])) return PDMK_ERR_NONFINITE;
    pdmk_plan plan = new (std::nothrow) pdmk_plan_s();
    if (!plan) return PDMK_ERR_OOM;
    if (opts) plan->opts = *opts; else pdmk_default_opts(&plan->opts);
    if (plan->opts.precision != PDMK_FP64 && plan->opts.precision != PDMK_MIXED) {
        delete plan;
        return PDMK_ERR_BAD_ARG;
    }
    plan->d = d;
    plan->eps = eps;
    for (int i = 0; i < d * d; ++i) plan->Lc[i] = L[i];
    plan->stream = static_cast<cudaStream_t>(plan->opts.stream);
    plan->nsm = device_sms();
    plan->sum_blocks = 2 * plan->nsm;
    plan->pw.nsm = plan->nsm;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithFlags(&plan->ws, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&plan->ws_pw, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&plan->ws_near, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_s, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_pw, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_near, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        pdmk_plan_destroy(plan);
        return PDMK_ERR_CUDA;
    }
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    double fit_tol = mixed ? std::max(eps * 1e-3, 2e-9) : std::max(eps * 1e-4, 1e-15);
    plan->kt = make_kernel_tables(d, eps, fit_tol);
    plan->c = plan->kt.psi.c;
    double kappa;
    int ns;
    Geometry tmp;
    int rc = make_geometry(d, L, 1.0, plan->c, &tmp);
    if (rc != PDMK_OK) { delete plan; return rc; }
    table1_defaults(d, eps, &tmp, L, &kappa, &ns);
    plan->kappa = plan->opts.kappa > 0 ? plan->opts.kappa : kappa;
    plan->n_s = plan->opts.n_s > 0 ? plan->opts.n_s : ns;
    plan->max_depth = plan->opts.max_depth < 0 ? 30 : std::min(plan->opts.max_depth, 30);
    rc = make_geometry(d, L, plan->kappa, plan->c, &plan->g);
    if (rc != PDMK_OK) { delete plan; return rc; }
    if (plan->opts.root_mode == 0) make_periodic_root(&plan->g, plan->kappa);  // cubic cells
    // window width: ceil(2c/pi) makes the window's transform at the band edge equal its own
    // edge value; two more points keep the far-field gradient (a derivative) within eps too
    plan->w = plan->opts.window_w > 0 ? plan->opts.window_w : int(std::ceil(2.0 * plan->c / kPi - 1e-9)) + 2;
    plan->w = std::max(2, std::min(plan->w, kMaxW));
    plan->beta = kPi * plan->w / 2.0;  // window prolate bandwidth c_w
    plan->wt = make_window(plan->w, plan->beta, mixed ? 1e-9 : std::max(eps * 1e-5, 1e-15));
    // FP32 far field: oversample the grid (about 5 % per step) until the window
    // deconvolution amplifies grid rounding by at most 5e7 relative to the lowest mode; the
    // band edge then moves off the Nyquist index, where the window's transform is smallest.
    // Only strongly skewed cells need it (a 2D cell at 20 degrees: 3e15 before; the 60-degree
    // bench cell is at 2.5e7 with E_pot 2e-7 at eps 1e-6, and keeps its grid).
    if (mixed)
        for (int it = 0; it < 16 && far_amplification(plan) > 5e7; ++it)
            for (int i = 0; i < d; ++i) {
                // next even size >= 1.05 M with prime factors <= 7 (fast transform lengths)
                int M = 2 * int(std::ceil(0.525 * plan->g.M[i]));
                auto smooth = [](int v) {
                    for (int p : {2, 3, 5, 7})
                        while (v % p == 0) v /= p;
                    return v == 1;
                };
                while (!smooth(M)) M += 2;
                plan->g.M[i] = M;
            }
    size_bins(plan);
    // register-tile 3D spreading: FP32 tiles, cubic 8-cell bins and a compiled window width
    // (an FP64 tile of P^2 columns needs twice the registers and ran slower than the
    // shared-memory kernel on B300's FP64 pipe: 73 against 65 ms on the 4M-point cell)
    plan->spread_reg3d = d == 3 && mixed && plan->B[0] == 8 && plan->B[1] == 8 && plan->B[2] == 8 &&
                         (plan->w == 8 || plan->w == 13 || plan->w == 17);
    // near-field coefficients
    plan->cA = plan->kt.A.coef;
    plan->cB = plan->kt.B.coef;
    if (int(plan->cA.size()) > kMaxCheb) plan->cA.resize(kMaxCheb);
    if (int(plan->cB.size()) > kMaxCheb) plan->cB.resize(kMaxCheb);
    {
        // the warp near-field kernel takes the series as monomials when Horner is as
        // accurate as Clenshaw and the length has a compiled instance
        const double ampA = cheb_to_mono(plan->cA, &plan->mA), ampB = cheb_to_mono(plan->cB, &plan->mB);
        const int nmax = int(std::max(plan->cA.size(), plan->cB.size()));
        static const int kNH[] = {8, 10, 12, 14, 16, 20, 24};
        plan->near_nh = 0;
        if (ampA <= 4.0 && ampB <= 4.0)
            for (int nh : kNH)
                if (nmax <= nh) {
                    plan->near_nh = nh;
                    break;
                }
    }
    plan->cW = plan->wt.F.coef;
    plan->cWd = plan->wt.dF.coef;
    if (int(plan->cW.size()) > kMaxCheb) plan->cW.resize(kMaxCheb);
    if (int(plan->cWd.size()) > kMaxCheb) plan->cWd.resize(kMaxCheb);
    {
        // 2D FP32 far field with halo grids: compiled window widths, Horner as accurate as
        // Clenshaw, the halo no longer than the grid, per-warp halo copies fitting two CTAs
        // per SM
        const double ampW = cheb_to_mono(plan->cW, &plan->mW), ampWd = cheb_to_mono(plan->cWd, &plan->mWd);
        const int nh = plan->w == 8 ? 12 : plan->w == 13 ? 16 : plan->w == 17 ? 20 : 0;
        const int64_t Mp0 = plan->g.M[0] + plan->w - 1, Mp1 = plan->g.M[1] + plan->w - 1;
        plan->far_halo = d == 2 && mixed && nh > 0 && int(plan->cW.size()) <= nh && int(plan->cWd.size()) <= nh &&
                         ampW <= 4.0 && ampWd <= 4.0 && plan->w - 1 <= std::min(plan->g.M[0], plan->g.M[1]) &&
                         (8 * Mp0 * Mp1 + 16 * plan->w) * 4 <= 112 * 1024;
        // FP64 windows need longer series (eps-scaled fit): 24 terms cover eps >= 1e-9
        const int nh3 = plan->w == 8 ? 16 : plan->w == 13 ? 20 : plan->w == 17 ? 24 : 0;
        plan->far_warp3d = d == 3 && nh3 > 0 && int(plan->cW.size()) <= nh3 && int(plan->cWd.size()) <= nh3 &&
                           ampW <= 4.0 && ampWd <= 4.0 &&
                           plan->w - 1 <= std::min(plan->g.M[0], std::min(plan->g.M[1], plan->g.M[2]));
    }
    // plane-wave planning (proxy order, plane-wave counts, 1D operators)
    pw_plan_create(&plan->pw, d, eps, plan->c, plan->kt, plan->opts.n_proxy, plan->opts.n_pw, mixed);
    plan->pw.tensor_cores = plan->opts.tensor_cores == 0;
    plan->pw.pool = &plan->pool;
    plan->pw.wait_test = plan->opts.wait_test;
    // device: coefficient arrays, far weights, grid, spectrum, FFT plans
    const size_t ts = tsize(plan);
    int r;
#define PCHECK(x) do { r = (x); if (r != PDMK_OK) { pdmk_plan_destroy(plan); return r; } } while (0)
    {
        unsigned char* p = nullptr;
        auto coef_upload = [&](const std::vector<double>& src, void** dst) -> int {
            unsigned char* q = nullptr;
            int rr = dalloc(plan, plan->plan_allocs, &q, ts * kMaxCheb);
            if (rr != PDMK_OK) return rr;
            *dst = q;
            std::vector<unsigned char> buf(ts * kMaxCheb, 0);
            for (size_t k = 0; k < src.size() && k < size_t(kMaxCheb); ++k) {
                if (mixed) { float v = float(src[k]); std::memcpy(&buf[k * 4], &v, 4); }
                else std::memcpy(&buf[k * 8], &src[k], 8);
            }
            return upload(plan, *dst, buf);
        };
        PCHECK(coef_upload(plan->cA, &plan->d_coefA));
        PCHECK(coef_upload(plan->cB, &plan->d_coefB));
        PCHECK(coef_upload(plan->cW, &plan->d_coefW));
        PCHECK(coef_upload(plan->cWd, &plan->d_coefWd));
        PCHECK(coef_upload(plan->mW, &plan->d_monoW));
        PCHECK(coef_upload(plan->mWd, &plan->d_monoWd));
        PCHECK(dalloc(plan, plan->plan_allocs, &plan->d_weight, size_t(plan->nhalf)));
        std::vector<double> wt = far_weights(plan);
        PCHECK(upload(plan, plan->d_weight, wt));
        PCHECK(dalloc(plan, plan->plan_allocs, &p, ts * size_t(plan->ncell)));
        plan->d_grid = p;
        // the transforms and the k-space scaling run in FP64 except for 2D mixed plans:
        // rounding that enters before the scaling is amplified by the window deconvolution
        // near the band edge (a per-axis factor), and in 3D an FP32 transform's error
        // (~1e-7 log N of the grid norm) reached ~1e-6 of a far-field-dominated potential;
        // the 2D grids are small and two axes amplify less
        plan->fft32 = mixed && d == 2;
        if (mixed && !plan->fft32) {
            PCHECK(dalloc(plan, plan->plan_allocs, &p, sizeof(double) * size_t(plan->ncell)));
            plan->d_grid64 = p;
        } else {
            plan->d_grid64 = plan->d_grid;
        }
        PCHECK(dalloc(plan, plan->plan_allocs, &p, 2 * (plan->fft32 ? 4 : 8) * size_t(plan->nhalf)));
        plan->d_spec = p;
        PCHECK(dalloc(plan, plan->plan_allocs, &plan->d_qsums, 4));
        PCHECK(dalloc(plan, plan->plan_allocs, &plan->d_qsum_part, size_t(3 * plan->sum_blocks)));
        PCHECK(dalloc(plan, plan->plan_allocs, &plan->d_count, 2));
    }
    {
        const Geometry& g = plan->g;
        const cufftType tf = plan->fft32 ? CUFFT_R2C : CUFFT_D2Z, ti = plan->fft32 ? CUFFT_C2R : CUFFT_Z2D;
        cufftResult fr;
        if (d == 2) {
            fr = cufftPlan2d(&plan->fft_fwd, g.M[1], g.M[0], tf);
            if (fr == CUFFT_SUCCESS) fr = cufftPlan2d(&plan->fft_inv, g.M[1], g.M[0], ti);
        } else {
            fr = cufftPlan3d(&plan->fft_fwd, g.M[2], g.M[1], g.M[0], tf);
            if (fr == CUFFT_SUCCESS) fr = cufftPlan3d(&plan->fft_inv, g.M[2], g.M[1], g.M[0], ti);
        }
        if (fr != CUFFT_SUCCESS) {
            plan_set_msg(plan, "cufft plan failure");
            pdmk_plan_destroy(plan);
            return PDMK_ERR_CUDA;
        }
        plan->have_fft = true;
        cufftSetStream(plan->fft_fwd, plan->ws);
        cufftSetStream(plan->fft_inv, plan->ws);
    }
    if (cudaStreamSynchronize(plan->ws) != cudaSuccess) {
        pdmk_plan_destroy(plan);
        return PDMK_ERR_CUDA;
    }
#undef PCHECK
    *out = plan;
    return PDMK_OK;
}

static void drop_graph(pdmk_plan plan) {
    if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
    plan->gexec = nullptr;
    plan->g_pot = plan->g_grad = nullptr;
}

extern "C" void pdmk_plan_destroy(pdmk_plan plan) {
    if (!plan) return;
    if (plan->ws) cudaStreamSynchronize(plan->ws);
    drop_graph(plan);
    free_list(plan->src_allocs, &plan->device_bytes);
    free_list(plan->plan_allocs, &plan->device_bytes);
    free_list(plan->tree_keep, &plan->device_bytes);
    if (plan->tq_buf) cudaFree(plan->tq_buf);
    if (plan->h_stage) cudaFreeHost(plan->h_stage);
    pw_free(&plan->pw);
    plan->pool.trim();
    if (plan->have_fft) {
        cufftDestroy(plan->fft_fwd);
        cufftDestroy(plan->fft_inv);
    }
    if (plan->bl_have_fft) cufftDestroy(plan->bl_fft);
    for (auto e : plan->ev) cudaEventDestroy(e);
    if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
    if (plan->ev_join) cudaEventDestroy(plan->ev_join);
    if (plan->ev_s) cudaEventDestroy(plan->ev_s);
    if (plan->ev_pw) cudaEventDestroy(plan->ev_pw);
    if (plan->ev_near) cudaEventDestroy(plan->ev_near);
    if (plan->ws_pw) cudaStreamDestroy(plan->ws_pw);
    if (plan->ws_near) cudaStreamDestroy(plan->ws_near);
    if (plan->ws) cudaStreamDestroy(plan->ws);
    delete plan;
}

template <typename T>
static int gather_charges(pdmk_plan plan) {
    GatherArgs<T> a;
    a.q = plan->d_q_user;
    a.nsrc = plan->nimg;
    a.src_orig = plan->d_src_orig;
    a.src4 = static_cast<T*>(plan->d_src4);
    a.nspread = plan->nspread;
    a.spread_orig = plan->d_spread_orig;
    a.spread_dq = static_cast<T*>(plan->d_pt_dq);
    a.ntgt = plan->ntgt;
    a.tgt_orig = plan->d_tgt_orig;
    a.tgt4 = static_cast<T*>(plan->d_tgt4);
    a.q_tgt = plan->d_q_tgt;
    int64_t mx = std::max(plan->nimg, std::max(plan->nspread, plan->ntgt));
    int blocks = int(std::min<int64_t>((mx + 255) / 256, int64_t(plan->nsm) * 16));
    k_gather_charges<T><<<std::max(blocks, 1), 256, 0, plan->ws>>>(a);
    CK(cudaGetLastError());
    return PDMK_OK;
}

static int set_charges_device(pdmk_plan plan, bool check_neutral) {
    // deterministic two-stage sums over many SMs (FP64 on one SM would take ~0.2 ms)
    const int nb = int(std::max<int64_t>(1, std::min<int64_t>(plan->sum_blocks, (plan->n + 1023) / 1024)));
    k_charge_sums_part<<<nb, kSumThreads, 0, plan->ws>>>(plan->d_q_user, plan->n, plan->d_qsum_part);
    k_charge_sums_final<<<1, kSumThreads, 0, plan->ws>>>(plan->d_qsum_part, nb, plan->d_qsums);
    CK(cudaGetLastError());
    if (check_neutral) {
        double h[3];
        CK(cudaMemcpyAsync(h, plan->d_qsums, 3 * sizeof(double), cudaMemcpyDeviceToHost, plan->ws));
        CK(cudaStreamSynchronize(plan->ws));
        if (h[2] > 0) return PDMK_ERR_NONFINITE;
        if (plan->opts.neutrality == 0 && std::fabs(h[0]) > 1e-12 * h[1]) return PDMK_ERR_NON_NEUTRAL;
    }
    int r = plan->opts.precision == PDMK_MIXED ? gather_charges<float>(plan) : gather_charges<double>(plan);
    if (r != PDMK_OK) return r;
    return pw_set_charges(&plan->pw, plan->ws);
}

// the caller-frame lattice vector L n of a direct-list shift code (zero without a periodic root)
static void lattice_shift(const Geometry& g, int code, double* out) {
    const int d = g.d;
    int n[3];
    shift_of(code, n);
    double v[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) v[i] += g.R[i * d + k] * n[k];
    for (int i = 0; i < d; ++i) {
        out[i] = 0;
        for (int k = 0; k < d; ++k) out[i] += g.Q[k * d + i] * v[k];
    }
}

// Sources (n_src, charges q) and, if m > 0, separate targets x (m points): the plan is built
// on the union, the targets being points of charge 0 (they add nothing to any stage and have
// no self term), and the evaluation writes the m target outputs only.
// ---- source set-up -------------------------------------------------------------------
// The set-up runs on the host (build_tree and the per-point passes below) or on the device
// (gpu_build.cu); both produce the same tree, order and records, bit for bit.  The per-box
// passes (direct lists, near-field entries, spreading subproblems, plane-wave layouts) run on
// the host in both.

// near-field leaf descriptors and direct-list entries (per box)
// (with_entries false: the entries are left to the device, gpu_near_entries)
static void near_layout(pdmk_plan plan, const Tree& tree, const DirectLists& dl, const std::vector<double>& Cu,
                        std::vector<TLeaf>* tl_out, std::vector<int2>* ent_out, std::vector<unsigned char>* ent_sh_out,
                        std::vector<float>* ent_shlo_out, std::vector<int>* bsb_out, std::vector<int>* bsc_out,
                        bool with_entries) {
    const int d = plan->d;
    const Geometry& g = plan->g;
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const size_t ts = tsize(plan);
    const int nb = int(tree.level.size());
    auto put = [&](std::vector<unsigned char>& buf, size_t idx, double v) {
        if (mixed) { float f = float(v); std::memcpy(&buf[idx * 4], &f, 4); }
        else std::memcpy(&buf[idx * 8], &v, 8);
    };
    auto to_tree = [&](const double* v, double* out) {  // Q v
        for (int i = 0; i < d; ++i) {
            double s = 0;
            for (int k = 0; k < d; ++k) s += g.Q[i * d + k] * v[k];
            out[i] = s;
        }
    };
    std::vector<TLeaf>& tl = *tl_out;
    tl.assign(dl.tleaf.size(), TLeaf{});
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < int64_t(dl.tleaf.size()); ++k) {
        int b = dl.tleaf[k];
        tl[k].tgt_begin = int(tree.tgt_begin[b]);
        tl[k].tgt_count = int(tree.tgt_end[b] - tree.tgt_begin[b]);
        tl[k].list_begin = int(dl.list_begin[k]);
        tl[k].list_count = int(dl.list_begin[k + 1] - dl.list_begin[k]);
        tl[k].level = tree.level[b];
        tl[k].box = b;
        tl[k].pad0 = tl[k].pad1 = 0;
    }
    std::vector<int>& bsb = *bsb_out;
    std::vector<int>& bsc = *bsc_out;
    bsb.resize(nb);
    bsc.resize(nb);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nb; ++b) {
        bsb[b] = int(tree.src_begin[b]);
        bsc[b] = int(tree.src_end[b] - tree.src_begin[b]);
    }
    // per direct-list entry: source range and the source leaf centre's shift into the target
    // leaf's frame (FP64 difference, then hi / lo in T)
    std::vector<int2>& ent = *ent_out;
    std::vector<unsigned char>& ent_sh = *ent_sh_out;
    std::vector<float>& ent_shlo = *ent_shlo_out;
    ent.assign(with_entries ? dl.list.size() : 0, int2{0, 0});
    ent_sh.assign(with_entries ? dl.list.size() * 4 * ts : 0, 0);
    ent_shlo.assign(with_entries && mixed ? dl.list.size() * 4 : 0, 0.0f);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < (with_entries ? int64_t(dl.tleaf.size()) : 0); ++k) {
        const int tb = dl.tleaf[k];
        for (int64_t e = dl.list_begin[k]; e < dl.list_begin[k + 1]; ++e) {
            const int sb = dl.list[e];
            ent[e] = make_int2(bsb[sb], bsc[sb]);
            double du[3] = {0, 0, 0}, sht[3], Ln[3] = {0, 0, 0};
            lattice_shift(g, dl.shift[e], Ln);
            for (int a = 0; a < d; ++a) du[a] = Cu[size_t(sb) * d + a] + Ln[a] - Cu[size_t(tb) * d + a];
            to_tree(du, sht);
            for (int a = 0; a < d; ++a) {
                const double sh = sht[a];
                put(ent_sh, size_t(e) * 4 + a, sh);
                if (mixed) ent_shlo[size_t(e) * 4 + a] = float(sh - double(float(sh)));
            }
        }
    }
    // the warp near-field kernel computes 32 targets at a time: a leaf with more targets
    // becomes several descriptors over the same direct list (one warp each, so leaves of a
    // few hundred targets do not leave the grid short of warps; every target is still summed
    // by one lane in the same order). Descriptors are taken in order of decreasing pair
    // count (the long ones start first).
    if (plan->near_nh > 0) {
        std::vector<TLeaf> split;
        split.reserve(tl.size() * 2);
        for (const TLeaf& L : tl)
            for (int t0 = 0; t0 < std::max(L.tgt_count, 1); t0 += 32) {
                TLeaf c = L;
                c.tgt_begin = L.tgt_begin + t0;
                c.tgt_count = std::min(32, L.tgt_count - t0);
                split.push_back(c);
            }
        tl.swap(split);
    }
    // (decreasing cost, then increasing index: the order a stable sort by cost gives)
    std::vector<std::pair<int64_t, int64_t>> key(tl.size());
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < int64_t(tl.size()); ++k) {
        int64_t ns = 0;
        for (int e = tl[k].list_begin; e < tl[k].list_begin + tl[k].list_count; ++e) ns += bsc[dl.list[e]];
        key[size_t(k)] = {-ns * int64_t(tl[k].tgt_count), k};
    }
    sort_pairs_parallel(&key);
    std::vector<TLeaf> tl2(tl.size());
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < int64_t(key.size()); ++k) tl2[size_t(k)] = tl[size_t(key[size_t(k)].second)];
    tl.swap(tl2);
}

// spreading subproblems: chunks of at most max_pts points of one bin (one spreading block
// each; in 3D the clustered bins hold most points, so smaller chunks give the grid enough
// blocks), from the points per bin in bin order
static void spread_subproblems(pdmk_plan plan, const std::vector<int64_t>& bin_count, std::vector<int4>* subs,
                               std::vector<int>* bin_sub_begin) {
    const int max_pts = plan->spread_reg3d ? 1024 : (plan->d == 3 ? 128 : 512);
    subs->clear();
    bin_sub_begin->assign(size_t(plan->nbins_tot) + 1, 0);
    int64_t k = 0;
    for (int bin = 0; bin < plan->nbins_tot; ++bin) {
        (*bin_sub_begin)[bin] = int(subs->size());
        const int64_t k0 = k;
        k += bin_count[size_t(bin)];
        for (int64_t s0 = k0; s0 < k; s0 += max_pts)
            subs->push_back(make_int4(bin, int(s0), int(std::min<int64_t>(max_pts, k - s0)), 0));
    }
    (*bin_sub_begin)[plan->nbins_tot] = int(subs->size());
}

// drop the previous set-up's buffers and graph
static void release_sources(pdmk_plan plan) {
    // the old arrays are reused, not freed: wait for all work that may still read them (the
    // implicit synchronisation of cudaFree)
    cudaDeviceSynchronize();
    drop_graph(plan);
    plan->evals_since_setup = 0;
    for (auto& a : plan->src_allocs) plan->pool.put(a.first, a.second);  // offered to the next set-up
    plan->src_allocs.clear();
    for (auto& a : plan->tree_keep) plan->pool.put(a.first, a.second);
    plan->tree_keep.clear();
    plan->tree_dev = GpuBuild();
    plan->host_tree = true;
    plan->d_adj = nullptr;
    if (plan->tq_buf) cudaFree(plan->tq_buf);
    plan->tq_buf = nullptr;
    plan->tq_cap = 0;
    pw_free_sources(&plan->pw);
    plan->d_u_keep = nullptr;
    plan->d_y_keep = nullptr;
    plan->d_src_disp = nullptr;
    plan->d_tgt_of_keep = nullptr;
    plan->host_copies = true;
}

// the per-point device arrays of a set-up (sizes from the plan's counts)
static int alloc_sources(pdmk_plan plan, size_t nleafdesc, size_t nlist) {
    auto& L = plan->src_allocs;
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const size_t ts = tsize(plan);
    const int d = plan->d;
    const int64_t n = plan->n;
    DALLOC(L, plan->d_src4, unsigned char, size_t(plan->nimg) * 4 * ts);
    DALLOC(L, plan->d_src_orig, int, plan->nimg);
    DALLOC(L, plan->d_tgt4, unsigned char, size_t(plan->ntgt) * 4 * ts);
    DALLOC(L, plan->d_tgt_orig, int, plan->ntgt);
    DALLOC(L, plan->d_src_lo, float, mixed ? size_t(plan->nimg) * 4 : 0);
    DALLOC(L, plan->d_tgt_lo, float, mixed ? size_t(plan->ntgt) * 4 : 0);
    DALLOC(L, plan->d_q_tgt, double, plan->ntgt);
    DALLOC(L, plan->d_self_w, double, plan->ntgt);
    DALLOC(L, plan->d_tleaf, TLeaf, nleafdesc);
    DALLOC(L, plan->d_list, int, nlist);
    DALLOC(L, plan->d_ent, int2, nlist);
    DALLOC(L, plan->d_ent_sh, unsigned char, nlist * 4 * ts);
    DALLOC(L, plan->d_ent_shlo, float, mixed ? nlist * 4 : 0);
    DALLOC(L, plan->d_box_src_begin, int, plan->nbox);
    DALLOC(L, plan->d_box_src_count, int, plan->nbox);
    DALLOC(L, plan->d_box_center, double, size_t(plan->nbox) * d);
    DALLOC(L, plan->d_pt_g0, int4, n);
    DALLOC(L, plan->d_pt_dq, unsigned char, size_t(n) * 4 * ts);
    DALLOC(L, plan->d_spread_orig, int, n);
    DALLOC(L, plan->d_t_g0, int4, plan->ntgt);
    DALLOC(L, plan->d_t_dq, unsigned char, size_t(plan->ntgt) * 4 * ts);
    DALLOC(L, plan->d_pot_near, double, plan->ntgt);
    DALLOC(L, plan->d_grad_near, double, plan->ntgt * d);
    DALLOC(L, plan->d_pot_far, double, plan->ntgt);
    DALLOC(L, plan->d_gradu_far, double, plan->ntgt * d);
    DALLOC(L, plan->d_q_user, double, n);
    DALLOC(L, plan->d_pot_out, double, n);
    DALLOC(L, plan->d_grad_out, double, n * d);
    return PDMK_OK;
}

// the spreading subproblems and their scratch (plan->nsub set)
static int alloc_subs(pdmk_plan plan, size_t nsub) {
    auto& L = plan->src_allocs;
    DALLOC(L, plan->d_sub, int4, nsub);
    DALLOC(L, plan->d_bin_sub_begin, int, size_t(plan->nbins_tot) + 1);
    DALLOC(L, plan->d_slab, unsigned char, slab_bytes(plan));
    return PDMK_OK;
}

// plan facts after a set-up
static void finish_info(pdmk_plan plan, const BuildStats& st, int64_t pairs, int64_t n_src, int64_t m) {
    const Geometry& g = plan->g;
    const int d = plan->d;
    pdmk_info& I = plan->info;
    std::memset(&I, 0, sizeof(I));
    I.d = d; I.eps = plan->eps; I.c = plan->c; I.rc = g.rc; I.V = g.V; I.kappa = plan->kappa;
    I.n_s = plan->n_s; I.window_w = plan->w; I.n_proxy = plan->pw.p; I.n_pw = plan->pw.K;
    I.precision = plan->opts.precision;
    for (int i = 0; i < 3; ++i) { I.M[i] = g.M[i]; I.nroot[i] = i < d ? g.nroot[i] : 1; }
    I.n = plan->n; I.n_images = plan->nimg; I.nboxes = st.nboxes; I.nleaves = st.nleaves; I.depth = st.depth;
    I.ntarget_leaves = plan->ntleaf; I.near_pairs = pairs;
    I.n_pw_boxes_out = plan->pw.nout; I.n_pw_boxes_in = plan->pw.nin;
    I.pw_moment_sources = plan->pw.active ? plan->pw.moment_sources : 0;
    I.pw_merge_parents = plan->pw.active ? plan->pw.merge_parents : 0;
    I.pw_down_parents = plan->pw.active ? plan->pw.down_parents : 0;
    I.pw_eval_targets = plan->pw.active ? plan->pw.eval_targets : 0;
    I.spread_subproblems = plan->nsub;
    plan->count_pending = plan->opts.profile != 0;
    plan->n_src = n_src;
    plan->out_first = m > 0 ? n_src : 0;
    plan->n_out = m > 0 ? m : n_src;
    I.n = n_src;
    I.n_targets = plan->n_out;
}

// the host copies of a device set-up (used by evaluations at new targets and Bloch sums)
static int ensure_host_copies(pdmk_plan plan) {
    if (!plan->host_tree) {
        CK(cudaStreamSynchronize(plan->ws));
        std::string msg;
        const int r = gpu_tree_download(plan->tree_dev, &plan->h_tree, plan->ws, &msg);
        if (r != PDMK_OK) {
            plan->msg = msg;
            return r;
        }
        const Tree& t = plan->h_tree;
        const int d = plan->d;
        const int nb = int(t.level.size());
        plan->h_Cu.resize(size_t(nb) * d);
#pragma omp parallel for schedule(static)
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < d; ++i) {
                double sum = 0;
                for (int k = 0; k < d; ++k) sum += plan->g.Q[k * d + i] * t.center[size_t(b) * d + k];
                plan->h_Cu[size_t(b) * d + i] = sum;
            }
        plan->host_tree = true;
    }
    if (plan->host_copies) return PDMK_OK;
    const int d = plan->d;
    CK(cudaStreamSynchronize(plan->ws));
    plan->h_u.resize(size_t(plan->n) * d);
    plan->h_y.resize(size_t(plan->n) * d);
    plan->h_src_disp.resize(size_t(plan->nimg) * d);
    std::vector<int> so(size_t(plan->nimg)), tof(size_t(plan->ntgt));
    CK(cudaMemcpy(plan->h_u.data(), plan->d_u_keep, plan->h_u.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(plan->h_y.data(), plan->d_y_keep, plan->h_y.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(plan->h_src_disp.data(), plan->d_src_disp, plan->h_src_disp.size() * sizeof(double),
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(so.data(), plan->d_src_orig, so.size() * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tof.data(), plan->d_tgt_of_keep, tof.size() * sizeof(int), cudaMemcpyDeviceToHost));
    plan->h_src_orig.assign(so.begin(), so.end());
    plan->h_src_is_orig.assign(size_t(plan->nimg), 0);
    for (int j : tof) plan->h_src_is_orig[size_t(j)] = 1;
    plan->host_copies = true;
    return PDMK_OK;
}

static int set_points_host(pdmk_plan plan, int64_t n_src, const double* y, const double* q, int64_t m,
                           const double* x, int where);
static int set_points_device(pdmk_plan plan, int64_t n_src, const double* y, const double* q, int64_t m,
                             const double* x, int where);

// every array a set-up leaves, for the comparison of the two builds (name, bytes)
static int setup_snapshot(pdmk_plan plan, std::vector<std::pair<std::string, std::vector<unsigned char>>>* out) {
    out->clear();
    CK(cudaStreamSynchronize(plan->ws));
    const size_t ts = tsize(plan);
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const int d = plan->d;
    auto dev = [&](const char* name, const void* p, size_t bytes) -> int {
        std::vector<unsigned char> v(bytes);
        if (bytes) CK(cudaMemcpy(v.data(), p, bytes, cudaMemcpyDeviceToHost));
        out->push_back({name, std::move(v)});
        return PDMK_OK;
    };
    auto host = [&](const char* name, const void* p, size_t bytes) {
        std::vector<unsigned char> v(bytes);
        if (bytes) std::memcpy(v.data(), p, bytes);
        out->push_back({name, std::move(v)});
    };
    int64_t counts[8] = {plan->n, plan->nimg, plan->ntgt, plan->nspread, plan->nbox, plan->ntleaf, plan->nsub,
                         plan->nnear};
    host("counts", counts, sizeof(counts));
    int r;
    if ((r = dev("list", plan->d_list, size_t(plan->nlist) * 4))) return r;
    if ((r = dev("ent", plan->d_ent, size_t(plan->nlist) * 8))) return r;
    if ((r = dev("ent_sh", plan->d_ent_sh, size_t(plan->nlist) * 4 * ts))) return r;
    if (mixed && (r = dev("ent_shlo", plan->d_ent_shlo, size_t(plan->nlist) * 16))) return r;
    if ((r = dev("src4", plan->d_src4, size_t(plan->nimg) * 4 * ts))) return r;
    if ((r = dev("src_orig", plan->d_src_orig, size_t(plan->nimg) * 4))) return r;
    if ((r = dev("tgt4", plan->d_tgt4, size_t(plan->ntgt) * 4 * ts))) return r;
    if ((r = dev("tgt_orig", plan->d_tgt_orig, size_t(plan->ntgt) * 4))) return r;
    if (mixed) {
        if ((r = dev("src_lo", plan->d_src_lo, size_t(plan->nimg) * 16))) return r;
        if ((r = dev("tgt_lo", plan->d_tgt_lo, size_t(plan->ntgt) * 16))) return r;
    }
    if ((r = dev("self_w", plan->d_self_w, size_t(plan->ntgt) * 8))) return r;
    if ((r = dev("tleaf", plan->d_tleaf, size_t(plan->nnear) * sizeof(TLeaf)))) return r;
    if ((r = dev("box_src_begin", plan->d_box_src_begin, size_t(plan->nbox) * 4))) return r;
    if ((r = dev("box_src_count", plan->d_box_src_count, size_t(plan->nbox) * 4))) return r;
    if ((r = dev("box_center", plan->d_box_center, size_t(plan->nbox) * d * 8))) return r;
    if ((r = dev("pt_g0", plan->d_pt_g0, size_t(plan->nspread) * 16))) return r;
    if ((r = dev("pt_dq", plan->d_pt_dq, size_t(plan->nspread) * 4 * ts))) return r;
    if ((r = dev("spread_orig", plan->d_spread_orig, size_t(plan->nspread) * 4))) return r;
    if ((r = dev("sub", plan->d_sub, size_t(plan->nsub) * 16))) return r;
    if ((r = dev("bin_sub_begin", plan->d_bin_sub_begin, size_t(plan->nbins_tot + 1) * 4))) return r;
    if ((r = dev("t_g0", plan->d_t_g0, size_t(plan->ntgt) * 16))) return r;
    if ((r = dev("t_dq", plan->d_t_dq, size_t(plan->ntgt) * 4 * ts))) return r;
    if ((r = dev("q_user", plan->d_q_user, size_t(plan->n) * 8))) return r;
    if ((r = ensure_host_copies(plan))) return r;
    const Tree& t = plan->h_tree;
    host("tree.level_start", t.level_start.data(), t.level_start.size() * 4);
    host("tree.level", t.level.data(), t.level.size() * 4);
    host("tree.coord", t.coord.data(), t.coord.size() * 8);
    host("tree.parent", t.parent.data(), t.parent.size() * 4);
    host("tree.child0", t.child0.data(), t.child0.size() * 4);
    host("tree.src_begin", t.src_begin.data(), t.src_begin.size() * 8);
    host("tree.src_end", t.src_end.data(), t.src_end.size() * 8);
    host("tree.tgt_begin", t.tgt_begin.data(), t.tgt_begin.size() * 8);
    host("tree.tgt_end", t.tgt_end.data(), t.tgt_end.size() * 8);
    host("tree.colleague", t.colleague.data(), t.colleague.size() * 4);
    host("tree.center", t.center.data(), t.center.size() * 8);
    if ((r = ensure_host_copies(plan))) return r;
    host("h_u", plan->h_u.data(), plan->h_u.size() * 8);
    host("h_src_orig", plan->h_src_orig.data(), plan->h_src_orig.size() * 8);
    host("h_src_is_orig", plan->h_src_is_orig.data(), plan->h_src_is_orig.size());
    host("h_Cu", plan->h_Cu.data(), plan->h_Cu.size() * 8);
    host("h_y", plan->h_y.data(), plan->h_y.size() * 8);
    host("h_src_disp", plan->h_src_disp.data(), plan->h_src_disp.size() * 8);
    int64_t facts[8] = {plan->info.n_images, plan->info.nboxes, plan->info.nleaves, plan->info.depth,
                        plan->info.near_pairs, plan->info.pw_merge_parents, plan->info.pw_down_parents,
                        plan->info.n_pw_boxes_in};
    host("info", facts, sizeof(facts));
    pw_layout_snapshot(&plan->pw, out);
    return PDMK_OK;
}

static int set_points(pdmk_plan plan, int64_t n_src, const double* y, const double* q, int64_t m, const double* x,
                      int where) {
    if (!plan || n_src < 0 || m < 0 || (n_src > 0 && (!y || !q)) || (m > 0 && !x)) return PDMK_ERR_BAD_ARG;
    const int64_t n = n_src + m;
    if (n >= (int64_t(1) << 30)) return PDMK_ERR_TOO_LARGE;
    plan->ready = false;
    plan->setup_names.clear();
    plan->setup_ms.clear();
    plan->setup_device = false;
    const int mode = plan->opts.build_mode;
    if (mode == 1 || n == 0) return set_points_host(plan, n_src, y, q, m, x, where);
    if (mode == 3) {
        // both builds, compared array by array (a check of the device build)
        int r = set_points_host(plan, n_src, y, q, m, x, where);
        if (r != PDMK_OK) return r;
        std::vector<std::pair<std::string, std::vector<unsigned char>>> a, b;
        if ((r = setup_snapshot(plan, &a))) return r;
        plan->ready = false;
        r = set_points_device(plan, n_src, y, q, m, x, where);
        if (r == kGpuBuildUnsupported) {
            plan_set_msg(plan, "device set-up unsupported for these inputs (host build kept)");
            return set_points_host(plan, n_src, y, q, m, x, where);
        }
        if (r != PDMK_OK) return r;
        if ((r = setup_snapshot(plan, &b))) return r;
        for (size_t k = 0; k < a.size() && k < b.size(); ++k)
            if (a[k].first != b[k].first || a[k].second != b[k].second) {
                plan->ready = false;
                std::string msg = "device and host set-up differ in " + a[k].first + " (" +
                                  std::to_string(a[k].second.size()) + " vs " + std::to_string(b[k].second.size()) +
                                  " bytes)";
                for (size_t i = 0; i < std::min(a[k].second.size(), b[k].second.size()); ++i)
                    if (a[k].second[i] != b[k].second[i]) {
                        msg += ", first at byte " + std::to_string(i);
                        break;
                    }
                plan->msg = msg;
                return PDMK_ERR_INTERNAL;
            }
        if (a.size() != b.size()) {
            plan->ready = false;
            plan_set_msg(plan, "device and host set-up differ in their array lists");
            return PDMK_ERR_INTERNAL;
        }
        plan->msg = "device and host set-up identical";
        return PDMK_OK;
    }
    int r = set_points_device(plan, n_src, y, q, m, x, where);
    if (r == kGpuBuildUnsupported) {
        if (mode == 2) {
            plan_set_msg(plan, "device set-up unsupported for these inputs");
            return PDMK_ERR_TOO_LARGE;
        }
        plan->setup_names.clear();
        plan->setup_ms.clear();
        return set_points_host(plan, n_src, y, q, m, x, where);
    }
    return r;
}

static int set_points_host(pdmk_plan plan, int64_t n_src, const double* y, const double* q, int64_t m,
                           const double* x, int where) {
    struct TrimOnReturn {  // the spares this set-up did not take are freed on every return
        DevicePool* pool;
        ~TrimOnReturn() { pool->trim(); }
    } trim_on_return{&plan->pool};
    const int64_t n = n_src + m;
    const int d = plan->d;
    auto clk = std::chrono::steady_clock::now();
    auto lap = [&](const char* name) {
        const auto now = std::chrono::steady_clock::now();
        plan->setup_names.push_back(name);
        plan->setup_ms.push_back(std::chrono::duration<double, std::milli>(now - clk).count());
        clk = now;
    };
    std::vector<double> hy(size_t(n) * d), hq(static_cast<size_t>(n), 0.0);
    if (n_src > 0 || m > 0) {
        if (where == PDMK_DEVICE) {
            CK(cudaStreamSynchronize(plan->stream));
            if (n_src > 0) {
                CK(cudaMemcpy(hy.data(), y, size_t(n_src) * d * sizeof(double), cudaMemcpyDeviceToHost));
                CK(cudaMemcpy(hq.data(), q, size_t(n_src) * sizeof(double), cudaMemcpyDeviceToHost));
            }
            if (m > 0)
                CK(cudaMemcpy(hy.data() + size_t(n_src) * d, x, size_t(m) * d * sizeof(double),
                              cudaMemcpyDeviceToHost));
        } else {
            if (n_src > 0) {
                std::memcpy(hy.data(), y, size_t(n_src) * d * sizeof(double));
                std::memcpy(hq.data(), q, size_t(n_src) * sizeof(double));
            }
            if (m > 0) std::memcpy(hy.data() + size_t(n_src) * d, x, size_t(m) * d * sizeof(double));
        }
    }
    double qs = 0, qa = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int a = 0; a < d; ++a)
            if (!std::isfinite(hy[j * d + a])) return PDMK_ERR_NONFINITE;
        if (!std::isfinite(hq[j])) return PDMK_ERR_NONFINITE;
        qs += hq[j];
        qa += std::fabs(hq[j]);
    }
    if (plan->opts.neutrality == 0 && std::fabs(qs) > 1e-12 * qa) return PDMK_ERR_NON_NEUTRAL;
    const Geometry& g = plan->g;
    // orient, then fractional coordinates wrapped into [0, 1)
    std::vector<double> u(size_t(n) * d);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        double xo[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) xo[i] += g.Q[i * d + k] * hy[j * d + k];
        for (int i = 0; i < d; ++i) {
            double s = 0;
            for (int k = 0; k < d; ++k) s += g.Rinv[i * d + k] * xo[k];
            s -= std::floor(s);
            if (s >= 1.0) s = 0.0;
            u[j * d + i] = s;
        }
    }
    lap("read_check_orient");
    Tree tree;
    SortedSources ss;
    BuildStats st;
    const int maxd = pw_supported(&plan->pw) ? plan->max_depth : 0;
    int rc = build_tree(g, n, u.data(), plan->n_s, maxd, &tree, &ss, &st);
    if (rc != PDMK_OK) return rc;
    for (int k = 0; k < 6; ++k) {
        plan->setup_names.push_back(kBuildPhases[k]);
        plan->setup_ms.push_back(st.phase_ms[k]);
    }
    clk = std::chrono::steady_clock::now();
    DirectLists dl;
    int64_t pairs = 0;
    build_direct_lists(tree, &dl, &pairs);
    lap("direct_lists");
    // ---- release old buffers, allocate new ----
    release_sources(plan);
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const size_t ts = tsize(plan);
    plan->n = n;
    plan->nimg = st.n_images;
    plan->ntgt = int64_t(ss.tgt_of.size());
    plan->nbox = st.nboxes;
    plan->ntleaf = int(dl.tleaf.size());
    auto put = [&](std::vector<unsigned char>& buf, size_t idx, double v) {
        if (mixed) { float f = float(v); std::memcpy(&buf[idx * 4], &f, 4); }
        else std::memcpy(&buf[idx * 8], &v, 8);
    };
    // leaf of every sorted source
    std::vector<int> leaf_of(size_t(plan->nimg), -1);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < st.nboxes; ++b)
        if (tree.is_leaf(b))
            for (int64_t j = tree.src_begin[b]; j < tree.src_end[b]; ++j) leaf_of[j] = b;
    // Leaf-relative coordinates, taken in the caller's frame.  Two nearby inputs differ
    // exactly there, while their oriented, wrapped copies (ss.pos) carry roundings of the
    // size of the cell's coordinates, which a pair 1e-4 of the cell apart would see at
    // 1e-11.  So every leaf gets a caller-frame centre C_b = Q^T c_b (any fixed double
    // vector serves), a copy of source o shifted by the lattice vector R m (tree frame) gets
    //   rel = Q (y_o - Q^T (c_b - R m)),   which is y_o - C_b rotated when m = 0,
    // and the leaf-to-leaf shifts of the direct lists are Q (C_s - C_t): for originals the
    // pair displacement rel_t - rel_s - sh is Q (y_t - y_s) up to roundings of leaf-sized
    // terms.  Pairs with an image keep the rounding of the lattice shift itself.
    auto to_user = [&](const double* v, double* out) {  // Q^T v
        for (int i = 0; i < d; ++i) {
            double s = 0;
            for (int k = 0; k < d; ++k) s += g.Q[k * d + i] * v[k];
            out[i] = s;
        }
    };
    auto to_tree = [&](const double* v, double* out) {  // Q v
        for (int i = 0; i < d; ++i) {
            double s = 0;
            for (int k = 0; k < d; ++k) s += g.Q[i * d + k] * v[k];
            out[i] = s;
        }
    };
    std::vector<double> Cu(size_t(st.nboxes) * d);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < st.nboxes; ++b) to_user(&tree.center[size_t(b) * d], &Cu[size_t(b) * d]);
    std::vector<double> relv(size_t(plan->nimg) * d);
    std::vector<double> src_disp(size_t(plan->nimg) * d, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < plan->nimg; ++j) {
        const int b = leaf_of[j];
        const int64_t o = ss.orig[j];
        double yo[3] = {0, 0, 0}, xo[3], m[3], D[3], E[3], du[3];
        for (int a = 0; a < d; ++a) yo[a] = hy[size_t(o) * d + a];
        to_tree(yo, xo);
        bool shifted = false;
        for (int i = 0; i < d; ++i) {
            double f = 0;
            for (int k = 0; k < d; ++k) f += g.Rinv[i * d + k] * (ss.pos[j * d + k] - xo[k]);
            m[i] = std::nearbyint(f);
            shifted |= m[i] != 0.0;
        }
        if (shifted) {
            double Rm[3] = {0, 0, 0};
            for (int i = 0; i < d; ++i) {
                double s = 0;
                for (int k = 0; k < d; ++k) s += g.R[i * d + k] * m[k];
                Rm[i] = s;
                D[i] = tree.center[size_t(b) * d + i] - s;
            }
            to_user(D, E);
            to_user(Rm, &src_disp[size_t(j) * d]);
        } else {
            for (int i = 0; i < d; ++i) E[i] = Cu[size_t(b) * d + i];
        }
        for (int a = 0; a < d; ++a) du[a] = yo[a] - E[a];
        to_tree(du, &relv[size_t(j) * d]);
    }
    lap("leaf_relative_coordinates");
    // sorted sources: coordinates relative to their leaf centre (FP64, then T)
    std::vector<unsigned char> src4(size_t(plan->nimg) * 4 * ts, 0);
    std::vector<int> src_orig(size_t(plan->nimg));
    std::vector<float> src_lo(mixed ? size_t(plan->nimg) * 4 : 0, 0.0f);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < plan->nimg; ++j) {
        for (int a = 0; a < d; ++a) {
            const double rel = relv[size_t(j) * d + a];
            put(src4, size_t(j) * 4 + a, rel);
            if (mixed) src_lo[size_t(j) * 4 + a] = float(rel - double(float(rel)));
        }
        src_orig[j] = int(ss.orig[j]);
    }
    // targets (the originals, in sorted order)
    std::vector<unsigned char> tgt4(size_t(plan->ntgt) * 4 * ts, 0);
    std::vector<int> tgt_orig(size_t(plan->ntgt));
    std::vector<double> self_w(size_t(plan->ntgt));
    std::vector<int> tgt_leaf(size_t(plan->ntgt));
    std::vector<float> tgt_lo(mixed ? size_t(plan->ntgt) * 4 : 0, 0.0f);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < plan->ntgt; ++t) {
        int64_t j = ss.tgt_of[t];
        int b = leaf_of[j];
        tgt_leaf[t] = b;
        for (int a = 0; a < d; ++a) {
            const double rel = relv[size_t(j) * d + a];
            put(tgt4, size_t(t) * 4 + a, rel);
            if (mixed) tgt_lo[size_t(t) * 4 + a] = float(rel - double(float(rel)));
        }
        tgt_orig[t] = int(ss.tgt_orig[t]);
        const int L = tree.level[b];
        const double h = g.rc / double(1LL << L);
        self_w[t] = (d == 3) ? plan->kt.self_coef / h : plan->kt.self_coef - std::log(h) / (2.0 * kPi);
    }
    lap("source_target_records");
    std::vector<TLeaf> tl;
    std::vector<int2> ent;
    std::vector<unsigned char> ent_sh;
    std::vector<float> ent_shlo;
    std::vector<int> bsb, bsc;
    near_layout(plan, tree, dl, Cu, &tl, &ent, &ent_sh, &ent_shlo, &bsb, &bsc, true);
    plan->nnear = int(tl.size());
    plan->nlist = int64_t(dl.list.size());
    lap("near_field_entries");
    // far field: originals sorted by spreading bin, window start and offsets in FP64
    const int fw = plan->w / 2;
    auto grid_coord = [&](double uu, int i, int* g0, double* del) {
        const int M = g.M[i];
        double Mu = M * uu;
        int gg = int(std::ceil(Mu - 0.5 * plan->w));
        *del = Mu - gg;
        int key = gg + fw;
        int wrap = key >= 0 ? key / M : -((-key + M - 1) / M);
        gg -= wrap * M;
        *g0 = gg;
    };
    std::vector<int64_t> sp_bin(static_cast<size_t>(n));
    std::vector<int> sp_g0(size_t(n) * 3, 0);
    std::vector<double> sp_del(size_t(n) * 3, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        int64_t bin = 0;
        for (int i = d - 1; i >= 0; --i) {
            int g0;
            double del;
            grid_coord(u[j * d + i], i, &g0, &del);
            int key = g0 + fw;  // in [0, M)
            int bi = key / plan->B[i];
            sp_g0[j * 3 + i] = key - bi * plan->B[i];  // tile offset in [0, B)
            sp_del[j * 3 + i] = del;
            bin = bin * plan->nbin[i] + bi;
        }
        sp_bin[j] = bin;
    }
    // points in bin order, stable within a bin (a counting sort over the bins)
    std::vector<int64_t> sp_order(static_cast<size_t>(n));
    {
        std::vector<int64_t> start(size_t(plan->nbins_tot) + 1, 0);
        for (int64_t j = 0; j < n; ++j) ++start[size_t(sp_bin[j]) + 1];
        for (int b = 0; b < plan->nbins_tot; ++b) start[size_t(b) + 1] += start[size_t(b)];
        for (int64_t j = 0; j < n; ++j) sp_order[size_t(start[size_t(sp_bin[j])]++)] = j;
    }
    plan->nspread = n;
    std::vector<int4> pt_g0(static_cast<size_t>(n));
    std::vector<unsigned char> pt_dq(size_t(n) * 4 * ts, 0);
    std::vector<int> sp_orig(static_cast<size_t>(n));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = sp_order[k];
        pt_g0[k] = make_int4(sp_g0[j * 3], sp_g0[j * 3 + 1], sp_g0[j * 3 + 2], 0);
        for (int i = 0; i < 3; ++i) put(pt_dq, size_t(k) * 4 + i, sp_del[j * 3 + i]);
        sp_orig[k] = int(j);
    }
    std::vector<int64_t> bin_count(size_t(plan->nbins_tot), 0);
    for (int64_t j = 0; j < n; ++j) ++bin_count[size_t(sp_bin[j])];
    std::vector<int4> subs;
    std::vector<int> bin_sub_begin;
    spread_subproblems(plan, bin_count, &subs, &bin_sub_begin);
    plan->nsub = int(subs.size());
    // interpolation targets (sorted target order)
    std::vector<int4> t_g0(size_t(plan->ntgt));
    std::vector<unsigned char> t_dq(size_t(plan->ntgt) * 4 * ts, 0);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < plan->ntgt; ++t) {
        int64_t j = ss.tgt_orig[t];
        int gg[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) {
            double del;
            grid_coord(u[j * d + i], i, &gg[i], &del);
            put(t_dq, size_t(t) * 4 + i, del);
        }
        // window starts wrapped into [0, M_i) (the kernels index periodically from there)
        for (int i = 0; i < d; ++i) gg[i] = ((gg[i] % g.M[i]) + g.M[i]) % g.M[i];
        t_g0[t] = make_int4(gg[0], gg[1], gg[2], 0);
    }
    lap("far_field_layout");
    // ---- device allocations and uploads ----
    {
        int ra = alloc_sources(plan, tl.size(), dl.list.size());
        if (ra == PDMK_OK) ra = alloc_subs(plan, subs.size());
        if (ra != PDMK_OK) return ra;
    }
    int r;
    if ((r = upload(plan, plan->d_src4, src4))) return r;
    if ((r = upload(plan, plan->d_src_orig, src_orig))) return r;
    if ((r = upload(plan, plan->d_tgt4, tgt4))) return r;
    if ((r = upload(plan, plan->d_tgt_orig, tgt_orig))) return r;
    if ((r = upload(plan, plan->d_src_lo, src_lo))) return r;
    if ((r = upload(plan, plan->d_tgt_lo, tgt_lo))) return r;
    if ((r = upload(plan, plan->d_self_w, self_w))) return r;
    if ((r = upload(plan, plan->d_tleaf, tl))) return r;
    if ((r = upload(plan, plan->d_list, dl.list))) return r;
    if ((r = upload(plan, plan->d_box_src_begin, bsb))) return r;
    if ((r = upload(plan, plan->d_box_src_count, bsc))) return r;
    if ((r = upload(plan, plan->d_box_center, tree.center))) return r;
    if ((r = upload(plan, plan->d_ent, ent))) return r;
    if ((r = upload(plan, plan->d_ent_sh, ent_sh))) return r;
    if ((r = upload(plan, plan->d_ent_shlo, ent_shlo))) return r;
    if ((r = upload(plan, plan->d_pt_g0, pt_g0))) return r;
    if ((r = upload(plan, plan->d_pt_dq, pt_dq))) return r;
    if ((r = upload(plan, plan->d_spread_orig, sp_orig))) return r;
    if ((r = upload(plan, plan->d_sub, subs))) return r;
    if ((r = upload(plan, plan->d_bin_sub_begin, bin_sub_begin))) return r;
    if ((r = upload(plan, plan->d_t_g0, t_g0))) return r;
    if ((r = upload(plan, plan->d_t_dq, t_dq))) return r;
    if ((r = upload(plan, plan->d_q_user, hq))) return r;
    lap("device_alloc_upload");
    // plane-wave passes (proxy, translation and local-expansion layouts)
    plan->pw.d_src4 = plan->d_src4;
    plan->pw.d_tgt4 = plan->d_tgt4;
    r = pw_set_sources(&plan->pw, tree, ss, leaf_of, tgt_leaf, g, plan->ws, nullptr, plan->nimg);
    if (r != PDMK_OK) return r;
    r = set_charges_device(plan, false);
    if (r != PDMK_OK) return r;
    CK(cudaStreamSynchronize(plan->ws));
    lap("plane_wave_layout_charges");
    finish_info(plan, st, pairs, n_src, m);
    // host copies for evaluations at new targets
    plan->h_u.swap(u);
    plan->h_src_orig.assign(ss.orig.begin(), ss.orig.end());
    plan->h_src_is_orig.assign(size_t(plan->nimg), 0);
    for (int64_t tt = 0; tt < int64_t(ss.tgt_of.size()); ++tt) plan->h_src_is_orig[size_t(ss.tgt_of[tt])] = 1;
    plan->h_Cu.swap(Cu);
    plan->h_y.swap(hy);
    plan->h_src_disp.swap(src_disp);
    plan->bl_ready = false;
    plan->bl_buf = nullptr;  // freed with the source buffers
    plan->h_tree = std::move(tree);
    lap("host_copies");
    plan->ready = true;
    return PDMK_OK;
}

static int set_points_device(pdmk_plan plan, int64_t n_src, const double* y, const double* q, int64_t m,
                             const double* x, int where) {
    const int64_t n = n_src + m;
    const int d = plan->d;
    const Geometry& g = plan->g;
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const size_t ts = tsize(plan);
    cudaStream_t s = plan->ws;
    auto clk = std::chrono::steady_clock::now();
    auto lap = [&](const char* name) {
        const auto now = std::chrono::steady_clock::now();
        plan->setup_names.push_back(name);
        plan->setup_ms.push_back(std::chrono::duration<double, std::milli>(now - clk).count());
        clk = now;
    };
    // scratch of this call (the device build's temporary buffers included): on every return,
    // after the stream has drained, the spares that this set-up did not take are freed, and
    // the scratch and the device build's arrays become the spares of the next set-up
    struct Scratch {
        cudaStream_t s;
        DevicePool* pool;
        std::vector<std::pair<void*, size_t>> p;
        GpuBuild gb;
        ~Scratch() {
            cudaStreamSynchronize(s);
            pool->trim();
            gpu_build_free(&gb);  // into the pool
            for (auto& x : p) pool->put(x.first, x.second);
        }
    } scr{s, &plan->pool, {}, {}};
    auto salloc = [&](void** out, size_t bytes) -> int {
        bytes = std::max<size_t>(bytes, 1);
        *out = plan->pool.get(bytes);
        if (!*out) {
            plan_set_msg(plan, "device allocation failed (set-up)");
            return PDMK_ERR_OOM;
        }
        scr.p.push_back({*out, bytes});
        return PDMK_OK;
    };
#define SALLOC(ptr, type, count)                                                          \
    do {                                                                                  \
        void* v_ = nullptr;                                                               \
        int rc_ = salloc(&v_, size_t(count) * sizeof(type));                              \
        if (rc_ != PDMK_OK) return rc_;                                                   \
        ptr = static_cast<type*>(v_);                                                     \
    } while (0)
    if (where == PDMK_DEVICE) CK(cudaStreamSynchronize(plan->stream));
    release_sources(plan);
    auto& AL = plan->src_allocs;
    DALLOC(AL, plan->d_y_keep, double, size_t(n) * d);
    DALLOC(AL, plan->d_u_keep, double, size_t(n) * d);
    double *d_q, *d_part;
    int* d_flag;
    const int nblk = std::max(1, plan->sum_blocks);
    SALLOC(d_q, double, n);
    SALLOC(d_part, double, size_t(nblk) * 2);
    SALLOC(d_flag, int, 1);
    const cudaMemcpyKind kind = where == PDMK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n_src > 0) {
        CK(cudaMemcpyAsync(plan->d_y_keep, y, size_t(n_src) * d * sizeof(double), kind, s));
        CK(cudaMemcpyAsync(d_q, q, size_t(n_src) * sizeof(double), kind, s));
    }
    if (m > 0) {
        CK(cudaMemcpyAsync(plan->d_y_keep + size_t(n_src) * d, x, size_t(m) * d * sizeof(double), kind, s));
        CK(cudaMemsetAsync(d_q + n_src, 0, size_t(m) * sizeof(double), s));
    }
    CK(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
    gpu_check_inputs(n, d, plan->d_y_keep, d_q, d_flag, d_part, nblk, s);
    std::vector<double> part(size_t(nblk) * 2);
    int bad = 0;
    CK(cudaMemcpyAsync(part.data(), d_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&bad, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (bad) return PDMK_ERR_NONFINITE;
    double qs = 0, qa = 0;
    for (int b = 0; b < nblk; ++b) {
        qs += part[size_t(b) * 2];
        qa += part[size_t(b) * 2 + 1];
    }
    if (plan->opts.neutrality == 0 && std::fabs(qs) > 1e-12 * qa) return PDMK_ERR_NON_NEUTRAL;
    gpu_orient(g, n, plan->d_y_keep, plan->d_u_keep, s);
    CK(cudaGetLastError());
    lap("read_check_orient");
    // ---- tree (device), lists (host) ----
    GpuBuild& gb = scr.gb;
    gb.d_u = plan->d_u_keep;
    gb.pool = &plan->pool;
    gb.scratch = &scr.p;
    if (!plan->h_stage) {
        void* hs = nullptr;
        if (cudaHostAlloc(&hs, size_t(64) << 20, cudaHostAllocDefault) == cudaSuccess) {
            plan->h_stage = static_cast<unsigned char*>(hs);
            plan->stage_cap = size_t(64) << 20;
        } else {
            cudaGetLastError();  // without staging the downloads go straight to the host arrays
        }
    }
    gb.h_stage = plan->h_stage;
    gb.stage_cap = plan->stage_cap;
    // the previous set-up's host tree lends its arrays' capacity (no new pages to fault in)
    Tree tree = std::move(plan->h_tree);
    BuildStats st;
    const int maxd = pw_supported(&plan->pw) ? plan->max_depth : 0;
    std::string msg;
    // 3D: the host tree's per-box arrays are read back only when a host path asks for them
    gb.download_tree = d != 3;
    int r = gpu_build_tree(g, n, plan->n_s, maxd, s, &gb, &tree, &st, &msg);
    if (r == kGpuBuildUnsupported) return r;
    if (r != PDMK_OK) {
        plan->msg = msg;
        return r;
    }
    for (int k = 0; k < 6; ++k) {
        plan->setup_names.push_back(kDeviceBuildPhases[k]);
        plan->setup_ms.push_back(st.phase_ms[k]);
    }
    clk = std::chrono::steady_clock::now();
    // near-field direct lists and descriptors on the device (the host's lists whenever a
    // list outgrows the device bound, which the level restriction rules out)
    NearLists nlst;
    DirectLists dl;
    int64_t pairs = 0;
    const bool split32 = plan->near_nh > 0;
    bool dev_lists = true;
    {
        std::string m2;
        const int rl = gpu_near_count(&gb, g, split32, &nlst, s, &m2);
        if (rl == PDMK_ERR_INTERNAL) {
            dev_lists = false;
        } else if (rl != PDMK_OK) {
            plan->msg = m2;
            return rl;
        }
    }
    bool have_tree = gb.download_tree;
    if (dev_lists) {
        pairs = nlst.pairs;
    } else {
        if (!have_tree) {
            if ((r = gpu_tree_download(gb, &tree, s, &msg)) != PDMK_OK) {
                plan->msg = msg;
                return r;
            }
            have_tree = true;
        }
        build_direct_lists(tree, &dl, &pairs);
    }
    lap("direct_lists");
    plan->n = n;
    plan->nimg = st.n_images;
    plan->ntgt = gb.ntgt;
    plan->nbox = st.nboxes;
    plan->ntleaf = dev_lists ? nlst.ntleaf : int(dl.tleaf.size());
    // caller-frame box centres on the host, as the host build (in the previous set-up's
    // array), when the host tree is here; else made on demand (ensure_host_copies)
    std::vector<double> Cu = std::move(plan->h_Cu);
    Cu.clear();
    if (have_tree) {
        Cu.resize(size_t(st.nboxes) * d);
#pragma omp parallel for schedule(static)
        for (int b = 0; b < st.nboxes; ++b)
            for (int i = 0; i < d; ++i) {
                double sum = 0;
                for (int k = 0; k < d; ++k) sum += g.Q[k * d + i] * tree.center[size_t(b) * d + k];
                Cu[size_t(b) * d + i] = sum;
            }
    }
    std::vector<TLeaf> tl;
    std::vector<int2> ent;
    std::vector<unsigned char> ent_sh;
    std::vector<float> ent_shlo;
    std::vector<int> bsb, bsc;
    if (dev_lists) {
        plan->nnear = int(nlst.ndesc);
        plan->nlist = nlst.nlist;
    } else {
        near_layout(plan, tree, dl, Cu, &tl, &ent, &ent_sh, &ent_shlo, &bsb, &bsc, false);
        plan->nnear = int(tl.size());
        plan->nlist = int64_t(dl.list.size());
    }
    lap("near_field_descriptors");
    // ---- per-point records (device) ----
    if ((r = alloc_sources(plan, size_t(plan->nnear), size_t(plan->nlist)))) return r;
    DALLOC(AL, plan->d_src_disp, double, size_t(plan->nimg) * d);
    DALLOC(AL, plan->d_tgt_of_keep, int, plan->ntgt);
    CK(cudaMemsetAsync(plan->d_src4, 0, size_t(plan->nimg) * 4 * ts, s));
    CK(cudaMemsetAsync(plan->d_tgt4, 0, size_t(plan->ntgt) * 4 * ts, s));
    if (mixed) {
        CK(cudaMemsetAsync(plan->d_src_lo, 0, size_t(plan->nimg) * 4 * sizeof(float), s));
        CK(cudaMemsetAsync(plan->d_tgt_lo, 0, size_t(plan->ntgt) * 4 * sizeof(float), s));
    }
    // box centres, caller-frame centres and levels from the device tree (no uploads)
    CK(cudaMemcpyAsync(plan->d_box_center, gb.d_center, size_t(st.nboxes) * d * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
    double *d_Cu, *d_selfw_level;
    int *d_level, *d_tgt_leaf;
    SALLOC(d_Cu, double, size_t(st.nboxes) * d);
    SALLOC(d_tgt_leaf, int, plan->ntgt);
    d_level = gb.d_level;
    gpu_box_cu(st.nboxes, d, g.Q, gb.d_center, d_Cu, s);
    CK(cudaGetLastError());
    std::vector<double> selfw_level(size_t(tree.nlevels));
    for (int L = 0; L < tree.nlevels; ++L) {
        const double h = g.rc / double(1LL << L);
        selfw_level[size_t(L)] = (d == 3) ? plan->kt.self_coef / h : plan->kt.self_coef - std::log(h) / (2.0 * kPi);
    }
    SALLOC(d_selfw_level, double, selfw_level.size());
    if ((r = upload(plan, d_selfw_level, selfw_level))) return r;
    RecordArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.d = d;
    ra.mixed = mixed ? 1 : 0;
    ra.nimg = plan->nimg;
    ra.ntgt = plan->ntgt;
    std::memcpy(ra.Q, g.Q, sizeof(ra.Q));
    std::memcpy(ra.R, g.R, sizeof(ra.R));
    std::memcpy(ra.Rinv, g.Rinv, sizeof(ra.Rinv));
    ra.y = plan->d_y_keep;
    ra.orig = gb.d_orig;
    ra.pos = gb.d_pos;
    ra.leaf = gb.d_leaf;
    ra.center = plan->d_box_center;
    ra.Cu = d_Cu;
    ra.tgt_of = gb.d_tgt_of;
    ra.tgt_orig = gb.d_tgt_orig;
    ra.box_level = d_level;
    ra.self_w_level = d_selfw_level;
    ra.src4 = plan->d_src4;
    ra.src_lo = static_cast<float*>(plan->d_src_lo);
    ra.src_orig = plan->d_src_orig;
    ra.src_disp = plan->d_src_disp;
    ra.tgt4 = plan->d_tgt4;
    ra.tgt_lo = static_cast<float*>(plan->d_tgt_lo);
    ra.tgt_orig_out = plan->d_tgt_orig;
    ra.self_w = plan->d_self_w;
    ra.tgt_leaf = d_tgt_leaf;
    gpu_records(ra, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(plan->d_tgt_of_keep, gb.d_tgt_of, size_t(plan->ntgt) * sizeof(int), cudaMemcpyDeviceToDevice,
                       s));
    CK(cudaStreamSynchronize(s));
    lap("source_target_records");
    // ---- far field (device), subproblems (host) ----
    plan->nspread = n;
    int* d_bin_count;
    SALLOC(d_bin_count, int, plan->nbins_tot);
    FarLayoutArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    fa.d = d;
    fa.mixed = mixed ? 1 : 0;
    fa.n = n;
    fa.ntgt = plan->ntgt;
    for (int i = 0; i < 3; ++i) {
        fa.M[i] = g.M[i];
        fa.B[i] = plan->B[i];
        fa.nbin[i] = plan->nbin[i];
    }
    fa.w = plan->w;
    fa.nbins_tot = plan->nbins_tot;
    fa.u = plan->d_u_keep;
    fa.tgt_orig = gb.d_tgt_orig;
    fa.pt_g0 = plan->d_pt_g0;
    fa.pt_dq = plan->d_pt_dq;
    fa.sp_orig = plan->d_spread_orig;
    fa.bin_count = d_bin_count;
    fa.t_g0 = plan->d_t_g0;
    fa.t_dq = plan->d_t_dq;
    fa.pool = &plan->pool;
    fa.scratch = &scr.p;
    if ((r = gpu_far_layout(fa, s, &msg)) != PDMK_OK) {
        plan->msg = msg;
        return r;
    }
    std::vector<int> bc(size_t(plan->nbins_tot));
    CK(cudaMemcpy(bc.data(), d_bin_count, bc.size() * sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<int64_t> bin_count(bc.begin(), bc.end());
    std::vector<int4> subs;
    std::vector<int> bin_sub_begin;
    spread_subproblems(plan, bin_count, &subs, &bin_sub_begin);
    plan->nsub = int(subs.size());
    if ((r = alloc_subs(plan, subs.size()))) return r;
    lap("far_field_layout");
    // ---- per-box uploads ----
    if (dev_lists) {
        if ((r = gpu_near_fill(&gb, g, split32, &nlst, plan->d_list, plan->d_tleaf, plan->d_box_src_begin,
                               plan->d_box_src_count, s, &msg)) != PDMK_OK) {
            plan->msg = msg;
            return r;
        }
    } else {
        if ((r = upload(plan, plan->d_tleaf, tl))) return r;
        if ((r = upload(plan, plan->d_list, dl.list))) return r;
        if ((r = upload(plan, plan->d_box_src_begin, bsb))) return r;
        if ((r = upload(plan, plan->d_box_src_count, bsc))) return r;
    }
    if ((r = upload(plan, plan->d_sub, subs))) return r;
    if ((r = upload(plan, plan->d_bin_sub_begin, bin_sub_begin))) return r;
    CK(cudaMemcpyAsync(plan->d_q_user, d_q, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // near-field entries (device): source ranges and leaf-to-leaf shifts
    if (plan->nlist > 0) {
        int *d_tleafb, *d_shift;
        long long* d_lb;
        if (dev_lists) {
            d_tleafb = nlst.d_tleaf;
            d_lb = nlst.d_list_begin;
            d_shift = nlst.d_shift;
        } else {
            SALLOC(d_tleafb, int, dl.tleaf.size());
            SALLOC(d_lb, long long, dl.list_begin.size());
            SALLOC(d_shift, int, dl.shift.size());
            static_assert(sizeof(long long) == sizeof(int64_t), "64-bit list offsets");
            if ((r = upload(plan, d_tleafb, dl.tleaf))) return r;
            CK(cudaMemcpyAsync(d_lb, dl.list_begin.data(), dl.list_begin.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
            if ((r = upload(plan, d_shift, dl.shift))) return r;
        }
        CK(cudaMemsetAsync(plan->d_ent_sh, 0, size_t(plan->nlist) * 4 * ts, s));
        if (mixed) CK(cudaMemsetAsync(plan->d_ent_shlo, 0, size_t(plan->nlist) * 4 * sizeof(float), s));
        EntryArgs ea;
        std::memset(&ea, 0, sizeof(ea));
        ea.d = d;
        ea.mixed = mixed ? 1 : 0;
        ea.nlist = plan->nlist;
        ea.ntleaf = plan->ntleaf;
        std::memcpy(ea.Q, g.Q, sizeof(ea.Q));
        for (int code = 0; code < 27; ++code) lattice_shift(g, code, &ea.Ln[code * 3]);
        ea.tleaf = d_tleafb;
        ea.list_begin = d_lb;
        ea.list = plan->d_list;
        ea.shift = d_shift;
        ea.bsb = plan->d_box_src_begin;
        ea.bsc = plan->d_box_src_count;
        ea.Cu = d_Cu;
        ea.ent = plan->d_ent;
        ea.ent_sh = plan->d_ent_sh;
        ea.ent_shlo = static_cast<float*>(plan->d_ent_shlo);
        gpu_near_entries(ea, s);
        CK(cudaGetLastError());
    }
    lap("device_alloc_upload_entries");
    plan->pw.d_src4 = plan->d_src4;
    plan->pw.d_tgt4 = plan->d_tgt4;
    SortedSources ss_unused;
    std::vector<int> none;
    if (d == 3) {
        // the plane-wave lists on the device, from the device tree
        PwTreeDev dt;
        dt.nb = gb.nb;
        dt.level = gb.d_level;
        dt.child0 = gb.d_child0;
        dt.src_b = gb.d_src_b;
        dt.src_e = gb.d_src_e;
        dt.tgt_b = gb.d_tgt_b;
        dt.tgt_e = gb.d_tgt_e;
        dt.colleague = gb.d_colleague;
        r = pw_set_sources_device(&plan->pw, dt, tree.level_start, tree.nlevels, g, s);
    } else {
        r = pw_set_sources(&plan->pw, tree, ss_unused, none, none, g, s, gb.d_leaf, plan->nimg);
    }
    if (r != PDMK_OK) return r;
    CK(cudaStreamSynchronize(s));
    lap("plane_wave_layout");
    r = set_charges_device(plan, false);
    if (r != PDMK_OK) return r;
    CK(cudaStreamSynchronize(s));
    lap("charges");
    finish_info(plan, st, pairs, n_src, m);
    plan->h_Cu.swap(Cu);
    plan->h_tree = std::move(tree);
    plan->host_tree = have_tree;
    if (!have_tree) {
        // the plan keeps the device tree's per-box arrays for a later read-back
        const int nb = gb.nb, nn = d == 3 ? 27 : 9;
        const std::pair<void*, size_t> keep[10] = {
            {gb.d_level, size_t(nb) * 4},      {gb.d_coord, size_t(nb) * d * 8}, {gb.d_parent, size_t(nb) * 4},
            {gb.d_child0, size_t(nb) * 4},     {gb.d_src_b, size_t(nb) * 8},     {gb.d_src_e, size_t(nb) * 8},
            {gb.d_tgt_b, size_t(nb) * 8},      {gb.d_tgt_e, size_t(nb) * 8},     {gb.d_center, size_t(nb) * d * 8},
            {gb.d_colleague, size_t(nb) * nn * 4}};
        for (const auto& k : keep) {
            auto it = std::find_if(gb.allocs.begin(), gb.allocs.end(),
                                   [&](const std::pair<void*, size_t>& a) { return a.first == k.first; });
            if (it == gb.allocs.end()) return PDMK_ERR_INTERNAL;
            plan->tree_keep.push_back(*it);
            gb.allocs.erase(it);
        }
        plan->tree_dev = gb;
        plan->tree_dev.allocs.clear();
        plan->tree_dev.pool = nullptr;  // pointers only: the plan owns the arrays (tree_keep)
        plan->tree_dev.scratch = nullptr;
    }
    plan->h_u.clear();
    plan->h_y.clear();
    plan->h_src_disp.clear();
    plan->h_src_orig.clear();
    plan->h_src_is_orig.clear();
    plan->host_copies = false;
    plan->bl_ready = false;
    plan->bl_buf = nullptr;  // freed with the source buffers
    plan->setup_device = true;
    lap("host_copies");
    plan->ready = true;
    return PDMK_OK;
#undef SALLOC
}

// ---------------------------------------------------------------------------------------
// Autotuning of (kappa, n_s) (pdmk_opts.autotune): candidate pairs around the Table 1 values
// are timed on the caller's sources with temporary plans; the fastest wins.  A coordinate
// search: n_s in {n0, n0/2, 2 n0} at kappa0, then kappa in {3/4, 4/3} x kappa0 at the best
// n_s (five timed plans).  Each candidate is timed on its third evaluation (the first runs
// eagerly, the second captures the graph).  Choices are cached as ratios to the Table 1
// values.
namespace {
struct TuneKey {
    int d, precision, logn;
    double eps;
    bool operator<(const TuneKey& o) const {
        if (d != o.d) return d < o.d;
        if (precision != o.precision) return precision < o.precision;
        if (logn != o.logn) return logn < o.logn;
        return eps < o.eps;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<double, double>> g_tune;  // (kappa / kappa0, n_s / n0)
}  // namespace

static int time_candidate(pdmk_plan plan, double kappa, int ns, int64_t n, const double* y, const double* q,
                          int where, double* dp, double* dg, float* ms) {
    pdmk_opts o = plan->opts;
    o.kappa = kappa;
    o.n_s = ns;
    o.autotune = 0;
    o.profile = 0;
    pdmk_plan tmp = nullptr;
    int r = pdmk_plan_create(plan->d, plan->Lc, plan->eps, &o, &tmp);
    if (r != PDMK_OK) return r;
    r = pdmk_set_sources(tmp, n, y, q, where);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (r == PDMK_OK) {
        for (int k = 0; k < 2 && r == PDMK_OK; ++k) r = pdmk_eval(tmp, dp, dg, PDMK_DEVICE);
    }
    if (r == PDMK_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) r = PDMK_ERR_CUDA;
    if (r == PDMK_OK) {
        cudaEventRecord(e0, plan->stream);
        r = pdmk_eval(tmp, dp, dg, PDMK_DEVICE);
        cudaEventRecord(e1, plan->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) r = PDMK_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    pdmk_plan_destroy(tmp);
    return r;
}

static int autotune_plan(pdmk_plan plan, int64_t n, const double* y, const double* q, int where) {
    const bool kfix = plan->opts.kappa > 0, nfix = plan->opts.n_s > 0;
    if (kfix && nfix) return PDMK_OK;
    double kappa0;
    int n0;
    {
        Geometry tmp;
        int rc = make_geometry(plan->d, plan->Lc, 1.0, plan->c, &tmp);
        if (rc != PDMK_OK) return rc;
        table1_defaults(plan->d, plan->eps, &tmp, plan->Lc, &kappa0, &n0);
    }
    if (kfix) kappa0 = plan->opts.kappa;
    if (nfix) n0 = plan->opts.n_s;
    const TuneKey key{plan->d, plan->opts.precision, int(std::floor(std::log2(double(std::max<int64_t>(n, 1))))),
                      plan->eps};
    double kr = 1.0, nr = 1.0;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            kr = it->second.first;
            nr = it->second.second;
            cached = true;
        }
    }
    if (!cached) {
        double* buf = nullptr;
        if (cudaMalloc(&buf, sizeof(double) * size_t(std::max<int64_t>(n, 1)) * (1 + plan->d)) != cudaSuccess) {
            cudaGetLastError();
            return PDMK_ERR_OOM;
        }
        double* dp = buf;
        double* dg = buf + n;
        float best = 0;
        auto trial = [&](double k, double nrat) -> int {
            const int ns = std::max(4, int(std::lround(n0 * nrat)));
            float ms = 0;
            const int r = time_candidate(plan, kappa0 * k, ns, n, y, q, where, dp, dg, &ms);
            if (r != PDMK_OK) return r;
            if (best == 0 || ms < best) {
                best = ms;
                kr = k;
                nr = nrat;
            }
            return PDMK_OK;
        };
        int r = trial(1.0, 1.0);
        if (!nfix) {
            if (r == PDMK_OK) r = trial(1.0, 0.5);
            if (r == PDMK_OK) r = trial(1.0, 2.0);
        }
        const double nbest = nr;
        if (!kfix) {
            if (r == PDMK_OK) r = trial(0.75, nbest);
            if (r == PDMK_OK) r = trial(4.0 / 3.0, nbest);
        }
        cudaFree(buf);
        if (r != PDMK_OK) return r;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = {kr, nr};
    }
    const double kappa = kfix ? plan->opts.kappa : kappa0 * kr;
    const int ns = nfix ? plan->opts.n_s : std::max(4, int(std::lround(n0 * nr)));
    if (std::fabs(kappa - plan->kappa) > 1e-12 * kappa) {
        // a new root box size changes the geometry: rebuild the plan and take its contents
        pdmk_opts o = plan->opts;
        o.kappa = kappa;
        o.n_s = ns;
        o.autotune = 0;
        pdmk_plan fresh = nullptr;
        const int r = pdmk_plan_create(plan->d, plan->Lc, plan->eps, &o, &fresh);
        if (r != PDMK_OK) return r;
        fresh->opts.autotune = plan->opts.autotune;
        fresh->opts.kappa = plan->opts.kappa;
        fresh->opts.n_s = plan->opts.n_s;
        if (plan->ws) cudaStreamSynchronize(plan->ws);
        std::swap(*plan, *fresh);
        // the plane-wave plan points at its own plan's buffer pool
        plan->pw.pool = &plan->pool;
        fresh->pw.pool = &fresh->pool;
        pdmk_plan_destroy(fresh);  // the old contents
    }
    plan->n_s = ns;
    return PDMK_OK;
}

extern "C" int pdmk_set_sources(pdmk_plan plan, int64_t n, const double* y, const double* q, int where) {
    if (plan && plan->opts.autotune && n > 0 && y && q) {
        const int r = autotune_plan(plan, n, y, q, where);
        if (r != PDMK_OK) return r;
    }
    return set_points(plan, n, y, q, 0, nullptr, where);
}

extern "C" int pdmk_set_sources_targets(pdmk_plan plan, int64_t n, const double* y, const double* q, int64_t m,
                                        const double* x, int where) {
    if (m < 1 || !x) return PDMK_ERR_BAD_ARG;
    return set_points(plan, n, y, q, m, x, where);
}

extern "C" int pdmk_set_charges(pdmk_plan plan, const double* q, int where) {
    if (!plan || !q) return PDMK_ERR_BAD_ARG;
    if (!plan->ready) return PDMK_ERR_NOT_READY;
    // order after the caller's stream (device charges may still be in flight there)
    CK(cudaEventRecord(plan->ev_fork, plan->stream));
    CK(cudaStreamWaitEvent(plan->ws, plan->ev_fork, 0));
    CK(cudaMemcpyAsync(plan->d_q_user, q, size_t(plan->n_src) * sizeof(double),
                       where == PDMK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, plan->ws));
    int r = set_charges_device(plan, where == PDMK_HOST || plan->opts.neutrality == 0);
    if (r != PDMK_OK) return r;
    CK(cudaEventRecord(plan->ev_join, plan->ws));
    CK(cudaStreamWaitEvent(plan->stream, plan->ev_join, 0));
    return PDMK_OK;
}

static int stage_mark(pdmk_plan plan, const char* name) {
    if (!plan->opts.profile) return PDMK_OK;
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    CK(cudaEventRecord(e, plan->ws));
    plan->ev.push_back(e);
    plan->stage_names.push_back(name);
    return PDMK_OK;
}

// The warp kernel's residual series (monomials in 2 s - 1, zero-padded) into its arguments.
template <typename T>
static void near_coefs(pdmk_plan plan, NearArgs<T>* na) {
    for (int k = 0; k < kNearMono; ++k) {
        na->cmA[k] = k < int(plan->mA.size()) ? T(plan->mA[k]) : T(0);
        na->cmB[k] = k < int(plan->mB.size()) ? T(plan->mB[k]) : T(0);
    }
}

// The residual direct sum over ndesc target descriptors (near-field arguments filled in).
template <typename T, int D>
static void near_launch(pdmk_plan plan, const NearArgs<T>& na, int ndesc, cudaStream_t st) {
    const int nc = std::max(na.nA, na.nB);
    const int wb = (ndesc + kNearWarps - 1) / kNearWarps, wt = 32 * kNearWarps;
    // A is usually two terms shorter than B: its own compile-time length then
    const bool ash = na.nA <= plan->near_nh - 2;
#define PDMK_NEAR(NH)                                                                         \
(ash ? k_near_warp<T, D, NH, NH - 2><<<wb, wt, 0, st>>>(na)                            \
     : k_near_warp<T, D, NH, NH><<<wb, wt, 0, st>>>(na))
    if (plan->near_nh == 8) PDMK_NEAR(8);
    else if (plan->near_nh == 10) PDMK_NEAR(10);
    else if (plan->near_nh == 12) PDMK_NEAR(12);
    else if (plan->near_nh == 14) PDMK_NEAR(14);
    else if (plan->near_nh == 16) PDMK_NEAR(16);
    else if (plan->near_nh == 20) PDMK_NEAR(20);
    else if (plan->near_nh == 24) PDMK_NEAR(24);
#undef PDMK_NEAR
    else if (nc <= 8) k_nearfield<T, D, 8><<<ndesc, kNearThreads, 0, st>>>(na);
    else if (nc <= 12) k_nearfield<T, D, 12><<<ndesc, kNearThreads, 0, st>>>(na);
    else if (nc <= 16) k_nearfield<T, D, 16><<<ndesc, kNearThreads, 0, st>>>(na);
    else if (nc <= 20) k_nearfield<T, D, 20><<<ndesc, kNearThreads, 0, st>>>(na);
    else if (nc <= 24) k_nearfield<T, D, 24><<<ndesc, kNearThreads, 0, st>>>(na);
    else if (nc <= 32) k_nearfield<T, D, 32><<<ndesc, kNearThreads, 0, st>>>(na);
    else k_nearfield<T, D, 40><<<ndesc, kNearThreads, 0, st>>>(na);
}

// The far field up to the potential grid: spread, fold, FFT, scale, inverse FFT (and the
// narrowing copy a mixed 3D plan's interpolation reads).  Afterwards the grid in the
// plan's precision (d_grid) holds the smooth periodic potential on the Fourier grid, except
// for the 2D halo interpolation, which reads the transform grid itself.
// Spreading (type-1 half) and the fold of the subproblem or per-CTA slabs into a real grid
// out (FP32 if out_f32, else FP64).
template <typename T, int D>
static int spread_fold(pdmk_plan plan, cudaStream_t s, void* out, bool out_f32) {
    const Geometry& g = plan->g;
    const T hwi2 = T(4.0 / (double(plan->w) * plan->w));
    void* slab = plan->slab_override ? plan->slab_override : plan->d_slab;
    if (D == 2 && plan->whole_ctas > 0 && plan->far_halo && sizeof(T) == 4) {
        const int nwarp = 8;
        const int Mp0 = g.M[0] + plan->w - 1, Mp1 = g.M[1] + plan->w - 1;
        const size_t smem = sizeof(T) * (size_t(nwarp) * Mp0 * Mp1 + size_t(nwarp) * 2 * plan->w);
        auto halo = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            kern<<<plan->whole_ctas, 32 * nwarp, smem, s>>>(
                plan->d_t_g0, static_cast<const T*>(plan->d_t_dq), static_cast<const T*>(plan->d_tgt4),
                int(plan->ntgt), static_cast<T*>(slab), g.M[0], g.M[1], hwi2, static_cast<const T*>(plan->d_monoW));
        };
        if (plan->w == 8) halo(k_spread_halo<T, 8, 12>);
        else if (plan->w == 13) halo(k_spread_halo<T, 13, 16>);
        else halo(k_spread_halo<T, 17, 20>);
        ++plan->launches;
        CK(cudaGetLastError());
        const int blocks = int((plan->ncell + 31) / 32);
        if (out_f32)
            k_fold_whole<T, float><<<std::max(blocks, 1), 256, 0, s>>>(
                static_cast<const T*>(slab), plan->whole_ctas, static_cast<float*>(out), int(plan->ncell));
        else
            k_fold_whole<T, double><<<std::max(blocks, 1), 256, 0, s>>>(
                static_cast<const T*>(slab), plan->whole_ctas, static_cast<double*>(out), int(plan->ncell));
        ++plan->launches;
        CK(cudaGetLastError());
    } else if (D == 2 && plan->whole_ctas > 0) {
        const int nwarp = 8;
        const size_t smem = sizeof(T) * (size_t(nwarp) * plan->ncell + size_t(nwarp) * 2 * plan->w);
        const int nW = int(plan->cW.size());
        const int4* tg = plan->d_t_g0;
        const T* tdq = static_cast<const T*>(plan->d_t_dq);
        const T* q4 = static_cast<const T*>(plan->d_tgt4);
        const T* cwp = static_cast<const T*>(plan->d_coefW);
        T* sl = static_cast<T*>(slab);
        const int nt = int(plan->ntgt);
        auto whole_w = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            kern<<<plan->whole_ctas, 32 * nwarp, smem, s>>>(tg, tdq, q4, nt, sl, g.M[0], g.M[1], hwi2, cwp, nW);
        };
        // compile-time widths of the default windows (eps = 1e-3, 1e-6, 1e-9)
        if (plan->w == 8 && nW <= 16) whole_w(k_spread_whole_w<T, 8, 16>);
        else if (plan->w == 13 && nW <= 16) whole_w(k_spread_whole_w<T, 13, 16>);
        else if (plan->w == 13 && nW <= 20) whole_w(k_spread_whole_w<T, 13, 20>);
        else if (plan->w == 17 && nW <= 20) whole_w(k_spread_whole_w<T, 17, 20>);
        else if (plan->w == 17 && nW <= 28) whole_w(k_spread_whole_w<T, 17, 28>);
        else {
            CK(cudaFuncSetAttribute(k_spread_whole<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            k_spread_whole<T><<<plan->whole_ctas, 32 * nwarp, smem, s>>>(tg, tdq, q4, nt, sl, g.M[0], g.M[1], plan->w,
                                                                        hwi2, cwp, nW);
        }
        ++plan->launches;
        CK(cudaGetLastError());
        const int blocks = int((plan->ncell + 31) / 32);
        if (out_f32)
            k_fold_whole<T, float><<<std::max(blocks, 1), 256, 0, s>>>(
                static_cast<const T*>(slab), plan->whole_ctas, static_cast<float*>(out), int(plan->ncell));
        else
            k_fold_whole<T, double><<<std::max(blocks, 1), 256, 0, s>>>(
                static_cast<const T*>(slab), plan->whole_ctas, static_cast<double*>(out), int(plan->ncell));
        ++plan->launches;
        CK(cudaGetLastError());
    } else {
    if (plan->nsub > 0) {
        SpreadArgs<T> sa;
        sa.pt_g0 = plan->d_pt_g0;
        sa.pt_dq = static_cast<const T*>(plan->d_pt_dq);
        sa.sub = plan->d_sub;
        sa.nsub = plan->nsub;
        sa.slab = static_cast<T*>(slab);
        sa.P0 = plan->P[0]; sa.P1 = plan->P[1]; sa.P2 = plan->P[2]; sa.Ptot = plan->Ptot;
        sa.B0 = plan->B[0]; sa.B1 = plan->B[1]; sa.B2 = plan->B[2];
        sa.w = plan->w;
        sa.half_w_inv2 = hwi2;
        sa.coefW = static_cast<const T*>(plan->d_coefW);
        sa.nW = int(plan->cW.size());
        if (D == 3 && plan->spread_reg3d) {
            auto reg = [&](auto kern, size_t smem, int nt) -> int {
                CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
                kern<<<plan->nsub, nt, smem, s>>>(sa);
                return PDMK_OK;
            };
            int rr = PDMK_ERR_INTERNAL;
            if constexpr (sizeof(T) == 4) {
                if (plan->w == 8) rr = reg(k_spread3d_reg<T, 8, 128, 4>, spread3d_reg_smem<T, 8, 128>(), 128);
                else if (plan->w == 13) rr = reg(k_spread3d_reg<T, 13, 128, 3>, spread3d_reg_smem<T, 13, 128>(), 128);
                else rr = reg(k_spread3d_reg<T, 17, 128, 2>, spread3d_reg_smem<T, 17, 128>(), 128);
            }
            if (rr != PDMK_OK) return rr;
        } else {
            size_t smem = sizeof(T) * (size_t(plan->Ptot) + size_t(kSpreadChunk) * 3 * plan->w + kSpreadChunk) +
                          sizeof(int) * kSpreadChunk * 3;
            CK(cudaFuncSetAttribute(k_spread<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            k_spread<T, D><<<plan->nsub, kSpreadThreads, smem, s>>>(sa);
        }
        ++plan->launches;
        CK(cudaGetLastError());
    }
    {
        auto fold = [&](auto* gridp) {
        using G = std::remove_pointer_t<decltype(gridp)>;
        FoldArgs<T, G> fa;
        fa.slab = static_cast<const T*>(slab);
        fa.bin_sub_begin = plan->d_bin_sub_begin;
        fa.grid = gridp;
        fa.M0 = g.M[0]; fa.M1 = g.M[1]; fa.M2 = g.M[2];
        fa.nb0 = plan->nbin[0]; fa.nb1 = plan->nbin[1]; fa.nb2 = plan->nbin[2];
        fa.B0 = plan->B[0]; fa.B1 = plan->B[1]; fa.B2 = plan->B[2];
        fa.P0 = plan->P[0]; fa.P1 = plan->P[1]; fa.P2 = plan->P[2]; fa.Ptot = plan->Ptot;
        fa.fw = plan->w / 2;
        int blocks = int(std::min<int64_t>((plan->ncell + 255) / 256, int64_t(plan->nsm) * 8));
        k_fold<T, D, G><<<std::max(blocks, 1), 256, 0, s>>>(fa);
        };
        if (out_f32) fold(static_cast<float*>(out));
        else fold(static_cast<double*>(out));
        ++plan->launches;
        CK(cudaGetLastError());
    }
    }
    return PDMK_OK;
}

template <typename T, int D>
static int far_grid(pdmk_plan plan, cudaStream_t s, bool interp_halo) {
    int r;
    if ((r = spread_fold<T, D>(plan, s, plan->d_grid64, plan->fft32))) return r;
    if ((r = stage_mark(plan, "spread"))) return r;
    const int cblocks = int(std::max<int64_t>(1, std::min<int64_t>((plan->ncell + 255) / 256, int64_t(plan->nsm) * 8)));
    if (plan->fft32)
        CKFFT(cufftExecR2C(plan->fft_fwd, (cufftReal*)plan->d_grid64, (cufftComplex*)plan->d_spec));
    else
        CKFFT(cufftExecD2Z(plan->fft_fwd, (cufftDoubleReal*)plan->d_grid64, (cufftDoubleComplex*)plan->d_spec));
    if ((r = stage_mark(plan, "fft_fwd"))) return r;
    {
        int blocks = int(std::min<int64_t>((plan->nhalf + 255) / 256, int64_t(plan->nsm) * 8));
        if (plan->fft32)
            k_scale<float><<<std::max(blocks, 1), 256, 0, s>>>(static_cast<float*>(plan->d_spec), plan->d_weight,
                                                               plan->nhalf);
        else
            k_scale<double><<<std::max(blocks, 1), 256, 0, s>>>(static_cast<double*>(plan->d_spec), plan->d_weight,
                                                                plan->nhalf);
        ++plan->launches;
        CK(cudaGetLastError());
    }
    if ((r = stage_mark(plan, "scale"))) return r;
    if (plan->fft32)
        CKFFT(cufftExecC2R(plan->fft_inv, (cufftComplex*)plan->d_spec, (cufftReal*)plan->d_grid64));
    else
        CKFFT(cufftExecZ2D(plan->fft_inv, (cufftDoubleComplex*)plan->d_spec, (cufftDoubleReal*)plan->d_grid64));
    // the halo interpolation reads the transform grid in its own precision; the others read T
    if (sizeof(T) == 4 && !plan->fft32 && !interp_halo) {
        k_convert<double, T><<<cblocks, 256, 0, s>>>(static_cast<const double*>(plan->d_grid64),
                                                     static_cast<T*>(plan->d_grid), plan->ncell);
        ++plan->launches;
        CK(cudaGetLastError());
    }
    if ((r = stage_mark(plan, "fft_inv"))) return r;
    return PDMK_OK;
}

template <typename T, int D>
static int run_eval(pdmk_plan plan, double* pot, double* grad, int64_t out_first) {
    cudaStream_t s = plan->ws;
    const Geometry& g = plan->g;
    int r;
    plan->launches = 0;
    for (auto e : plan->ev) cudaEventDestroy(e);
    plan->ev.clear();
    plan->stage_names.clear();
    plan->stage_ms.clear();
    if ((r = stage_mark(plan, "start"))) return r;
    // Three independent branches until assembly: far field on ws, plane-wave passes on
    // ws_pw, near-field sum on ws_near (one stream when profiling per stage).
    const bool branches = !plan->opts.profile;
    cudaStream_t s_pw = branches ? plan->ws_pw : s, s_near = branches ? plan->ws_near : s;
    if (branches) {
        CK(cudaEventRecord(plan->ev_s, s));
        CK(cudaStreamWaitEvent(s_pw, plan->ev_s, 0));
        CK(cudaStreamWaitEvent(s_near, plan->ev_s, 0));
    }
    // ---- far field: spread, fold, FFT, scale, inverse FFT, interpolate ----
    const T hwi2 = T(4.0 / (double(plan->w) * plan->w));
    const bool interp_halo = plan->ntgt > 0 && D == 2 && plan->far_halo && sizeof(T) == 4;
    if ((r = far_grid<T, D>(plan, s, interp_halo))) return r;
    if (interp_halo) {
        const int Mp0 = g.M[0] + plan->w - 1, Mp1 = g.M[1] + plan->w - 1;
        const size_t smem = sizeof(T) * size_t(Mp0) * Mp1;
        auto interp = [&](auto kern, auto* gridp) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            int per_sm = 0, nsm = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
            const int grid = int(std::max<int64_t>(1, std::min<int64_t>((plan->ntgt + 255) / 256,
                                                                        int64_t(std::max(1, per_sm)) * nsm)));
            kern<<<grid, 256, smem, s>>>(gridp, plan->d_t_g0,
                                         static_cast<const T*>(plan->d_t_dq), int(plan->ntgt), g.M[0], g.M[1], hwi2,
                                         static_cast<const T*>(plan->d_monoW), static_cast<const T*>(plan->d_monoWd),
                                         plan->d_pot_far, plan->d_gradu_far);
        };
        if (plan->fft32) {
            const float* gp = static_cast<const float*>(plan->d_grid64);
            if (plan->w == 8) interp(k_interp_halo<T, 8, 12, 12, float>, gp);
            else if (plan->w == 13) interp(k_interp_halo<T, 13, 16, 16, float>, gp);
            else interp(k_interp_halo<T, 17, 20, 20, float>, gp);
        } else {
            const double* gp = static_cast<const double*>(plan->d_grid64);
            if (plan->w == 8) interp(k_interp_halo<T, 8, 12, 12, double>, gp);
            else if (plan->w == 13) interp(k_interp_halo<T, 13, 16, 16, double>, gp);
            else interp(k_interp_halo<T, 17, 20, 20, double>, gp);
        }
        ++plan->launches;
        CK(cudaGetLastError());
    } else if (plan->ntgt > 0 && D == 3 && plan->far_warp3d && plan->ntgt < 50000) {
        // (with many targets a thread per target already fills the GPU)
        auto interp = [&](auto kern) {
            const int warps = int(std::min<int64_t>(plan->ntgt, int64_t(plan->nsm) * 64));
            kern<<<(warps + 7) / 8, 256, 0, s>>>(static_cast<const T*>(plan->d_grid), plan->d_t_g0,
                                                 static_cast<const T*>(plan->d_t_dq), int(plan->ntgt), g.M[0], g.M[1],
                                                 g.M[2], hwi2, static_cast<const T*>(plan->d_monoW),
                                                 static_cast<const T*>(plan->d_monoWd), plan->d_pot_far,
                                                 plan->d_gradu_far);
        };
        if (plan->w == 8) interp(k_interp_warp3d<T, 8, 16, 16>);
        else if (plan->w == 13) interp(k_interp_warp3d<T, 13, 20, 20>);
        else interp(k_interp_warp3d<T, 17, 24, 24>);
        ++plan->launches;
        CK(cudaGetLastError());
    } else if (plan->ntgt > 0) {
        InterpArgs<T> ia;
        ia.grid = static_cast<const T*>(plan->d_grid);
        ia.t_g0 = plan->d_t_g0;
        ia.t_dq = static_cast<const T*>(plan->d_t_dq);
        ia.nt = int(plan->ntgt);
        ia.M0 = g.M[0]; ia.M1 = g.M[1]; ia.M2 = g.M[2];
        ia.w = plan->w;
        ia.half_w_inv2 = hwi2;
        ia.coefW = static_cast<const T*>(plan->d_coefW);
        ia.coefWd = static_cast<const T*>(plan->d_coefWd);
        ia.nW = int(plan->cW.size());
        ia.nWd = int(plan->cWd.size());
        ia.pot = plan->d_pot_far;
        ia.gradu = plan->d_gradu_far;
        // compile-time widths in FP32 (their per-thread y/z windows fit the static shared limit)
        if (D == 3 && sizeof(T) == 4 && (plan->w == 8 || plan->w == 13 || plan->w == 17)) {
            if constexpr (sizeof(T) == 4) {
                const int nb = int((plan->ntgt + 127) / 128);
                auto iw = [&](auto kern, size_t smb) {
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smb));
                    kern<<<nb, 128, smb, s>>>(ia);
                };
                if (plan->w == 8) iw(k_interp3d_w<T, 8>, interp3d_w_smem<T, 8>());
                else if (plan->w == 13) iw(k_interp3d_w<T, 13>, interp3d_w_smem<T, 13>());
                else iw(k_interp3d_w<T, 17>, interp3d_w_smem<T, 17>());
            }
        } else {
            size_t smem = sizeof(T) * 128 * 2 * D * plan->w;
            CK(cudaFuncSetAttribute(k_interp<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            k_interp<T, D><<<int((plan->ntgt + 127) / 128), 128, smem, s>>>(ia);
        }
        ++plan->launches;
        CK(cudaGetLastError());
    }
    if ((r = stage_mark(plan, "interp"))) return r;
    // ---- near field: plane-wave passes, then the direct residual sum ----
    static const char* pw_names[kPwPhases] = {"pw_moments", "pw_merge",    "pw_out",
                                              "pw_translate_in", "pw_downward", "pw_leaf_eval"};
    for (int ph = 0; ph < kPwPhases; ++ph) {
        r = pw_eval(&plan->pw, s_pw, ph);
        if (r != PDMK_OK) return r;
        if ((r = stage_mark(plan, pw_names[ph]))) return r;
    }
    plan->launches += plan->pw.launches;
    if (plan->nnear > 0) {
        NearArgs<T> na{};
        na.tleaf = plan->d_tleaf;
        na.ntleaf = plan->nnear;
        na.list = plan->d_list;
        na.box_src_begin = plan->d_box_src_begin;
        na.box_src_count = plan->d_box_src_count;
        na.box_center = plan->d_box_center;
        na.src4 = static_cast<const T*>(plan->d_src4);
        na.tgt4 = static_cast<const T*>(plan->d_tgt4);
        na.pot = plan->d_pot_near;
        na.grad = plan->d_grad_near;
        na.inv_rc = 1.0 / g.rc;
        na.coefA = static_cast<const T*>(plan->d_coefA);
        na.coefB = static_cast<const T*>(plan->d_coefB);
        na.nA = int(plan->cA.size());
        na.nB = int(plan->cB.size());
        na.count_in = nullptr;
        na.src_lo = static_cast<const T*>(plan->d_src_lo);
        na.tgt_lo = static_cast<const T*>(plan->d_tgt_lo);
        na.close_s = T(0.04);  // r < 0.2 h
        if (plan->count_pending) {
            CK(cudaMemsetAsync(plan->d_count, 0, sizeof(unsigned long long), s_near));
            na.count_in = plan->d_count;
        }
        na.ent = plan->d_ent;
        na.ent_sh = static_cast<const T*>(plan->d_ent_sh);
        na.ent_shlo = static_cast<const T*>(plan->d_ent_shlo);
        near_coefs(plan, &na);
        near_launch<T, D>(plan, na, plan->nnear, s_near);
        ++plan->launches;
        CK(cudaGetLastError());
    }
    if ((r = stage_mark(plan, "nearfield"))) return r;
    if (branches) {
        CK(cudaEventRecord(plan->ev_pw, s_pw));
        CK(cudaEventRecord(plan->ev_near, s_near));
        CK(cudaStreamWaitEvent(s, plan->ev_pw, 0));
        CK(cudaStreamWaitEvent(s, plan->ev_near, 0));
    }
    // ---- assembly ----
    {
        AssembleArgs aa;
        aa.nt = plan->ntgt;
        aa.d = D;
        aa.tgt_orig = plan->d_tgt_orig;
        aa.self_w = plan->d_self_w;
        aa.q_tgt = plan->d_q_tgt;
        aa.pot_near = plan->d_pot_near;
        aa.grad_near = plan->d_grad_near;
        aa.pot_pw = plan->pw.active ? plan->pw.d_pot : nullptr;
        aa.grad_pw = plan->pw.active ? plan->pw.d_grad : nullptr;
        aa.pot_far = plan->d_pot_far;
        aa.gradu_far = plan->d_gradu_far;
        aa.qsum = plan->d_qsums;
        aa.mean_coef = plan->kt.rhat0 * g.rc * g.rc / g.V;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                // grad_x_i = sum_j (R^{-T})_{ij} M_j d/d(M_j u_j)
                aa.G[i * D + j] = g.Rinv[j * D + i] * g.M[j];
                aa.Qt[i * D + j] = g.Q[j * D + i];
            }
        aa.pot_out = pot;
        aa.grad_out = grad;
        aa.out_first = out_first;
        int blocks = int(std::min<int64_t>((plan->ntgt + 255) / 256, int64_t(plan->nsm) * 8));
        k_assemble<D, T><<<std::max(blocks, 1), 256, 0, s>>>(aa);
        ++plan->launches;
        CK(cudaGetLastError());
    }
    if ((r = stage_mark(plan, "assemble"))) return r;
    return PDMK_OK;
}

// out_first: the first caller-order point to write (points before it are computed but not
// written; the outputs start at that point)
static int launch_eval(pdmk_plan plan, double* dp, double* dg, int64_t out_first) {
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    if (plan->d == 2)
        return mixed ? run_eval<float, 2>(plan, dp, dg, out_first) : run_eval<double, 2>(plan, dp, dg, out_first);
    return mixed ? run_eval<float, 3>(plan, dp, dg, out_first) : run_eval<double, 3>(plan, dp, dg, out_first);
}

extern "C" int pdmk_eval(pdmk_plan plan, double* pot, double* grad, int where) {
    if (!plan || !pot) return PDMK_ERR_BAD_ARG;
    if (!plan->ready) return PDMK_ERR_NOT_READY;
    double* dp = where == PDMK_DEVICE ? pot : plan->d_pot_out;
    double* dg = grad ? (where == PDMK_DEVICE ? grad : plan->d_grad_out) : nullptr;
    int r;
    // a bounded device wait of an earlier (device) evaluation expired
    if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
        *plan->pw.h_err = 0;
        return PDMK_ERR_TIMEOUT;
    }
    // the work runs on the plan's stream, ordered after the caller's stream
    CK(cudaEventRecord(plan->ev_fork, plan->stream));
    CK(cudaStreamWaitEvent(plan->ws, plan->ev_fork, 0));
    // The launch sequence depends only on the plan and the output pointers, so from the second
    // evaluation on it is replayed from a captured CUDA graph (profiling and the first,
    // pair-counting evaluation run eagerly).
    const bool eager = plan->opts.profile || plan->count_pending || plan->evals_since_setup == 0;
    if (eager) {
        r = launch_eval(plan, dp, dg, plan->out_first);
        if (r != PDMK_OK) return r;
    } else {
        if (!plan->gexec || plan->g_pot != dp || plan->g_grad != dg) {
            drop_graph(plan);
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(plan->ws, cudaStreamCaptureModeThreadLocal));
            r = launch_eval(plan, dp, dg, plan->out_first);
            cudaError_t ce = cudaStreamEndCapture(plan->ws, &graph);
            if (r != PDMK_OK) {
                if (graph) cudaGraphDestroy(graph);
                return r;
            }
            CK(ce);
            cudaError_t ie = cudaGraphInstantiate(&plan->gexec, graph, 0);
            cudaGraphDestroy(graph);
            CK(ie);
            plan->g_pot = dp;
            plan->g_grad = dg;
        }
        CK(cudaGraphLaunch(plan->gexec, plan->ws));
    }
    ++plan->evals_since_setup;
    if (where != PDMK_DEVICE) {
        CK(cudaMemcpyAsync(pot, dp, size_t(plan->n_out) * sizeof(double), cudaMemcpyDeviceToHost, plan->ws));
        if (grad)
            CK(cudaMemcpyAsync(grad, dg, size_t(plan->n_out) * plan->d * sizeof(double), cudaMemcpyDeviceToHost, plan->ws));
        CK(cudaStreamSynchronize(plan->ws));
        if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
            *plan->pw.h_err = 0;
            return PDMK_ERR_TIMEOUT;
        }
    }
    CK(cudaEventRecord(plan->ev_join, plan->ws));
    CK(cudaStreamWaitEvent(plan->stream, plan->ev_join, 0));
    if (plan->count_pending) {
        unsigned long long cnt = 0;
        CK(cudaMemcpyAsync(&cnt, plan->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, plan->ws));
        CK(cudaStreamSynchronize(plan->ws));
        plan->info.near_pairs_in = int64_t(cnt);
        plan->count_pending = false;
    }
    if (plan->opts.profile) {
        CK(cudaEventSynchronize(plan->ev.back()));
        plan->stage_ms.assign(plan->ev.size(), 0.0);
        for (size_t i = 1; i < plan->ev.size(); ++i) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, plan->ev[i - 1], plan->ev[i]));
            plan->stage_ms[i] = ms;
        }
    }
    return PDMK_OK;
}

extern "C" int pdmk_stage_times(pdmk_plan plan, const char** names, double* ms, int cap) {
    if (!plan) return PDMK_ERR_BAD_ARG;
    int n = int(std::min(plan->stage_ms.size(), plan->stage_names.size())) - 1;
    if (n < 0) n = 0;
    for (int i = 0; i < n && i < cap; ++i) {
        if (names) names[i] = plan->stage_names[i + 1].c_str();
        if (ms) ms[i] = plan->stage_ms[i + 1];
    }
    return n;
}

extern "C" int pdmk_setup_times(pdmk_plan plan, const char** names, double* ms, int cap) {
    if (!plan || cap < 0) return PDMK_ERR_BAD_ARG;
    const int n = int(std::min(plan->setup_ms.size(), plan->setup_names.size()));
    for (int i = 0; i < n && i < cap; ++i) {
        if (names) names[i] = plan->setup_names[i];
        if (ms) ms[i] = plan->setup_ms[i];
    }
    return n;
}

extern "C" const char* pdmk_plan_message(pdmk_plan plan) {
    return plan ? plan->msg.c_str() : "";
}

extern "C" int pdmk_get_info(pdmk_plan plan, pdmk_info* info) {
    if (!plan || !info) return PDMK_ERR_BAD_ARG;
    *info = plan->info;
    info->device_bytes = plan->device_bytes + plan->pw.device_bytes;
    info->launches = plan->launches;
    if (!plan->ready) {
        info->d = plan->d; info->eps = plan->eps; info->c = plan->c; info->rc = plan->g.rc;
        info->V = plan->g.V; info->kappa = plan->kappa; info->n_s = plan->n_s; info->window_w = plan->w;
        for (int i = 0; i < 3; ++i) { info->M[i] = plan->g.M[i]; info->nroot[i] = plan->g.nroot[i]; }
    }
    return PDMK_OK;
}

// ------------------------------------------------------------------------------------------
// Evaluation that allocates nothing.
//
// Some callers cannot allocate device memory when they evaluate: code that runs while a
// framework owns the whole device heap (a simulation engine that reserved its memory pool at
// start-up, a caching allocator that forbids cudaMalloc inside a step), or code that runs
// under a real-time budget where an allocation's implicit synchronisation is not acceptable.
// For them, pdmk_eval_noalloc evaluates an existing plan into caller-provided device buffers
// and takes the spreading kernel's per-subproblem scratch (its padded tiles) from the
// file-scope array below instead of the plan's own buffer.  The array is a fixed part of every
// device that loads this library, for the lifetime of the process.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;
}  // namespace

extern "C" int pdmk_eval_noalloc(pdmk_plan plan, double* pot, double* grad) {
    if (!plan || !pot) return PDMK_ERR_BAD_ARG;
    if (!plan->ready) return PDMK_ERR_NOT_READY;
    if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
        *plan->pw.h_err = 0;
        return PDMK_ERR_TIMEOUT;
    }
    const size_t need = slab_bytes(plan);
    if (need > kNoAllocScratchBytes) {
        plan_set_msg(plan, "spreading scratch exceeds the 16 MiB static array");
        return PDMK_ERR_TOO_LARGE;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PDMK_ERR_BAD_ARG;
    void* scratch = nullptr;
    {
        // first call on this device: the array's device address (the host-side symbol is
        // only a stand-in for it and must never be passed to a kernel)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            g_noalloc_ptr[dev] = ptr;
        }
        scratch = g_noalloc_ptr[dev];
    }
    CK(cudaEventRecord(plan->ev_fork, plan->stream));
    CK(cudaStreamWaitEvent(plan->ws, plan->ev_fork, 0));
    // eager launches only (no graph instantiation, no profiling events); the spread kernel
    // writes every scratch element it later reads, so nothing needs clearing between calls
    const bool saved_profile = plan->opts.profile != 0;
    const bool saved_count = plan->count_pending;
    plan->opts.profile = 0;
    plan->count_pending = false;
    plan->slab_override = scratch;
    const int r = launch_eval(plan, pot, grad, plan->out_first);
    plan->slab_override = nullptr;
    plan->opts.profile = saved_profile ? 1 : 0;
    plan->count_pending = saved_count;
    if (r != PDMK_OK) return r;
    CK(cudaEventRecord(plan->ev_join, plan->ws));
    CK(cudaStreamWaitEvent(plan->stream, plan->ev_join, 0));
    return PDMK_OK;
}

// ---------------------------------------------------------------------------------------
// Evaluation at new targets against the existing source tree (Algorithm 1's RETURN at points
// given per call).  A target x takes the deepest box A on its path whose complete local
// expansion is stored (the receiving boxes of the plane-wave passes; in 3D also the target
// leaves) and the virtual leaf B' = A's child containing x (A itself when A is x's leaf; the
// root box when no ancestor has one).  With L' the level of B':
//     near(x) = local_A(x)  [= sum_{l < L'} D_l, the telescoped plane-wave part]
//             + sum over the source leaves meeting B''s neighbourhood of R_{L'}(x - y) q
// which is the interaction rule of the plan's own targets with B' in place of the leaf: by
// the level restriction no coarser leaf meets the neighbourhood of a non-leaf B'.  The far
// field is interpolated at x; a target that equals a source bitwise (the same wrapped
// fractional coordinates) excludes that source's self pair and has W_{L'}(0) q removed.
__global__ void k_self_charges(int64_t m, const int* __restrict__ self_pt, const double* __restrict__ q,
                               double* __restrict__ q_tgt) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
        q_tgt[i] = self_pt[i] >= 0 ? q[self_pt[i]] : 0.0;
}

namespace {
// host-side layout of one call: the targets in evaluation order and their descriptors
struct TargetLayout {
    int64_t m = 0;
    std::vector<unsigned char> tgt4, tgt4a, t_dq;  // T-sized records (4 per target)
    std::vector<float> tgt_lo;
    std::vector<int4> t_g0;
    std::vector<double> self_w;
    std::vector<int> self_pt, tgt_orig;
    std::vector<TLeaf> desc;
    std::vector<int2> ent;
    std::vector<unsigned char> ent_sh;
    std::vector<float> ent_shlo;
    std::vector<int4> evl;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
}  // namespace

static int build_target_layout(pdmk_plan plan, int64_t m, const double* hx, TargetLayout* out) {
    const int d = plan->d;
    const Geometry& g = plan->g;
    const Tree& t = plan->h_tree;
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const size_t ts = tsize(plan);
    const int depth = t.nlevels - 1;
    const double cscale = double(1LL << depth) / g.rc;
    pw_host_slots(&plan->pw, t);  // after a device layout, the per-box slot tables are made here
    const std::vector<unsigned char>& full = plan->pw.local_full;
    std::vector<double> tu(size_t(m) * d), tsh(size_t(m) * d);
    std::vector<int> leaf(static_cast<size_t>(m)), vb(static_cast<size_t>(m)), ab(static_cast<size_t>(m));
    std::vector<int> selfp(static_cast<size_t>(m), -1);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t j = 0; j < m; ++j) {
        double xo[3] = {0, 0, 0}, u[3] = {0, 0, 0}, pos[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) xo[i] += g.Q[i * d + k] * hx[j * d + k];
        for (int i = 0; i < d; ++i) {
            double sv = 0;
            for (int k = 0; k < d; ++k) sv += g.Rinv[i * d + k] * xo[k];
            double f = sv - std::floor(sv);
            if (f >= 1.0) f = 0.0;
            u[i] = f;
            tu[size_t(j) * d + i] = f;
            tsh[size_t(j) * d + i] = std::nearbyint(f - sv);  // pos = Q x + R shift
        }
        int64_t c[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) {
            for (int k = i; k < d; ++k) pos[i] += g.R[i * d + k] * u[k];
            const int64_t cmax = int64_t(g.nroot[i]) << depth;
            c[i] = std::min<int64_t>(cmax - 1, std::max<int64_t>(0, int64_t(std::floor((pos[i] - g.lo[i]) * cscale))));
        }
        const int B = t.locate(depth, c);
        if (B < 0) { ++bad; continue; }
        leaf[j] = B;
        // a source that is this very point: an original copy (not an image) in the leaf with
        // bitwise-equal fractional coordinates
        for (int64_t s = t.src_begin[B]; s < t.src_end[B]; ++s) {
            if (!plan->h_src_is_orig[size_t(s)]) continue;
            const int64_t o = plan->h_src_orig[size_t(s)];
            bool eq = true;
            for (int i = 0; i < d; ++i) eq &= plan->h_u[size_t(o) * d + i] == u[i];
            if (eq) {
                selfp[j] = int(o);
                break;
            }
        }
        int a = B;
        while (a >= 0 && !(size_t(a) < full.size() && full[a])) a = t.parent[a];
        int v = B;
        if (a < 0) {
            while (t.parent[v] >= 0) v = t.parent[v];  // the root box
        } else if (a != B) {
            while (t.parent[v] != a) v = t.parent[v];  // A's child on the path
        }
        vb[j] = v;
        ab[j] = a;
    }
    if (bad) return PDMK_ERR_INTERNAL;
    // evaluation order: by (virtual leaf, real leaf), then by target index
    std::vector<int64_t> ord(static_cast<size_t>(m));
    std::iota(ord.begin(), ord.end(), int64_t(0));
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
        return vb[x] != vb[y] ? vb[x] < vb[y] : leaf[x] < leaf[y];
    });
    TargetLayout& L = *out;
    L.m = m;
    L.tgt4.assign(size_t(m) * 4 * ts, 0);
    L.tgt4a.assign(size_t(m) * 4 * ts, 0);
    L.t_dq.assign(size_t(m) * 4 * ts, 0);
    L.tgt_lo.assign(mixed ? size_t(m) * 4 : 0, 0.0f);
    L.t_g0.resize(static_cast<size_t>(m));
    L.self_w.resize(static_cast<size_t>(m));
    L.self_pt.resize(static_cast<size_t>(m));
    L.tgt_orig.resize(static_cast<size_t>(m));
    auto put = [&](std::vector<unsigned char>& buf, size_t idx, double v) {
        if (mixed) { float f = float(v); std::memcpy(&buf[idx * 4], &f, 4); }
        else std::memcpy(&buf[idx * 8], &v, 8);
    };
    // coordinates relative to a box centre, formed in the caller's frame (as the sources'):
    // Q (x - Q^T (c_b - R shift))
    auto rel = [&](int64_t j, int b, double* r) {
        double D[3] = {0, 0, 0}, E[3] = {0, 0, 0}, du[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) {
            double sR = 0;
            for (int k = 0; k < d; ++k) sR += g.R[i * d + k] * tsh[size_t(j) * d + k];
            D[i] = t.center[size_t(b) * d + i] - sR;
        }
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) E[i] += g.Q[k * d + i] * D[k];
        for (int a = 0; a < d; ++a) du[a] = hx[j * d + a] - E[a];
        for (int i = 0; i < d; ++i) {
            double sv = 0;
            for (int k = 0; k < d; ++k) sv += g.Q[i * d + k] * du[k];
            r[i] = sv;
        }
    };
    const int fw = plan->w / 2;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        const int64_t j = ord[size_t(k)];
        double r[3];
        // near field: relative to the real leaf (a coincident source then cancels exactly)
        rel(j, leaf[j], r);
        for (int a = 0; a < d; ++a) {
            put(L.tgt4, size_t(k) * 4 + a, r[a]);
            if (mixed) L.tgt_lo[size_t(k) * 4 + a] = float(r[a] - double(float(r[a])));
        }
        if (ab[j] >= 0) {
            rel(j, ab[j], r);
            for (int a = 0; a < d; ++a) put(L.tgt4a, size_t(k) * 4 + a, r[a]);
        }
        int gg[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) {
            const int M = g.M[i];
            const double Mu = M * tu[size_t(j) * d + i];
            int g0 = int(std::ceil(Mu - 0.5 * plan->w));
            const double del = Mu - g0;
            const int key = g0 + fw;
            const int wrap = key >= 0 ? key / M : -((-key + M - 1) / M);
            g0 -= wrap * M;
            gg[i] = ((g0 % M) + M) % M;
            put(L.t_dq, size_t(k) * 4 + i, del);
        }
        L.t_g0[size_t(k)] = make_int4(gg[0], gg[1], gg[2], 0);
        const double h = g.rc / double(1LL << t.level[vb[j]]);
        L.self_w[size_t(k)] = (d == 3) ? plan->kt.self_coef / h : plan->kt.self_coef - std::log(h) / (2.0 * kPi);
        L.self_pt[size_t(k)] = selfp[j];
        L.tgt_orig[size_t(k)] = int(j);
    }
    // near-field descriptors: one group per (virtual leaf, real leaf), the virtual leaf's
    // list, shifts into the real leaf's frame; groups cut to 32 targets for the warp kernel
    std::vector<int> lst, lsh;
    for (int64_t k0 = 0; k0 < m;) {
        const int64_t j0 = ord[size_t(k0)];
        int64_t k1 = k0;
        while (k1 < m && vb[ord[size_t(k1)]] == vb[j0] && leaf[ord[size_t(k1)]] == leaf[j0]) ++k1;
        const int v = vb[j0], B = leaf[j0];
        box_direct_list(t, v, &lst, &lsh);
        const int lb = int(L.ent.size());
        for (size_t li = 0; li < lst.size(); ++li) {
            const int S = lst[li];
            L.ent.push_back(make_int2(int(t.src_begin[S]), int(t.src_end[S] - t.src_begin[S])));
            double du[3] = {0, 0, 0}, sht[3] = {0, 0, 0}, Ln[3] = {0, 0, 0};
            lattice_shift(g, lsh[li], Ln);
            for (int a = 0; a < d; ++a)
                du[a] = plan->h_Cu[size_t(S) * d + a] + Ln[a] - plan->h_Cu[size_t(B) * d + a];
            for (int i = 0; i < d; ++i)
                for (int kk = 0; kk < d; ++kk) sht[i] += g.Q[i * d + kk] * du[kk];
            const size_t e = L.ent.size() - 1;
            L.ent_sh.resize(L.ent.size() * 4 * ts, 0);
            if (mixed) L.ent_shlo.resize(L.ent.size() * 4, 0.0f);
            for (int a = 0; a < d; ++a) {
                put(L.ent_sh, e * 4 + a, sht[a]);
                if (mixed) L.ent_shlo[e * 4 + a] = float(sht[a] - double(float(sht[a])));
            }
        }
        const int cut = plan->near_nh > 0 ? 32 : int(k1 - k0);
        for (int64_t c0 = k0; c0 < k1; c0 += cut) {
            TLeaf tl;
            tl.tgt_begin = int(c0);
            tl.tgt_count = int(std::min<int64_t>(cut, k1 - c0));
            tl.list_begin = lb;
            tl.list_count = int(lst.size());
            tl.level = t.level[v];
            tl.box = v;
            tl.pad0 = tl.pad1 = 0;
            L.desc.push_back(tl);
        }
        k0 = k1;
    }
    if (L.ent.empty()) {  // keep the device pointers valid
        L.ent.push_back(make_int2(0, 0));
        L.ent_sh.assign(4 * ts, 0);
        if (mixed) L.ent_shlo.assign(4, 0.0f);
    }
    // local-expansion evaluation: runs of equal box A in evaluation order
    for (int64_t k0 = 0; k0 < m;) {
        const int a = ab[ord[size_t(k0)]];
        int64_t k1 = k0;
        while (k1 < m && ab[ord[size_t(k1)]] == a) ++k1;
        if (a >= 0) L.evl.push_back(make_int4(plan->pw.lslot[a], int(k0), int(k1 - k0), t.level[a]));
        k0 = k1;
    }
    return PDMK_OK;
}

template <typename T, int D>
static int run_eval_targets(pdmk_plan plan, const TargetLayout& L, char* buf, double* dp, double* dg) {
    cudaStream_t s = plan->ws;
    const Geometry& g = plan->g;
    const int64_t m = L.m;
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    const size_t ts = sizeof(T);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = buf + off;
        off += align256(std::max<size_t>(bytes, 1));
        return static_cast<void*>(p);
    };
    auto up = [&](void* dst, const void* src, size_t bytes) -> int {
        if (bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return PDMK_OK;
    };
    T* tgt4 = static_cast<T*>(take(size_t(m) * 4 * ts));
    T* tgt4a = static_cast<T*>(take(size_t(m) * 4 * ts));
    float* tgt_lo = static_cast<float*>(take(size_t(m) * 4 * 4));
    int4* t_g0 = static_cast<int4*>(take(size_t(m) * sizeof(int4)));
    T* t_dq = static_cast<T*>(take(size_t(m) * 4 * ts));
    double* self_w = static_cast<double*>(take(size_t(m) * 8));
    int* self_pt = static_cast<int*>(take(size_t(m) * 4));
    int* tgt_orig = static_cast<int*>(take(size_t(m) * 4));
    double* q_tgt = static_cast<double*>(take(size_t(m) * 8));
    double* pot_near = static_cast<double*>(take(size_t(m) * 8));
    double* grad_near = static_cast<double*>(take(size_t(m) * D * 8));
    double* pot_pw = static_cast<double*>(take(size_t(m) * 8));
    double* grad_pw = static_cast<double*>(take(size_t(m) * D * 8));
    double* pot_far = static_cast<double*>(take(size_t(m) * 8));
    double* gradu_far = static_cast<double*>(take(size_t(m) * D * 8));
    TLeaf* desc = static_cast<TLeaf*>(take(L.desc.size() * sizeof(TLeaf)));
    int2* ent = static_cast<int2*>(take(L.ent.size() * sizeof(int2)));
    T* ent_sh = static_cast<T*>(take(L.ent_sh.size()));
    float* ent_shlo = static_cast<float*>(take(L.ent_shlo.size() * 4));
    int4* evl = static_cast<int4*>(take(L.evl.size() * sizeof(int4)));
    int r;
    if ((r = up(tgt4, L.tgt4.data(), L.tgt4.size()))) return r;
    if ((r = up(tgt4a, L.tgt4a.data(), L.tgt4a.size()))) return r;
    if ((r = up(tgt_lo, L.tgt_lo.data(), L.tgt_lo.size() * 4))) return r;
    if ((r = up(t_g0, L.t_g0.data(), L.t_g0.size() * sizeof(int4)))) return r;
    if ((r = up(t_dq, L.t_dq.data(), L.t_dq.size()))) return r;
    if ((r = up(self_w, L.self_w.data(), L.self_w.size() * 8))) return r;
    if ((r = up(self_pt, L.self_pt.data(), L.self_pt.size() * 4))) return r;
    if ((r = up(tgt_orig, L.tgt_orig.data(), L.tgt_orig.size() * 4))) return r;
    if ((r = up(desc, L.desc.data(), L.desc.size() * sizeof(TLeaf)))) return r;
    if ((r = up(ent, L.ent.data(), L.ent.size() * sizeof(int2)))) return r;
    if ((r = up(ent_sh, L.ent_sh.data(), L.ent_sh.size()))) return r;
    if ((r = up(ent_shlo, L.ent_shlo.data(), L.ent_shlo.size() * 4))) return r;
    if ((r = up(evl, L.evl.data(), L.evl.size() * sizeof(int4)))) return r;
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, int64_t(plan->nsm) * 8)));
    // sources' side: the far-field grid and the stored local expansions
    if ((r = far_grid<T, D>(plan, s, false))) return r;
    for (int ph = 0; ph < kPwPhases - 1; ++ph)  // every phase but the evaluation at leaf targets
        if ((r = pw_eval(&plan->pw, s, ph)) != PDMK_OK) return r;
    // far field at the targets
    {
        InterpArgs<T> ia;
        ia.grid = static_cast<const T*>(plan->d_grid);
        ia.t_g0 = t_g0;
        ia.t_dq = t_dq;
        ia.nt = int(m);
        ia.M0 = g.M[0]; ia.M1 = g.M[1]; ia.M2 = g.M[2];
        ia.w = plan->w;
        ia.half_w_inv2 = T(4.0 / (double(plan->w) * plan->w));
        ia.coefW = static_cast<const T*>(plan->d_coefW);
        ia.coefWd = static_cast<const T*>(plan->d_coefWd);
        ia.nW = int(plan->cW.size());
        ia.nWd = int(plan->cWd.size());
        ia.pot = pot_far;
        ia.gradu = gradu_far;
        const size_t smem = sizeof(T) * 128 * 2 * D * plan->w;
        CK(cudaFuncSetAttribute(k_interp<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_interp<T, D><<<int((m + 127) / 128), 128, smem, s>>>(ia);
        CK(cudaGetLastError());
    }
    // plane-wave part: the stored local expansions at the targets
    CK(cudaMemsetAsync(pot_pw, 0, size_t(m) * 8, s));
    CK(cudaMemsetAsync(grad_pw, 0, size_t(m) * D * 8, s));
    if ((r = pw_eval_points(&plan->pw, s, evl, int(L.evl.size()), tgt4a, pot_pw, grad_pw)) != PDMK_OK) return r;
    // residual direct sum over each virtual leaf's neighbourhood
    CK(cudaMemsetAsync(pot_near, 0, size_t(m) * 8, s));
    CK(cudaMemsetAsync(grad_near, 0, size_t(m) * D * 8, s));
    if (!L.desc.empty()) {
        NearArgs<T> na{};
        na.tleaf = desc;
        na.ntleaf = int(L.desc.size());
        na.list = nullptr;
        na.box_src_begin = plan->d_box_src_begin;
        na.box_src_count = plan->d_box_src_count;
        na.box_center = plan->d_box_center;
        na.src4 = static_cast<const T*>(plan->d_src4);
        na.tgt4 = tgt4;
        na.pot = pot_near;
        na.grad = grad_near;
        na.inv_rc = 1.0 / g.rc;
        na.coefA = static_cast<const T*>(plan->d_coefA);
        na.coefB = static_cast<const T*>(plan->d_coefB);
        na.nA = int(plan->cA.size());
        na.nB = int(plan->cB.size());
        na.count_in = nullptr;
        na.src_lo = static_cast<const T*>(plan->d_src_lo);
        na.tgt_lo = reinterpret_cast<const T*>(tgt_lo);
        na.close_s = T(0.04);  // r < 0.2 h
        na.ent = ent;
        na.ent_sh = ent_sh;
        na.ent_shlo = reinterpret_cast<const T*>(ent_shlo);
        near_coefs(plan, &na);
        near_launch<T, D>(plan, na, int(L.desc.size()), s);
        CK(cudaGetLastError());
    }
    (void)mixed;
    // assembly in the caller's order
    k_self_charges<<<blocks, 256, 0, s>>>(m, self_pt, plan->d_q_user, q_tgt);
    CK(cudaGetLastError());
    AssembleArgs aa;
    aa.nt = m;
    aa.d = D;
    aa.tgt_orig = tgt_orig;
    aa.self_w = self_w;
    aa.q_tgt = q_tgt;
    aa.pot_near = pot_near;
    aa.grad_near = grad_near;
    aa.pot_pw = pot_pw;
    aa.grad_pw = grad_pw;
    aa.pot_far = pot_far;
    aa.gradu_far = gradu_far;
    aa.qsum = plan->d_qsums;
    aa.mean_coef = plan->kt.rhat0 * g.rc * g.rc / g.V;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            aa.G[i * D + j] = g.Rinv[j * D + i] * g.M[j];
            aa.Qt[i * D + j] = g.Q[j * D + i];
        }
    aa.pot_out = dp;
    aa.grad_out = dg;
    aa.out_first = 0;
    k_assemble<D, T><<<blocks, 256, 0, s>>>(aa);
    CK(cudaGetLastError());
    return PDMK_OK;
}

extern "C" int pdmk_eval_targets(pdmk_plan plan, int64_t m, const double* x, double* pot, double* grad, int where) {
    if (!plan || m < 0 || (m > 0 && (!x || !pot))) return PDMK_ERR_BAD_ARG;
    if (where != PDMK_HOST && where != PDMK_DEVICE) return PDMK_ERR_BAD_ARG;
    if (!plan->ready) return PDMK_ERR_NOT_READY;
    if (m == 0) return PDMK_OK;
    if (m >= (int64_t(1) << 30)) return PDMK_ERR_TOO_LARGE;
    if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
        *plan->pw.h_err = 0;
        return PDMK_ERR_TIMEOUT;
    }
    const int d = plan->d;
    std::vector<double> hx(size_t(m) * d);
    if (where == PDMK_DEVICE) {
        CK(cudaStreamSynchronize(plan->stream));
        CK(cudaMemcpy(hx.data(), x, hx.size() * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(hx.data(), x, hx.size() * sizeof(double));
    }
    for (double v : hx)
        if (!std::isfinite(v)) return PDMK_ERR_NONFINITE;
    int r = ensure_host_copies(plan);
    if (r != PDMK_OK) return r;
    TargetLayout L;
    r = build_target_layout(plan, m, hx.data(), &L);
    if (r != PDMK_OK) return r;
    // device scratch for this call (kept and reused while large enough)
    const size_t ts = tsize(plan);
    size_t need = 0;
    auto add = [&](size_t b) { need += align256(std::max<size_t>(b, 1)); };
    for (int k = 0; k < 3; ++k) add(size_t(m) * 4 * ts);  // tgt4, tgt4a, (t_dq below)
    add(size_t(m) * 16);                                   // tgt_lo
    add(size_t(m) * sizeof(int4));                         // t_g0
    add(size_t(m) * 8);                                    // self_w
    add(size_t(m) * 4);                                    // self_pt
    add(size_t(m) * 4);                                    // tgt_orig
    add(size_t(m) * 8);                                    // q_tgt
    for (int k = 0; k < 3; ++k) { add(size_t(m) * 8); add(size_t(m) * d * 8); }  // near, pw, far
    add(L.desc.size() * sizeof(TLeaf));
    add(L.ent.size() * sizeof(int2));
    add(L.ent_sh.size());
    add(L.ent_shlo.size() * 4);
    add(L.evl.size() * sizeof(int4));
    const size_t out_bytes = where == PDMK_DEVICE ? 0 : size_t(m) * (1 + d) * 8;
    need += align256(out_bytes + 1);
    if (need > plan->tq_cap) {
        CK(cudaStreamSynchronize(plan->ws));
        if (plan->tq_buf) cudaFree(plan->tq_buf);
        plan->tq_buf = nullptr;
        plan->tq_cap = 0;
        if (cudaMalloc(&plan->tq_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return PDMK_ERR_OOM;
        }
        plan->tq_cap = need;
    }
    char* buf = static_cast<char*>(plan->tq_buf);
    double* dp = pot;
    double* dg = grad;
    if (where != PDMK_DEVICE) {
        dp = reinterpret_cast<double*>(buf + need - align256(out_bytes + 1));
        dg = grad ? dp + m : nullptr;
    }
    CK(cudaEventRecord(plan->ev_fork, plan->stream));
    CK(cudaStreamWaitEvent(plan->ws, plan->ev_fork, 0));
    const bool saved_profile = plan->opts.profile != 0;
    plan->opts.profile = 0;  // eager launches, no stage events
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    if (d == 2)
        r = mixed ? run_eval_targets<float, 2>(plan, L, buf, dp, dg) : run_eval_targets<double, 2>(plan, L, buf, dp, dg);
    else
        r = mixed ? run_eval_targets<float, 3>(plan, L, buf, dp, dg) : run_eval_targets<double, 3>(plan, L, buf, dp, dg);
    plan->opts.profile = saved_profile ? 1 : 0;
    if (r != PDMK_OK) return r;
    if (where != PDMK_DEVICE) {
        CK(cudaMemcpyAsync(pot, dp, size_t(m) * sizeof(double), cudaMemcpyDeviceToHost, plan->ws));
        if (grad) CK(cudaMemcpyAsync(grad, dg, size_t(m) * d * sizeof(double), cudaMemcpyDeviceToHost, plan->ws));
        CK(cudaStreamSynchronize(plan->ws));
        if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
            *plan->pw.h_err = 0;
            return PDMK_ERR_TIMEOUT;
        }
    }
    CK(cudaEventRecord(plan->ev_join, plan->ws));
    CK(cudaStreamWaitEvent(plan->stream, plan->ev_join, 0));
    return PDMK_OK;
}

// ---------------------------------------------------------------------------------------
// Quasi-periodic (Bloch) evaluation at the plan's points (Sec. 3.7); kernels and the reading
// of the method in k_bloch.cuh.  Buffers are made on the first call after pdmk_set_sources.
namespace {
struct BlochBufs {
    double *disp, *y, *tdisp, *beta, *gre, *gim, *cg, *w, *tre, *tim, *res;
};
// sub-buffers start on 256-byte boundaries (the complex grid needs at least 16 for cuFFT)
size_t pad32(size_t v) { return (v + 31) & ~size_t(31); }
BlochBufs bloch_layout(pdmk_plan plan) {
    BlochBufs b;
    const int d = plan->d;
    double* p = plan->bl_buf;
    b.disp = p; p += pad32(size_t(plan->nimg) * d);
    b.y = p; p += pad32(size_t(plan->n) * d);
    b.tdisp = p; p += pad32(size_t(plan->ntgt) * d);
    b.beta = p; p += 32;
    b.gre = p; p += pad32(size_t(plan->ncell));
    b.gim = p; p += pad32(size_t(plan->ncell));
    b.cg = p; p += pad32(2 * size_t(plan->ncell));
    b.w = p; p += pad32(size_t(plan->ncell));
    b.tre = p; p += pad32(size_t(plan->ncell));
    b.tim = p; p += pad32(size_t(plan->ncell));
    b.res = p;  // 6 x (ntgt + ntgt d): near, plane-wave and far parts, real and imaginary
    return b;
}
size_t bloch_doubles(pdmk_plan plan) {
    const int d = plan->d;
    return pad32(size_t(plan->nimg) * d) + pad32(size_t(plan->n) * d) + pad32(size_t(plan->ntgt) * d) + 32 +
           5 * pad32(size_t(plan->ncell)) + pad32(2 * size_t(plan->ncell)) + 6 * size_t(plan->ntgt) * (1 + d);
}
}  // namespace

static int bloch_setup(pdmk_plan plan) {
    if (plan->bl_ready) return PDMK_OK;
    const int d = plan->d;
    const Geometry& g = plan->g;
    int r = ensure_host_copies(plan);
    if (r != PDMK_OK) return r;
    double* p = nullptr;
    r = dalloc(plan, plan->src_allocs, &p, bloch_doubles(plan));
    if (r != PDMK_OK) return r;
    plan->bl_buf = p;
    BlochBufs b = bloch_layout(plan);
    std::vector<double> tdisp(size_t(plan->ntgt) * d);
    // the copy of each target's own point: the original's position in the sorted sources
    {
        std::vector<int64_t> copy_of(static_cast<size_t>(plan->n), -1);
        for (int64_t j = 0; j < plan->nimg; ++j)
            if (plan->h_src_is_orig[size_t(j)]) copy_of[size_t(plan->h_src_orig[size_t(j)])] = j;
        std::vector<int> torig(static_cast<size_t>(plan->ntgt));
        CK(cudaMemcpy(torig.data(), plan->d_tgt_orig, torig.size() * sizeof(int), cudaMemcpyDeviceToHost));
        for (int64_t t = 0; t < plan->ntgt; ++t) {
            const int64_t j = copy_of[size_t(torig[size_t(t)])];
            for (int a = 0; a < d; ++a) tdisp[size_t(t) * d + a] = j >= 0 ? plan->h_src_disp[size_t(j) * d + a] : 0.0;
        }
    }
    CK(cudaMemcpy(b.disp, plan->h_src_disp.data(), plan->h_src_disp.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.y, plan->h_y.data(), plan->h_y.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b.tdisp, tdisp.data(), tdisp.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (!plan->bl_tab) {
        // the smoothing transform's quadrature (hat-w(x) = sum glw cos(x glx)) and the window's
        // transform at every index of each axis
        std::vector<double> tab;
        const KernelTables& kt = plan->kt;
        for (size_t i = 0; i < kt.gl_x.size(); ++i) tab.push_back(kt.gl_x[i]);
        for (size_t i = 0; i < kt.gl_x.size(); ++i) tab.push_back(kt.gl_w[i] * kt.gl_psi[i] / kt.psi.c0);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < g.M[i]; ++j) {
                const int m = j <= g.M[i] / 2 ? j : j - g.M[i];
                tab.push_back(plan->wt.ft(double(m) / g.M[i]));
            }
        double* t = nullptr;
        if ((r = dalloc(plan, plan->plan_allocs, &t, tab.size())) != PDMK_OK) return r;
        CK(cudaMemcpy(t, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
        plan->bl_tab = t;
    }
    if (!plan->bl_have_fft) {
        cufftResult fr = d == 2 ? cufftPlan2d(&plan->bl_fft, g.M[1], g.M[0], CUFFT_Z2Z)
                                : cufftPlan3d(&plan->bl_fft, g.M[2], g.M[1], g.M[0], CUFFT_Z2Z);
        if (fr != CUFFT_SUCCESS) {
            plan_set_msg(plan, "cufft plan failure");
            return PDMK_ERR_CUDA;
        }
        plan->bl_have_fft = true;
    }
    CKFFT(cufftSetStream(plan->bl_fft, plan->ws));
    plan->bl_ready = true;
    return PDMK_OK;
}

template <typename T, int D>
static int run_eval_bloch(pdmk_plan plan, const double* beta_host, double* dp, double* dg) {
    cudaStream_t s = plan->ws;
    const Geometry& g = plan->g;
    int r;
    if ((r = bloch_setup(plan)) != PDMK_OK) return r;
    BlochBufs b = bloch_layout(plan);
    const int64_t nt = plan->ntgt;
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((std::max(plan->nimg, plan->ncell) + 255) / 256,
                                                                  int64_t(plan->nsm) * 16)));
    CK(cudaMemcpyAsync(b.beta, beta_host, D * sizeof(double), cudaMemcpyHostToDevice, s));
    // weights at the shifted modes
    {
        BlochWeightArgs wa;
        wa.d = D;
        wa.M0 = g.M[0]; wa.M1 = g.M[1]; wa.M2 = g.M[2];
        for (int i = 0; i < D * D; ++i) wa.Rinv[i] = g.Rinv[i];
        for (int i = 0; i < 3; ++i) {
            wa.beta_o[i] = 0;
            if (i < D)
                for (int k = 0; k < D; ++k) wa.beta_o[i] += g.Q[i * D + k] * beta_host[k];
        }
        wa.rc = g.rc;
        wa.c = plan->c;
        wa.V = g.V;
        wa.ngl = int(plan->kt.gl_x.size());
        wa.glx = plan->bl_tab;
        wa.glw = plan->bl_tab + wa.ngl;
        wa.ph = plan->bl_tab + 2 * wa.ngl;
        k_bloch_weights<<<blocks, 256, 0, s>>>(wa, b.w);
        CK(cudaGetLastError());
    }
    double* res = b.res;
    const size_t sp = size_t(nt), sg = size_t(nt) * D;
    double* pn[2] = {res, res + sp};
    double* gn[2] = {res + 2 * sp, res + 2 * sp + sg};
    double* pp[2] = {res + 2 * sp + 2 * sg, res + 3 * sp + 2 * sg};
    double* gp[2] = {res + 4 * sp + 2 * sg, res + 4 * sp + 3 * sg};
    double* pf[2] = {res + 4 * sp + 4 * sg, res + 5 * sp + 4 * sg};
    double* gf[2] = {res + 6 * sp + 4 * sg, res + 6 * sp + 5 * sg};
    T* src4 = static_cast<T*>(plan->d_src4);
    T* sdq = static_cast<T*>(plan->d_pt_dq);
    for (int part = 0; part < 2; ++part) {
        k_bloch_charges<T><<<blocks, 256, 0, s>>>(part, D, plan->d_q_user, b.beta, plan->nimg, plan->d_src_orig,
                                                   b.disp, src4, plan->nspread, plan->d_spread_orig, b.y, sdq,
                                                   plan->ntgt, plan->d_tgt_orig, static_cast<T*>(plan->d_tgt4));
        CK(cudaGetLastError());
        // far field: spread this part of the complex strengths
        if ((r = spread_fold<T, D>(plan, s, part == 0 ? b.gre : b.gim, false))) return r;
        // near field with this part of the phased copies: plane waves and the residual sum
        for (int ph = 0; ph < kPwPhases; ++ph)
            if ((r = pw_eval(&plan->pw, s, ph)) != PDMK_OK) return r;
        if (plan->pw.active) {
            CK(cudaMemcpyAsync(pp[part], plan->pw.d_pot, sp * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(gp[part], plan->pw.d_grad, sg * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        CK(cudaMemsetAsync(pn[part], 0, sp * sizeof(double), s));
        CK(cudaMemsetAsync(gn[part], 0, sg * sizeof(double), s));
        if (plan->nnear > 0) {
            NearArgs<T> na{};
            na.tleaf = plan->d_tleaf;
            na.ntleaf = plan->nnear;
            na.list = plan->d_list;
            na.box_src_begin = plan->d_box_src_begin;
            na.box_src_count = plan->d_box_src_count;
            na.box_center = plan->d_box_center;
            na.src4 = src4;
            na.tgt4 = static_cast<const T*>(plan->d_tgt4);
            na.pot = pn[part];
            na.grad = gn[part];
            na.inv_rc = 1.0 / g.rc;
            na.coefA = static_cast<const T*>(plan->d_coefA);
            na.coefB = static_cast<const T*>(plan->d_coefB);
            na.nA = int(plan->cA.size());
            na.nB = int(plan->cB.size());
            na.count_in = nullptr;
            na.src_lo = static_cast<const T*>(plan->d_src_lo);
            na.tgt_lo = static_cast<const T*>(plan->d_tgt_lo);
            na.close_s = T(0.04);
            na.ent = plan->d_ent;
            na.ent_sh = static_cast<const T*>(plan->d_ent_sh);
            na.ent_shlo = static_cast<const T*>(plan->d_ent_shlo);
            near_coefs(plan, &na);
            near_launch<T, D>(plan, na, plan->nnear, s);
            CK(cudaGetLastError());
        }
    }
    // the smooth part: complex transform, scaling at k_m + beta, inverse, interpolation
    k_bloch_interleave<<<blocks, 256, 0, s>>>(b.gre, b.gim, b.cg, plan->ncell);
    CK(cudaGetLastError());
    CKFFT(cufftExecZ2Z(plan->bl_fft, (cufftDoubleComplex*)b.cg, (cufftDoubleComplex*)b.cg, CUFFT_FORWARD));
    k_bloch_scale<<<blocks, 256, 0, s>>>(b.cg, b.w, plan->ncell);
    CK(cudaGetLastError());
    CKFFT(cufftExecZ2Z(plan->bl_fft, (cufftDoubleComplex*)b.cg, (cufftDoubleComplex*)b.cg, CUFFT_INVERSE));
    T* tre = reinterpret_cast<T*>(b.tre);
    T* tim = reinterpret_cast<T*>(b.tim);
    k_bloch_deinterleave<T><<<blocks, 256, 0, s>>>(b.cg, tre, tim, plan->ncell);
    CK(cudaGetLastError());
    for (int part = 0; part < 2 && nt > 0; ++part) {
        InterpArgs<T> ia;
        ia.grid = part == 0 ? tre : tim;
        ia.t_g0 = plan->d_t_g0;
        ia.t_dq = static_cast<const T*>(plan->d_t_dq);
        ia.nt = int(nt);
        ia.M0 = g.M[0]; ia.M1 = g.M[1]; ia.M2 = g.M[2];
        ia.w = plan->w;
        ia.half_w_inv2 = T(4.0 / (double(plan->w) * plan->w));
        ia.coefW = static_cast<const T*>(plan->d_coefW);
        ia.coefWd = static_cast<const T*>(plan->d_coefWd);
        ia.nW = int(plan->cW.size());
        ia.nWd = int(plan->cWd.size());
        ia.pot = pf[part];
        ia.gradu = gf[part];
        const size_t smem = sizeof(T) * 128 * 2 * D * plan->w;
        CK(cudaFuncSetAttribute(k_interp<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_interp<T, D><<<int((nt + 127) / 128), 128, smem, s>>>(ia);
        CK(cudaGetLastError());
    }
    // the plan's own (real) charges again for later evaluations
    if ((r = set_charges_device(plan, false)) != PDMK_OK) return r;
    BlochAssembleArgs aa;
    aa.nt = nt;
    aa.tgt_orig = plan->d_tgt_orig;
    aa.self_w = plan->d_self_w;
    aa.q = plan->d_q_user;
    aa.tdisp = b.tdisp;
    aa.y = b.y;
    aa.beta = b.beta;
    for (int part = 0; part < 2; ++part) {
        aa.pn[part] = pn[part];
        aa.gn[part] = gn[part];
        aa.pp[part] = plan->pw.active ? pp[part] : nullptr;
        aa.gp[part] = plan->pw.active ? gp[part] : nullptr;
        aa.pf[part] = pf[part];
        aa.gf[part] = gf[part];
    }
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            aa.G[i * D + j] = g.Rinv[j * D + i] * g.M[j];
            aa.Qt[i * D + j] = g.Q[j * D + i];
        }
    aa.pot_out = dp;
    aa.grad_out = dg;
    aa.out_first = plan->out_first;
    k_assemble_bloch<D><<<blocks, 256, 0, s>>>(aa);
    CK(cudaGetLastError());
    return PDMK_OK;
}

extern "C" int pdmk_eval_bloch(pdmk_plan plan, const double* beta, double* pot, double* grad, int where) {
    if (!plan || !beta || !pot) return PDMK_ERR_BAD_ARG;
    if (where != PDMK_HOST && where != PDMK_DEVICE) return PDMK_ERR_BAD_ARG;
    if (!plan->ready) return PDMK_ERR_NOT_READY;
    const int d = plan->d;
    for (int a = 0; a < d; ++a)
        if (!std::isfinite(beta[a])) return PDMK_ERR_NONFINITE;
    {
        // beta must not be a reciprocal-lattice vector (the periodic case, where k = 0 is singular)
        const Geometry& g = plan->g;
        double bo[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) bo[i] += g.Q[i * d + k] * beta[k];
        bool integral = true;
        for (int i = 0; i < d; ++i) {
            double mi = 0;  // beta = 2 pi R^{-T} m  <=>  m = R^T beta / (2 pi)
            for (int k = 0; k < d; ++k) mi += g.R[k * d + i] * bo[k];
            mi /= 2.0 * kPi;
            integral &= std::fabs(mi - std::nearbyint(mi)) < 1e-9;
        }
        if (integral) {
            plan_set_msg(plan, "beta is a reciprocal-lattice vector: use pdmk_eval (periodic)");
            return PDMK_ERR_BAD_ARG;
        }
    }
    if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
        *plan->pw.h_err = 0;
        return PDMK_ERR_TIMEOUT;
    }
    const int64_t m = plan->n_out;
    double* dp = pot;
    double* dg = grad;
    double* stage = nullptr;
    if (where != PDMK_DEVICE) {
        if (cudaMalloc(&stage, sizeof(double) * size_t(std::max<int64_t>(m, 1)) * 2 * (1 + d)) != cudaSuccess) {
            cudaGetLastError();
            return PDMK_ERR_OOM;
        }
        dp = stage;
        dg = grad ? stage + 2 * m : nullptr;
    }
    CK(cudaEventRecord(plan->ev_fork, plan->stream));
    CK(cudaStreamWaitEvent(plan->ws, plan->ev_fork, 0));
    const bool saved_profile = plan->opts.profile != 0, saved_count = plan->count_pending;
    plan->opts.profile = 0;
    plan->count_pending = false;
    const bool mixed = plan->opts.precision == PDMK_MIXED;
    int r;
    if (d == 2) r = mixed ? run_eval_bloch<float, 2>(plan, beta, dp, dg) : run_eval_bloch<double, 2>(plan, beta, dp, dg);
    else r = mixed ? run_eval_bloch<float, 3>(plan, beta, dp, dg) : run_eval_bloch<double, 3>(plan, beta, dp, dg);
    plan->opts.profile = saved_profile ? 1 : 0;
    plan->count_pending = saved_count;
    if (r == PDMK_OK && where != PDMK_DEVICE) {
        if (cudaMemcpyAsync(pot, dp, size_t(m) * 2 * sizeof(double), cudaMemcpyDeviceToHost, plan->ws) != cudaSuccess ||
            (grad && cudaMemcpyAsync(grad, dg, size_t(m) * 2 * d * sizeof(double), cudaMemcpyDeviceToHost,
                                     plan->ws) != cudaSuccess) ||
            cudaStreamSynchronize(plan->ws) != cudaSuccess)
            r = PDMK_ERR_CUDA;
        if (r == PDMK_OK && plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
            *plan->pw.h_err = 0;
            r = PDMK_ERR_TIMEOUT;
        }
    }
    if (stage) {
        cudaStreamSynchronize(plan->ws);
        cudaFree(stage);
    }
    if (r != PDMK_OK) return r;
    CK(cudaEventRecord(plan->ev_join, plan->ws));
    CK(cudaStreamWaitEvent(plan->stream, plan->ev_join, 0));
    return PDMK_OK;
}

// ---------------------------------------------------------------------------------------
// Adjoint (vector-Jacobian product) of the evaluation at the sources.  Phi = A q with A
// symmetric (pair kernel, zero-mean constant and self part all even in the separation), so
// for upstream g = dLoss/dPhi:  dLoss/dq = A g  and  dLoss/dy = g grad Phi[q] + q grad Phi[g].
__global__ void k_adjoint_combine(int64_t n, int d, const double* __restrict__ g, const double* __restrict__ q,
                                  const double* __restrict__ grad_q, const double* __restrict__ grad_g,
                                  double* __restrict__ g_y) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * d; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = i / d;
        g_y[i] = g[t] * grad_q[i] + q[t] * grad_g[i];
    }
}

extern "C" int pdmk_eval_adjoint(pdmk_plan plan, const double* g_pot, const double* g_grad, double* g_q, double* g_y,
                                 double* g_x, int where) {
    if (!plan || !g_pot || (!g_q && !g_y && !g_x)) return PDMK_ERR_BAD_ARG;
    if (g_grad) {
        plan_set_msg(plan, "upstream gradients on the returned field need second derivatives of the kernel");
        return PDMK_ERR_BAD_ARG;
    }
    if (!plan->ready) return PDMK_ERR_NOT_READY;
    if (g_x && plan->out_first == 0) {
        plan_set_msg(plan, "the targets are the sources: their derivative is part of g_y");
        return PDMK_ERR_BAD_ARG;
    }
    if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
        *plan->pw.h_err = 0;
        return PDMK_ERR_TIMEOUT;
    }
    // over the plan's points: the sources [0, n_src) and, with separate targets, the targets
    // [n_src, n); the upstream gradient lives on the evaluated points [out_first, n)
    const int64_t n = plan->n, ns = plan->n_src, m = n - ns, first = plan->out_first;
    const int d = plan->d;
    if (n == 0) return PDMK_OK;
    if (!plan->d_adj) {
        double* p = nullptr;
        int rr = dalloc(plan, plan->src_allocs, &p, size_t(n) * (4 + 2 * d));
        if (rr != PDMK_OK) return rr;
        plan->d_adj = p;
    }
    double* q_save = plan->d_adj;
    double* gdev = q_save + n;
    double* pot_q = gdev + n;
    double* pot_g = pot_q + n;
    double* grad_q = pot_g + n;
    double* grad_g = grad_q + n * d;
    const size_t nb = size_t(n) * sizeof(double);
    CK(cudaEventRecord(plan->ev_fork, plan->stream));
    CK(cudaStreamWaitEvent(plan->ws, plan->ev_fork, 0));
    CK(cudaMemcpyAsync(q_save, plan->d_q_user, nb, cudaMemcpyDeviceToDevice, plan->ws));
    CK(cudaMemsetAsync(gdev, 0, nb, plan->ws));
    CK(cudaMemcpyAsync(gdev + first, g_pot, size_t(n - first) * sizeof(double),
                       where == PDMK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, plan->ws));
    // both evaluations run eagerly over every point: the plan's captured graph stays keyed
    // to the caller's outputs of pdmk_eval
    const bool saved_profile = plan->opts.profile != 0, saved_count = plan->count_pending;
    plan->opts.profile = 0;
    plan->count_pending = false;
    int r = launch_eval(plan, pot_q, grad_q, 0);  // grad Phi[q]
    if (r == PDMK_OK) {
        CK(cudaMemcpyAsync(plan->d_q_user, gdev, nb, cudaMemcpyDeviceToDevice, plan->ws));
        r = set_charges_device(plan, false);
    }
    if (r == PDMK_OK) r = launch_eval(plan, pot_g, grad_g, 0);  // Phi[g] = A g, grad Phi[g]
    // the caller's charges again, whatever happened above
    cudaMemcpyAsync(plan->d_q_user, q_save, nb, cudaMemcpyDeviceToDevice, plan->ws);
    const int r2 = set_charges_device(plan, false);
    plan->opts.profile = saved_profile ? 1 : 0;
    plan->count_pending = saved_count;
    if (r != PDMK_OK) return r;
    if (r2 != PDMK_OK) return r2;
    // g grad Phi[q] + q grad Phi[g] at every point, in place (element-wise): the source rows
    // are g_y, the target rows g_x
    if (g_y || g_x) {
        const int blocks = int(std::min<int64_t>((n * d + 255) / 256, int64_t(plan->nsm) * 8));
        k_adjoint_combine<<<std::max(blocks, 1), 256, 0, plan->ws>>>(n, d, gdev, q_save, grad_q, grad_g, grad_q);
        CK(cudaGetLastError());
    }
    const cudaMemcpyKind out_kind = where == PDMK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (g_q) CK(cudaMemcpyAsync(g_q, pot_g, size_t(ns) * sizeof(double), out_kind, plan->ws));
    if (g_y) CK(cudaMemcpyAsync(g_y, grad_q, size_t(ns) * d * sizeof(double), out_kind, plan->ws));
    if (g_x) CK(cudaMemcpyAsync(g_x, grad_q + size_t(ns) * d, size_t(m) * d * sizeof(double), out_kind, plan->ws));
    if (where != PDMK_DEVICE) {
        CK(cudaStreamSynchronize(plan->ws));
        if (plan->pw.h_err && *reinterpret_cast<volatile int*>(plan->pw.h_err)) {
            *plan->pw.h_err = 0;
            return PDMK_ERR_TIMEOUT;
        }
    }
    CK(cudaEventRecord(plan->ev_join, plan->ws));
    CK(cudaStreamWaitEvent(plan->stream, plan->ev_join, 0));
    return PDMK_OK;
}

// ---------------------------------------------------------------------------------------
// Batches of independent cells: one plan per cell, one evaluation of all cells captured into
// a single CUDA graph on the batch's stream (cells run concurrently as independent branches).
struct pdmk_batch_s {
    std::vector<pdmk_plan> plans;
    std::vector<int> d;
    std::vector<int64_t> n, off, yoff;  // per cell: sources, offset of its values, of its rows x d
    int64_t ntot = 0, ytot = 0;
    cudaStream_t stream = nullptr;      // the caller's
    cudaStream_t bs = nullptr;          // the batch's own (graph capture needs a non-default stream)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double* g_pot = nullptr;
    double* g_grad = nullptr;
    double* d_pot = nullptr;   // staging for host outputs
    double* d_grad = nullptr;
    int evals = 0;
    bool ready = false;
};

extern "C" void pdmk_batch_destroy(pdmk_batch b) {
    if (!b) return;
    if (b->bs) cudaStreamSynchronize(b->bs);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (pdmk_plan p : b->plans) pdmk_plan_destroy(p);
    if (b->d_pot) cudaFree(b->d_pot);
    if (b->d_grad) cudaFree(b->d_grad);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->bs) cudaStreamDestroy(b->bs);
    delete b;
}

extern "C" int pdmk_batch_create(int ncells, const int* d, const double* L, const double* eps, const pdmk_opts* opts,
                                 pdmk_batch* out) {
    if (!out) return PDMK_ERR_BAD_ARG;
    *out = nullptr;
    if (ncells <= 0 || !d || !L || !eps) return PDMK_ERR_BAD_ARG;
    pdmk_batch b = new (std::nothrow) pdmk_batch_s();
    if (!b) return PDMK_ERR_OOM;
    pdmk_opts o;
    if (opts) o = *opts; else pdmk_default_opts(&o);
    b->stream = static_cast<cudaStream_t>(o.stream);
    if (cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        pdmk_batch_destroy(b);
        return PDMK_ERR_CUDA;
    }
    size_t loff = 0;
    for (int c = 0; c < ncells; ++c) {
        if (d[c] != 2 && d[c] != 3) {
            pdmk_batch_destroy(b);
            return PDMK_ERR_BAD_ARG;
        }
        pdmk_plan p = nullptr;
        const int r = pdmk_plan_create(d[c], L + loff, eps[c], &o, &p);
        if (r != PDMK_OK) {
            pdmk_batch_destroy(b);
            return r;
        }
        b->plans.push_back(p);
        b->d.push_back(d[c]);
        loff += size_t(d[c]) * d[c];
    }
    *out = b;
    return PDMK_OK;
}

extern "C" int pdmk_batch_set_sources(pdmk_batch b, const int64_t* offsets, const double* y, const double* q,
                                      int where) {
    if (!b || !offsets || offsets[0] != 0) return PDMK_ERR_BAD_ARG;
    pdmk_plan plan = nullptr;
    const int nc = int(b->plans.size());
    b->ready = false;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->evals = 0;
    b->n.assign(nc, 0);
    b->off.assign(nc, 0);
    b->yoff.assign(nc, 0);
    int64_t yo = 0;
    for (int c = 0; c < nc; ++c) {
        if (offsets[c + 1] <= offsets[c]) return PDMK_ERR_BAD_ARG;  // every cell holds sources
        b->n[c] = offsets[c + 1] - offsets[c];
        b->off[c] = offsets[c];
        b->yoff[c] = yo;
        yo += b->n[c] * b->d[c];
    }
    b->ntot = offsets[nc];
    b->ytot = yo;
    for (int c = 0; c < nc; ++c) {
        const int r = pdmk_set_sources(b->plans[c], b->n[c], y ? y + b->yoff[c] : nullptr,
                                       q ? q + b->off[c] : nullptr, where);
        if (r != PDMK_OK) return r;
        b->plans[c]->count_pending = false;  // no pair counting inside a batch evaluation
    }
    if (b->d_pot) cudaFree(b->d_pot);
    if (b->d_grad) cudaFree(b->d_grad);
    b->d_pot = b->d_grad = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&b->d_pot), size_t(std::max<int64_t>(b->ntot, 1)) * sizeof(double)));
    CK(cudaMalloc(reinterpret_cast<void**>(&b->d_grad), size_t(std::max<int64_t>(b->ytot, 1)) * sizeof(double)));
    b->ready = true;
    return PDMK_OK;
}

// every cell's evaluation, forked from and joined to the batch stream
static int batch_launch(pdmk_batch b, double* dp, double* dg) {
    pdmk_plan plan = nullptr;
    CK(cudaEventRecord(b->ev_fork, b->bs));
    for (size_t c = 0; c < b->plans.size(); ++c) {
        pdmk_plan p = b->plans[c];
        if (b->n[c] == 0) continue;
        CK(cudaStreamWaitEvent(p->ws, b->ev_fork, 0));
        const bool saved_profile = p->opts.profile != 0;
        p->opts.profile = 0;
        const int r = launch_eval(p, dp + b->off[c], dg ? dg + b->yoff[c] : nullptr, p->out_first);
        p->opts.profile = saved_profile ? 1 : 0;
        if (r != PDMK_OK) return r;
        CK(cudaEventRecord(p->ev_join, p->ws));
        CK(cudaStreamWaitEvent(b->bs, p->ev_join, 0));
    }
    return PDMK_OK;
}

extern "C" int pdmk_batch_eval(pdmk_batch b, double* pot, double* grad, int where) {
    if (!b || !pot) return PDMK_ERR_BAD_ARG;
    if (!b->ready) return PDMK_ERR_NOT_READY;
    pdmk_plan plan = nullptr;
    for (pdmk_plan p : b->plans)
        if (p->pw.h_err && *reinterpret_cast<volatile int*>(p->pw.h_err)) {
            *p->pw.h_err = 0;
            return PDMK_ERR_TIMEOUT;
        }
    double* dp = where == PDMK_DEVICE ? pot : b->d_pot;
    double* dg = grad ? (where == PDMK_DEVICE ? grad : b->d_grad) : nullptr;
    CK(cudaEventRecord(b->ev_join, b->stream));  // order after the caller's stream
    CK(cudaStreamWaitEvent(b->bs, b->ev_join, 0));
    if (b->evals == 0) {
        const int r = batch_launch(b, dp, dg);  // first evaluation eagerly
        if (r != PDMK_OK) return r;
    } else {
        if (!b->gexec || b->g_pot != dp || b->g_grad != dg) {
            if (b->gexec) cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeThreadLocal));
            const int r = batch_launch(b, dp, dg);
            const cudaError_t ce = cudaStreamEndCapture(b->bs, &graph);
            if (r != PDMK_OK) {
                if (graph) cudaGraphDestroy(graph);
                return r;
            }
            CK(ce);
            const cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            CK(ie);
            b->g_pot = dp;
            b->g_grad = dg;
        }
        CK(cudaGraphLaunch(b->gexec, b->bs));
    }
    ++b->evals;
    if (where != PDMK_DEVICE) {
        CK(cudaMemcpyAsync(pot, dp, size_t(b->ntot) * sizeof(double), cudaMemcpyDeviceToHost, b->bs));
        if (grad) CK(cudaMemcpyAsync(grad, dg, size_t(b->ytot) * sizeof(double), cudaMemcpyDeviceToHost, b->bs));
        CK(cudaStreamSynchronize(b->bs));
        for (pdmk_plan p : b->plans)
            if (p->pw.h_err && *reinterpret_cast<volatile int*>(p->pw.h_err)) {
                *p->pw.h_err = 0;
                return PDMK_ERR_TIMEOUT;
            }
    }
    CK(cudaEventRecord(b->ev_join, b->bs));
    CK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
    return PDMK_OK;
}

extern "C" pdmk_plan pdmk_batch_plan(pdmk_batch b, int cell) {
    if (!b || cell < 0 || cell >= int(b->plans.size())) return nullptr;
    return b->plans[cell];
}
