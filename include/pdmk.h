/*
 * pdmk.h -- C ABI of the B300 periodic DMK library (libpdmk.so).
 *
 * The library evaluates periodic Coulomb lattice sums (paper Eq. (1.1)): for N point
 * charges q_j at y_j in the unit cell spanned by the columns a_1..a_d of L (d = 2 or 3),
 *
 *   Phi(x) = sum_{n in Z^d} sum_j q_j G(x - y_j - L n),
 *   G(r) = -log(r)/(2 pi) (2D),  1/(4 pi r) (3D)          (Eq. (1.2))
 *
 * with the n = 0 self term excluded at a target that coincides with its source, under
 * the tin-foil convention (the k = 0 Fourier mode is zero, Sec. 1).  For non-neutral
 * charges the returned potential is the zero-mean one (uniform neutralising background),
 * so the result is well defined for any charges.  The gradient is grad_x Phi (the field
 * is its negative).
 *
 * The method is the periodic dual-space multilevel kernel splitting of Algorithm 1:
 * the near field G - W_0 by a free-space DMK on the extended root grid (inner block
 * covering the cell plus a one-cube halo of image sources, Sec. 3.3-3.5), and the smooth
 * periodic W_0 by spreading, FFT, diagonal scaling with k = 0 dropped, inverse FFT and
 * interpolation (Sec. 3.6-3.7), followed by the self-interaction correction (Sec. 3.8).
 *
 * Conventions common to all entry points
 *  - Every function returns PDMK_OK (0) or a negative PDMK_ERR_* code; no exception,
 *    abort or trap crosses the ABI.  pdmk_strerror() names a code.
 *  - The caller owns every array it passes.  The plan owns its device buffers.
 *  - Positions are row-major (n x d doubles); L is column-major (column j = a_j).
 *  - `where` says where a pointer lives: PDMK_HOST (pageable or pinned host memory) or
 *    PDMK_DEVICE (device memory of the plan's GPU).
 *  - Work is enqueued on the plan's CUDA stream (pdmk_opts.stream).  With device
 *    pointers pdmk_eval is asynchronous; with host pointers it returns after the results
 *    are in host memory.  A plan must not be used from two threads at once.
 */
#ifndef PDMK_H
#define PDMK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define PDMK_OK 0
#define PDMK_ERR_BAD_ARG (-1)          /* null pointer, d not 2/3, n < 0, bad option   */
#define PDMK_ERR_SINGULAR_LATTICE (-2) /* |det L| <= 1e-14 prod |a_i|                  */
#define PDMK_ERR_NON_NEUTRAL (-3)      /* |sum q| > 1e-12 sum |q| with neutrality = 0  */
#define PDMK_ERR_BAD_EPS (-4)          /* eps outside [1e-12, 1e-2]                     */
#define PDMK_ERR_NONFINITE (-5)        /* NaN or Inf in L, positions or charges         */
#define PDMK_ERR_OOM (-6)              /* device or host allocation failed              */
#define PDMK_ERR_CUDA (-7)             /* a CUDA / cuFFT call failed                    */
#define PDMK_ERR_TIMEOUT (-8)          /* a bounded device wait expired                 */
#define PDMK_ERR_NOT_READY (-9)        /* pdmk_eval before pdmk_set_sources             */
#define PDMK_ERR_INTERNAL (-10)        /* a consistency check inside the library failed */
#define PDMK_ERR_TOO_LARGE (-11)       /* a size exceeds a documented maximum           */

#define PDMK_HOST 0
#define PDMK_DEVICE 1

#define PDMK_FP64 0  /* every stage in FP64                                         */
#define PDMK_MIXED 1 /* FP32 bulk with compensated sums; FP64 set-up, scaling, assembly.
                        FP32 rounding bounds its relative error near 1e-7: for eps below
                        1e-6 use PDMK_FP64 (mixed plans are accepted but do not reach it) */

typedef struct pdmk_plan_s* pdmk_plan;

/* Options.  Zero / negative numeric fields select the defaults noted. */
typedef struct {
    double kappa;   /* root box side r_c = L_min / kappa (Algorithm 1 step 1); <= 0: Table 1 */
    int n_s;        /* leaf capacity (Algorithm 1 step 2); <= 0: Table 1                     */
    int precision;  /* PDMK_FP64 or PDMK_MIXED                                               */
    int window_w;   /* spreading window width in grid points; <= 0: ceil(2 c / pi) + 2,
                       at most 20.  In mixed precision a wider window than the default
                       amplifies FP32 rounding through the deconvolution (FP64 plans only) */
    int n_proxy;    /* Chebyshev proxy points per dimension p; <= 0: from eps                */
    int n_pw;       /* plane-wave half-width K (nodes -K..K per dimension); <= 0: from eps   */
    int max_depth;  /* deepest tree level; < 0: 30; 0: every root box is a leaf              */
    int neutrality; /* 0: require |sum q| <= 1e-12 sum|q|; 1: allow (zero-mean potential)     */
    int profile;    /* 1: record per-stage CUDA-event times (pdmk_stage_times)               */
    void* stream;   /* cudaStream_t for all work; NULL: the legacy default stream            */
    int wait_test;  /* test hook, 0 in normal use.  1: the first dependent item of the
                       single-launch downward pass waits on a flag that nothing sets, so its
                       bounded wait (about 1 s) expires and the evaluation reports
                       PDMK_ERR_TIMEOUT (2D compile-time orders only; no effect elsewhere) */
    int autotune;   /* 0: kappa and n_s from Table 1 (or as given).  1: pdmk_set_sources times
                       candidate (kappa, n_s) pairs around the Table 1 values (those not given
                       explicitly) on the given sources with temporary plans, keeps the fastest
                       evaluation and rebuilds the plan with it (the paper's Sec. 5 sweep of
                       kappa and n_s, done at run time).  The choice, as ratios to the Table 1
                       values, is cached per (d, precision, eps, floor(log2 n)) for the process,
                       so later plans of similar size reuse it without timing.  The chosen values
                       are reported by pdmk_get_info. */
    int root_mode;  /* 0: a cubic (square) cell with an integer kappa >= 3 takes the periodic root
                       of Remark 3.3: the root grid is the cell itself, no image sources are
                       made, and neighbours across the faces are virtual copies shifted by
                       L n, n in {-1, 0, 1}^d (pdmk_get_info reports n_images = n).  Any other
                       cell takes the multi-cube root with its halo of images (Sec. 3.3-3.4).
                       1: always the multi-cube root with images. */
    int build_mode; /* where pdmk_set_sources builds the tree and the per-point records:
                       0: on the device, falling back to the host for inputs the device build
                       does not take (trees deeper than its 64-bit point keys hold, about 16
                       levels in 3D and 25 in 2D, or 2^30 images or more); 1: on the host;
                       2: on the device only (PDMK_ERR_TOO_LARGE otherwise); 3: both, compared
                       array by array (a check of the device build: PDMK_ERR_INTERNAL with
                       pdmk_plan_message naming the first array that differs).  Both builds
                       give the same tree, order and records, bit for bit. */
    int tensor_cores; /* 0: the 3D leaf evaluation of mixed plans (orders 16 and 24) runs on the
                       tensor cores (tcgen05, TF32 with each operand split in two, FP32
                       accumulation: about the accuracy of FP32); 1: on the FP32 FMA pipes. */
} pdmk_opts;

/* Fills *opts with the defaults (all fields "auto", FP64, neutrality allowed). */
void pdmk_default_opts(pdmk_opts* opts);

/*
 * Creates a plan for lattice L (d x d, column-major, host memory) and target relative L2
 * precision eps in [1e-12, 1e-2].  Orients L to upper-triangular form (Sec. 3.2, Eq. (3.4)),
 * picks r_c and n_s, sizes the root grid (Eq. (3.10), (3.12)) and the Fourier grid
 * (Eq. (3.15), each length rounded up to an even size with prime factors <= 13; mixed plans
 * of strongly skewed cells enlarge it further so that FP32 rounding is not amplified by the
 * window deconvolution; pdmk_get_info reports the sizes as M), and computes the prolate
 * tables in FP64.  opts may be NULL (defaults).
 * Errors: BAD_ARG, BAD_EPS, SINGULAR_LATTICE, NONFINITE, CUDA, OOM.
 */
int pdmk_plan_create(int d, const double* L, double eps, const pdmk_opts* opts, pdmk_plan* out);

/*
 * Sets the sources (positions y, n x d; charges q, n) and builds everything that depends on
 * them: fractional wrap, image sources filling the extended domain (Sec. 3.4), the adaptive
 * level-restricted tree and its lists (Algorithm 1 step 2), and the device layouts.  The
 * targets of pdmk_eval are these sources.  Inputs may be freed on return.
 * Errors: BAD_ARG, NONFINITE, NON_NEUTRAL, OOM, CUDA.
 */
int pdmk_set_sources(pdmk_plan plan, int64_t n, const double* y, const double* q, int where);

/*
 * As pdmk_set_sources, with m >= 1 separate targets x (m x d, row-major, the caller's frame;
 * wrapped into the cell like the sources): pdmk_eval then writes the potential and gradient
 * at the m targets (m values, m x d), the sources' field only.  The plan is built on the union
 * of sources and targets, the targets being points of charge 0: they add nothing to any stage
 * and carry no self term, so the cost is that of evaluating the union.  A target that
 * coincides exactly with a source is singular; the pair is skipped.  pdmk_set_charges still
 * takes the n source charges.  Errors: as pdmk_set_sources.
 */
int pdmk_set_sources_targets(pdmk_plan plan, int64_t n, const double* y, const double* q, int64_t m, const double* x,
                             int where);

/*
 * Replaces the charges (n values, the same n and order as pdmk_set_sources) without
 * rebuilding the tree.  Errors: NOT_READY, NONFINITE, NON_NEUTRAL, CUDA.
 */
int pdmk_set_charges(pdmk_plan plan, const double* q, int where);

/*
 * Evaluates the periodic potential (pot, n) and, if grad is not NULL, its gradient
 * (grad, n x d row-major) at every source, self term excluded (Algorithm 1 steps 3-5):
 * near-field DMK, far-field five-step procedure, assembly and self-correction.
 * Outputs are in the caller's source order and frame.  Errors: NOT_READY, CUDA, TIMEOUT.
 * TIMEOUT: a bounded wait of the single-launch downward pass (2D, compile-time orders)
 * expired; the kernel skipped the remaining work and the outputs are invalid, the CUDA
 * context stays usable.  A host evaluation reports it on return; a device evaluation does
 * not synchronise, so its timeout is reported by the next pdmk_eval of the plan.
 */
int pdmk_eval(pdmk_plan plan, double* pot, double* grad, int where);

/*
 * pdmk_eval_targets -- the potential (pot, m values) and, if grad is not NULL, its gradient
 * (grad, m x d row-major) of the plan's sources at m targets x (m x d row-major, the caller's
 * frame; any position: wrapped into the cell since Phi is periodic), evaluated against the
 * tree built by pdmk_set_sources: no rebuild (Algorithm 1 returns Phi at the targets it is
 * given; here the targets may change on every call while the sources stay).
 * Each target is located in the source tree on the host.  Its plane-wave part comes from the
 * deepest box on its path that holds a complete local expansion, and its residual sum runs
 * over the source leaves meeting the neighbourhood of that box's child containing it (the
 * level restriction of Algorithm 1 step 2 makes this the same telescoped interaction as at
 * the plan's own targets); the far field is interpolated at the target.  A target whose
 * wrapped fractional coordinates equal a source's bitwise excludes that source's self term,
 * as pdmk_eval does at the sources.  The plan's charges are those of the last
 * pdmk_set_sources / pdmk_set_charges.  where: PDMK_HOST or PDMK_DEVICE for x, pot and grad.
 * Each call recomputes the sources' far-field grid and local expansions, and keeps an
 * m-sized device scratch (grown on demand, freed by pdmk_set_sources / pdmk_plan_destroy).
 * Ordered after the plan's stream like pdmk_eval; a host call returns after the copies.
 * Errors: BAD_ARG, NOT_READY, NONFINITE, TOO_LARGE (m >= 2^30), OOM, CUDA, TIMEOUT, INTERNAL.
 */
int pdmk_eval_targets(pdmk_plan plan, int64_t m, const double* x, double* pot, double* grad, int where);

/*
 * pdmk_eval_bloch -- the quasi-periodic lattice sum of Sec. 3.7 at the plan's points: for a
 * Bloch wave vector beta (d values, the caller's frame; not a reciprocal-lattice vector, which
 * is the periodic case of pdmk_eval)
 *     Phi(x) = sum_n sum_j q_j e^{i beta.L n} G(x - y_j - L n),   Phi(x + L n) = e^{i beta.L n} Phi(x),
 * self term excluded, no neutrality requirement (every Fourier mode k_m + beta is kept; none
 * vanishes).  Complex results: pot (2 values per point: real, imaginary) and, if grad is not
 * NULL, grad (2 d values per point: for each axis real, imaginary), in the caller's order and
 * frame.  The near field runs the plan's real kernels twice, on the real and imaginary parts
 * of the phased image charges q_j e^{i beta.L n}; the smooth part spreads q_j e^{-i beta.y_j},
 * transforms the full grid (complex, FP64), scales by hat-W_0(|k_m + beta|), transforms back,
 * interpolates and multiplies by e^{i beta.x}.  The first call after pdmk_set_sources makes
 * its buffers (about 7 grid sizes and 12 values per point of FP64, kept until the next
 * pdmk_set_sources).  where as pdmk_eval; the plan's charges are unchanged on return.
 * Errors: BAD_ARG (also beta a reciprocal-lattice vector), NOT_READY, NONFINITE, OOM, CUDA,
 * TIMEOUT.
 */
int pdmk_eval_bloch(pdmk_plan plan, const double* beta, double* pot, double* grad, int where);

/*
 * pdmk_eval_noalloc -- the evaluation of pdmk_eval (device outputs) for callers that cannot
 * allocate device memory at evaluation time: for example code running inside an engine that
 * reserved the whole device heap for its own pool at start-up, or under a caching allocator
 * that forbids cudaMalloc during a time step, or under a real-time budget that cannot absorb
 * an allocation's implicit synchronisation.  The paper has no counterpart; this is a property
 * of the library, not of the method.
 *
 * pot (n) and grad (n x d, or NULL) are device buffers owned by the caller; the plan must have
 * been set up (pdmk_set_sources) beforehand by a caller that could allocate.  The call itself
 * calls no cudaMalloc, cudaFree or allocating library routine: the scratch of the spreading
 * kernel (its per-subproblem padded tiles) is a file-scope static device array of 16 MiB
 * that every device loading the library holds until the process exits.
 *  - Returns PDMK_ERR_TOO_LARGE (and does nothing) if the plan's spreading scratch, roughly
 *    (n / 512 + number of grid bins) x (B + w - 1)^d x element size, exceeds 16 MiB.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    for that device; make that first call outside any stream capture.
 *  - Every call, from every plan, shares the one array: calls whose work overlaps on the GPU
 *    (different streams or plans without ordering between them) race on it.  Calls ordered
 *    on one stream are safe; the array keeps the last call's contents, and nothing in it
 *    needs to start at zero.
 *  - Launches are eager (never replayed from a captured graph) and on the plan's stream
 *    order, asynchronous like pdmk_eval with device pointers.
 * Errors: BAD_ARG, NOT_READY, TOO_LARGE, CUDA, TIMEOUT.  TIMEOUT: as for pdmk_eval; the call
 * does not synchronise, so a bounded wait that expires during it is reported by the plan's
 * next call (pdmk_eval, pdmk_eval_noalloc or pdmk_eval_adjoint), and an expiry left by an
 * earlier evaluation is reported by this call before it launches anything.
 */
int pdmk_eval_noalloc(pdmk_plan plan, double* pot, double* grad);

/*
 * pdmk_eval_adjoint -- vector-Jacobian product of pdmk_eval (the backward pass of a loss on
 * the potential at the sources).  The evaluation is linear in the charges, Phi = A q, and A is
 * symmetric: its entries are the periodic pair kernel G_p(y_i - y_j) (Eq. (1.1)-(1.2), zero
 * mean under the tin-foil convention, Sec. 1), the mean correction (a constant, Eq. (3.17))
 * and the diagonal self part, all even in the separation.  For the upstream gradient
 * g = dLoss/dPhi (g_pot, n values):
 *     g_q = dLoss/dq = A g                              (n values)
 *     g_y = dLoss/dy = g grad Phi[q] + q grad Phi[g]    (n x d, row-major, caller's frame)
 * computed with two evaluations on the device (charges q, then charges g; neutrality of g is
 * not required) and a combine kernel; the plan's charges are the caller's again on return.
 * With separate targets (pdmk_set_sources_targets) g_pot has one value per target and
 *     g_q = (B^T g)  the sources' potential of charges g at the targets   (n values)
 *     g_y = q grad Phi[g at x](y),   g_x = g grad Phi[q](x)                (n x d, m x d)
 * from the same two evaluations over the union of points.  g_q, g_y or g_x may be NULL (not
 * wanted).  g_grad (an upstream gradient on the returned field) must be NULL: it would need
 * second derivatives of the kernel.  Without separate targets g_x must be NULL: the targets
 * are the sources, so their derivative is part of g_y.  where = PDMK_HOST / PDMK_DEVICE for
 * all pointers.  The first call after pdmk_set_sources allocates n (4 + 2 d) doubles of
 * scratch (kept until the next pdmk_set_sources or pdmk_plan_destroy).  Ordered after the
 * plan's stream like pdmk_eval; a host call returns after the copies.
 * Errors: BAD_ARG, NOT_READY, OOM, CUDA, TIMEOUT.
 */
int pdmk_eval_adjoint(pdmk_plan plan, const double* g_pot, const double* g_grad, double* g_q, double* g_y,
                      double* g_x, int where);

/*
 * Batches of independent cells (many lattices of uneven N and different shapes evaluated
 * together).  Each cell is a full plan (Algorithm 1 per cell); one evaluation of every cell is
 * captured into a single CUDA graph on the batch's own stream, where the cells run as
 * independent branches.  There is no coupling between cells.
 *
 * pdmk_batch_create: ncells cells; d[c] in {2, 3}; L packs each cell's d[c] x d[c] lattice
 *   (column-major, as pdmk_plan_create) one after another; eps[c] per cell; opts (NULL:
 *   defaults) applies to every cell.  Errors: those of pdmk_plan_create, BAD_ARG, CUDA.
 * pdmk_batch_set_sources: offsets (ncells + 1 values, offsets[0] = 0, strictly increasing:
 *   every cell holds at least one source) place cell c's sources at [offsets[c],
 *   offsets[c+1]) of q, and its positions at rows offsets[c].. of y with d[c] values per row,
 *   rows packed cell after cell (row-major within a cell).  where as pdmk_set_sources.
 *   Allocates the per-cell buffers and, for host evaluations, one staging pair.
 * pdmk_batch_eval: potential (pot, offsets layout) and gradient (grad, the y layout, or
 *   NULL) at every source of every cell.  The first call runs eagerly, later calls replay the
 *   captured graph (re-captured when the output pointers change).  Ordered after the stream
 *   of opts; a host call returns after the copies.  Errors: NOT_READY, CUDA, TIMEOUT.
 * pdmk_batch_plan: cell c's plan (for pdmk_get_info; owned by the batch), or NULL.
 */
typedef struct pdmk_batch_s* pdmk_batch;
int pdmk_batch_create(int ncells, const int* d, const double* L, const double* eps, const pdmk_opts* opts,
                      pdmk_batch* out);
int pdmk_batch_set_sources(pdmk_batch batch, const int64_t* offsets, const double* y, const double* q, int where);
int pdmk_batch_eval(pdmk_batch batch, double* pot, double* grad, int where);
pdmk_plan pdmk_batch_plan(pdmk_batch batch, int cell);
void pdmk_batch_destroy(pdmk_batch batch);

/*
 * Multi-GPU runs over independent cells.  The cells of a batch share nothing, so ranks split
 * them and exchange nothing on the data path.  The paper has no counterpart (its runs use one
 * CPU thread); the estimate follows the cost of Algorithm 1's steps.  Host only; neither call
 * touches a GPU.
 * pdmk_cell_work: estimated flops of one evaluation of a cell of n sources with lattice L
 *   (d x d column-major), precision eps and options opts (NULL: defaults), from the plan's
 *   parameters alone (no tree): n (10 3^d n_s + 4 p^d + 6 w^d) + 10 prod(M) log2 prod(M).
 *   Errors: BAD_ARG, BAD_EPS, NONFINITE, SINGULAR_LATTICE.
 * pdmk_partition_cells: assigns each of ncells cells (work[c] >= 0) to one of nranks ranks,
 *   rank_of_cell[c] in [0, nranks): cells by decreasing work (ties by index) each go to the
 *   least-loaded rank (ties to the lowest).  Deterministic: every rank computes the same
 *   partition locally.  Errors: BAD_ARG.
 */
int pdmk_cell_work(int d, const double* L, double eps, const pdmk_opts* opts, int64_t n, double* work);
int pdmk_partition_cells(int ncells, const double* work, int nranks, int* rank_of_cell);

/* Per-stage device times (ms) of the last pdmk_eval when opts.profile = 1.  names/ms
 * receive up to cap entries; returns the number of stages (or a negative error).     */
int pdmk_stage_times(pdmk_plan plan, const char** names, double* ms, int cap);

/* Host wall-clock times (ms) of the phases of the last pdmk_set_sources (or
 * pdmk_set_sources_targets) of the plan: reading and checking the inputs, the tree build's
 * phases (images, root sort, refinement, level restriction, renumbering and colleagues,
 * sorted outputs), the direct lists, the per-point records, the near-field entries, the far
 * field's layout, the device uploads and the plane-wave layouts.  Recorded on every call,
 * whatever opts.profile.  names/ms (either may be NULL) receive up to cap entries; the names
 * are static strings.  Returns the number of phases (0 before the first set-up), or
 * PDMK_ERR_BAD_ARG for a NULL plan or cap < 0. */
int pdmk_setup_times(pdmk_plan plan, const char** names, double* ms, int cap);

/* Plan facts (sizes, counts) for reporting and roofline accounting. */
typedef struct {
    int d;
    double eps, c, rc, V, kappa;
    int n_s, window_w, n_proxy, n_pw, precision;
    int M[3];           /* Fourier grid                        */
    int nroot[3];       /* extended root grid (m_i + 2)         */
    int64_t n;          /* sources                              */
    int64_t n_images;   /* sources + images in the extended domain (N') */
    int nboxes, nleaves, depth, ntarget_leaves;
    int n_pw_boxes_out, n_pw_boxes_in;
    int64_t near_pairs; /* target-source pairs visited by the direct near field */
    int64_t near_pairs_in; /* of those, pairs inside the residual kernel's support (counted
                              on the first evaluation after pdmk_set_sources when profile = 1) */
    int64_t device_bytes;
    int launches;       /* kernels this library launched in the last pdmk_eval (cuFFT excluded) */
    /* work counts of the plane-wave passes (for roofline accounting) */
    int64_t pw_moment_sources; /* sources summed into leaf moments            */
    int pw_merge_parents;      /* boxes whose moments are merged from children */
    int pw_down_parents;       /* boxes whose local expansion is passed down   */
    int64_t pw_eval_targets;   /* targets evaluated from a leaf local expansion */
    int spread_subproblems;    /* spreading subproblems (tile, point range)     */
    int64_t n_targets;         /* points written by pdmk_eval: the separate targets
                                  of pdmk_set_sources_targets, else the sources  */
} pdmk_info;
int pdmk_get_info(pdmk_plan plan, pdmk_info* info);

/* Destroys the plan and frees its device memory (NULL is a no-op). */
void pdmk_plan_destroy(pdmk_plan plan);

/* Static message for an error code. */
const char* pdmk_strerror(int code);

/* Detail of the plan's last failure (the CUDA or cuFFT error text, or the violated condition),
 * "" if none; owned by the plan, valid until its next call. */
const char* pdmk_plan_message(pdmk_plan plan);

/*
 * Debug / verification access to the FP64 kernel tables (host only, no GPU needed).
 * kind: 0 = residual kernel R_1(t) (scale-free, t = r/h in (0, 1]), 1 = dR_1/dt,
 *       2 = hat-w(x) (transform of the smoothing density), 3 = bandwidth c (x ignored),
 *       4 = self value W_1(0) (3D: psi(0)/(4 pi c0); 2D: W_1(0)),
 *       5 = integral of the residual kernel (hat-R_h(0) = value * h^2; x ignored),
 *       6 = the default spreading window's F(s) at s = x in [0, 1] (window w = ceil(2c/pi) + 2),
 *       7 = that window's Fourier transform at grid frequency x (cycles per grid point).
 * Returns 0 and writes *value, or a negative error.
 */
int pdmk_kernel_table_eval(int d, double eps, int kind, double x, double* value);

#ifdef __cplusplus
}
#endif
#endif /* PDMK_H */
