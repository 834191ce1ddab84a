// host_plan.h -- host-side (FP64) planning for the periodic DMK evaluation:
// prolate spheroidal wave functions and the kernel tables derived from them, cell
// geometry, the Fourier grid, image enumeration and the adaptive tree with its lists.
// Nothing here runs per evaluation; eval() only launches device kernels.
#pragma once
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

namespace pdmk {

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------------
// Prolate spheroidal wave function psi_0^c (Sec. 2.2, Eq. (2.3)) on [-1, 1], expanded in
// normalised Legendre polynomials of even degree; zero outside [-1, 1].
struct Pswf {
    double c = 0;
    std::vector<double> beta;  // coefficient of sqrt(n + 1/2) P_n, n = 2k
    double psi0 = 0, psi1 = 0, c0 = 0;  // psi(0), psi(1), int_0^1 psi (Eq. (2.9))
    double eval(double x) const;         // psi(x) for |x| <= 1
};
Pswf pswf_make(double c);
// bandwidth c such that psi(1)/psi(0) = eps (the calibration of Sec. 2.2, normalised)
double pswf_calibrate(double eps);

// Chebyshev series on [a, b]: f(x) ~ sum_k coef[k] T_k((2x - a - b)/(b - a))
struct Cheb {
    double a = 0, b = 1;
    std::vector<double> coef;
    double eval(double x) const;
};
// interpolate f at n Chebyshev points and keep the terms needed for absolute accuracy tol
template <class F>
Cheb cheb_fit(F f, double a, double b, int n, double tol);

// ---------------------------------------------------------------------------------
// Scale-free kernel data, all FP64.  t = r/h in [0, 1], s = t^2.
struct KernelTables {
    int d = 3;
    double eps = 1e-6;
    Pswf psi;            // the splitting prolate (bandwidth c)
    double mu2 = 0;      // (1/c0) int_0^1 psi t^2 dt : hat-w(x) = 1 - mu2 x^2/2 + ...
    // residual kernel R_h(r) = R_1(r/h) (Eq. (2.7)-(2.8); 2D by radial transform):
    //  3D: R = (1 - t A(s)) / (4 pi r),  grad R = -(1 - t A + t B) dr/(4 pi r^3)
    //      A(s) = phi(t)/t, B(s) = phi'(t) = psi(t)/c0
    //  2D: R = -log(s)/(4 pi) - A(s),    grad R = -sqrt(1-s) B(s) dr/(2 pi r^2)
    //      A(s) = W_1(t) = (1/2pi) int_t^1 Q(u)/u du,  sqrt(1-s) B(s) = 1 - Q(t),
    //      Q(t) = charge of the radial smoothing density inside radius t
    Cheb A, B;
    double self_coef = 0;  // 3D: W_h(0) = self_coef / h;  2D: W_h(0) = self_coef - log(h)/(2 pi)
    double rhat0 = 0;      // hat-R_h(0) = rhat0 * h^2 (integral of the residual kernel)
    // Fourier transform of the radial smoothing density, hat-w(x) = (1/c0) int_0^1 psi cos(x t)
    double what(double x) const;
    std::vector<double> gl_x, gl_w, gl_psi;  // Gauss-Legendre nodes on [0,1], psi at nodes
};
KernelTables make_kernel_tables(int d, double eps, double fit_tol);

// spreading window phi(z) = F((2z/w)^2) for |z| < w/2 grid units, F = psi_{cw}/psi_{cw}(0)
struct WindowTables {
    int w = 0;
    double cw = 0;
    Cheb F, dF;  // F(s) and dF/ds, s in [0, 1]
    // continuous Fourier transform of the window at grid frequency nu (cycles/grid point)
    double ft(double nu) const;
    std::vector<double> gl_x, gl_w;
};
WindowTables make_window(int w, double cw, double fit_tol);

// Gauss-Legendre nodes and weights on [a, b]
void gl_interval(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
// continuous Fourier transform at grid frequency nu of the exponential-of-semicircle
// window phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)), |z| < w/2 (computed with t = sin theta)
double es_window_ft(int w, double beta, double nu, const std::vector<double>& gx,
                    const std::vector<double>& gw);

// ---------------------------------------------------------------------------------
// Cell geometry (Sec. 3.2, Eq. (3.4)-(3.9)) and Fourier grid (Sec. 3.7, Eq. (3.15)).
struct Geometry {
    int d = 3;
    int perm[3] = {0, 1, 2};  // oriented column i = user column perm[i]
    double Q[9] = {0};        // x_oriented = Q x_user (row-major, d x d)
    double R[9] = {0};        // oriented upper-triangular lattice matrix (row-major)
    double Rinv[9] = {0};
    double V = 0;
    double anorm[3] = {0, 0, 0};
    double Lmin = 0, rc = 0;
    int m[3] = {1, 1, 1};        // inner block
    int nroot[3] = {1, 1, 1};    // extended domain m + 2
    double lo[3] = {0, 0, 0};    // lower corner of the extended domain
    int M[3] = {1, 1, 1};        // Fourier grid
    // cubic cell (Remark 3.3): the root grid is the cell itself, tiled by m cubes per axis,
    // with no halo and no image sources; neighbours across the cell's faces are the boxes on
    // the opposite side, shifted by a lattice vector (periodic box coordinates)
    bool periodic_root = false;
};
// switches a cubic (square) cell with an integer kappa >= 3 to the periodic root; returns
// whether it did (the cell's oriented matrix must be a multiple of the identity to 1e-13)
bool make_periodic_root(Geometry* g, double kappa);
// returns 0 or a negative PDMK error code
int make_geometry(int d, const double* Lcolmajor, double kappa, double c, Geometry* g);

// ---------------------------------------------------------------------------------
// Adaptive tree on the extended domain (Sec. 3.3, Algorithm 1 steps 1-2).
struct Tree {
    int d = 3;
    int nlevels = 1;
    std::vector<int> level_start;     // boxes of level l: [level_start[l], level_start[l+1])
    std::vector<int> level;           // per box
    std::vector<int64_t> coord;       // d per box, integer coords at the box's level
    std::vector<int> parent, child0;  // child0: first of 2^d contiguous children, or -1
    std::vector<int64_t> src_begin, src_end;  // sorted-source range of each box
    std::vector<int64_t> tgt_begin, tgt_end;  // sorted-target range of each box
    std::vector<int> colleague;       // 3^d per box (same-level neighbour or -1)
    std::vector<double> center;       // d per box
    double h(int l, double rc) const { return rc / double(1LL << l); }
    bool is_leaf(int b) const { return child0[b] < 0; }
    int64_t nroot[3] = {1, 1, 1};
    bool periodic = false;  // box coordinates wrap (cubic cell, Remark 3.3)
    // deepest existing box of level <= L containing the level-L cell c, or -1 outside (with
    // periodic coordinates, c is wrapped first)
    int locate(int L, const int64_t* c) const;
    // the shift code (n_0 + 1) + 3 (n_1 + 1) + 9 (n_2 + 1) of the lattice vector that brings the
    // level-L cell c into the root grid (periodic coordinates), with c replaced by the wrapped
    // cell; 13 (no shift) otherwise
    int wrap(int L, int64_t* c) const;
};

// A source record after image enumeration and sorting.
struct SortedSources {
    std::vector<int64_t> orig;    // original source index of each sorted source
    std::vector<double> pos;      // d per sorted source (oriented frame, absolute)
    std::vector<int64_t> tgt_of;  // sorted target t -> sorted source index of the original
    std::vector<int64_t> tgt_orig;  // sorted target t -> original index
};

struct BuildStats {
    int64_t n = 0, n_images = 0;
    int nboxes = 0, nleaves = 0, depth = 0;
    int64_t near_pairs = 0;
    // host milliseconds of the phases of build_tree, in the order of kBuildPhases
    double phase_ms[6] = {0, 0, 0, 0, 0, 0};
};
constexpr const char* kBuildPhases[6] = {"tree_images", "tree_root_sort", "tree_refine",
                                         "tree_level_restriction", "tree_renumber_colleagues",
                                         "tree_sorted_outputs"};

// The lattice shifts n of the images (Sec. 3.4, bounds of Eq. (3.13)): index 0 is no shift,
// then the nested loops with n_d outermost; none for a periodic root.  sidx maps the flat
// index of n + Bx (axis 0 fastest, extents dimx) to the shift's index or -1; trs holds R n
// (3 per shift).
struct ImageShifts {
    int ns = 1;
    int Bx[3] = {0, 0, 0};
    int64_t dimx[3] = {1, 1, 1};
    std::vector<int> sidx;
    std::vector<double> trs;
};
void image_shifts(const Geometry& g, ImageShifts* out);

// Images + tree + sort.  u: n*d fractional coordinates of the originals in [0,1).
int build_tree(const Geometry& g, int64_t n, const double* u, int n_s, int max_depth, Tree* t,
               SortedSources* s, BuildStats* st);

// near-field direct lists: for each target leaf, the source leaves it must visit
struct DirectLists {
    std::vector<int> tleaf;           // target leaves (boxes with targets that are leaves)
    std::vector<int64_t> list_begin;  // CSR over tleaf
    std::vector<int> list;            // source leaf box ids
    std::vector<int> shift;           // per entry: shift code of the lattice vector added to the
                                      // source leaf (13 = none; periodic roots only)
};
void build_direct_lists(const Tree& t, DirectLists* dl, int64_t* pairs);
// the source leaves meeting the 3^d neighbourhood of box b (any box, leaf or not), sorted,
// with the shift code of each (a leaf may appear once per distinct shift)
void box_direct_list(const Tree& t, int b, std::vector<int>* out, std::vector<int>* shift);
// lattice shift n (integer per axis) of a shift code
inline void shift_of(int code, int* n) {
    n[0] = code % 3 - 1;
    n[1] = (code / 3) % 3 - 1;
    n[2] = code / 9 - 1;
}

// sort (ascending, lexicographic) on the host's threads: the same order as std::sort
void sort_pairs_parallel(std::vector<std::pair<int64_t, int64_t>>* v);

// default (kappa, n_s) from the paper's Table 1
void table1_defaults(int d, double eps, const Geometry* g_or_null, const double* Lcol,
                     double* kappa, int* n_s);

}  // namespace pdmk
