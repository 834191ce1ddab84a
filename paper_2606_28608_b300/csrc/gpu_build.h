// gpu_build.h -- the source set-up on the device (Algorithm 1, steps 1-2, and Sec. 3.4):
// orientation and wrapping, image enumeration, the adaptive tree with its level restriction,
// the sorted order of sources and targets, and the per-point records of the near field, the
// plane-wave passes and the far field.  It produces exactly the tree, order and records of
// the host build (host_plan.cpp): the same arithmetic in the same order (FP64, no
// contraction), images in shift order, boxes in level order with children in order, and
// sources sorted by leaf and then by image index.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "dev_pool.h"
#include "host_plan.h"

namespace pdmk {

// device arrays of one build, freed by gpu_build_free
struct GpuBuild {
    int64_t n = 0, nimg = 0, ntgt = 0;
    int key_levels = 0;         // depth of the point keys (levels a tree may reach)
    double* d_u = nullptr;      // n x d fractional coordinates of the points in [0, 1)
    int* d_orig = nullptr;      // per sorted source: point index
    double* d_pos = nullptr;    // per sorted source: oriented position (d)
    int* d_leaf = nullptr;      // per sorted source: leaf box
    int* d_tgt_of = nullptr;    // per sorted target: sorted source index of the point
    int* d_tgt_orig = nullptr;  // per sorted target: point index
    std::vector<std::pair<void*, size_t>> allocs;  // the arrays below that b owns (buffer, bytes)
    // with a pool: b's arrays come from it and go back to it (gpu_build_free), and the
    // build's temporary buffers come from it and are appended to *scratch, for the caller
    // to return once the stream has drained; without one, cudaMalloc and cudaFree
    DevicePool* pool = nullptr;
    std::vector<std::pair<void*, size_t>>* scratch = nullptr;
    unsigned char* h_stage = nullptr;  // optional page-locked staging buffer of the caller
    size_t stage_cap = 0;              // its bytes (used when at least 1 MiB)
    // the tree's box arrays on the device, in the host tree's box order (nb boxes)
    int nb = 0;
    int* d_level = nullptr;
    long long* d_coord = nullptr;   // d per box
    int* d_parent = nullptr;
    int* d_child0 = nullptr;
    long long* d_src_b = nullptr;
    long long* d_src_e = nullptr;
    long long* d_tgt_b = nullptr;
    long long* d_tgt_e = nullptr;
    int* d_colleague = nullptr;     // 3^d per box
    double* d_center = nullptr;     // d per box (tree frame)
    bool download_tree = true;      // gpu_build_tree fills the host tree's per-box arrays
};
void gpu_build_free(GpuBuild* b);

// Returned when the tree would need more levels than the 64-bit point keys hold (or more
// images than 32-bit indices): the host build serves these inputs.
constexpr int kGpuBuildUnsupported = 1;

// u (device, n x d) must already hold the wrapped fractional coordinates.  Fills the host
// tree t (every per-box array, as build_tree does), the device arrays of b and st (whose
// phase_ms take the phases below, host wall clock with the stream drained at each boundary).
constexpr const char* kDeviceBuildPhases[6] = {"tree_device_images",      "tree_device_keys_sort",
                                               "tree_device_refinement",  "tree_device_level_restriction",
                                               "tree_device_boxes_order", "tree_device_download"};
int gpu_build_tree(const Geometry& g, int64_t n, int n_s, int max_depth, cudaStream_t s, GpuBuild* b, Tree* t,
                   BuildStats* st, std::string* msg);

// the per-box arrays of b's device tree into the host tree t (whose scalars gpu_build_tree set)
int gpu_tree_download(const GpuBuild& b, Tree* t, cudaStream_t s, std::string* msg);

// ---- per-point passes (launchers; all arrays on the device) ----
// the caller's positions (n x d) to wrapped fractional coordinates u (the orientation Q, then
// R^{-1}, minus the floor)
void gpu_orient(const Geometry& g, int64_t n, const double* y, double* u, cudaStream_t s);
// nonfinite inputs (flag), and per-block partial sums of q and |q| (nblk x 2, summed by the
// caller in block order)
void gpu_check_inputs(int64_t n, int d, const double* y, const double* q, int* d_nonfinite, double* d_part,
                      int nblk, cudaStream_t s);

// leaf-relative records of the sorted sources and of the targets (the host build's
// "leaf-relative coordinates": caller-frame leaf centres Cu, lattice-shift displacement of
// every copy, hi/lo split in mixed precision)
struct RecordArgs {
    int d;
    int mixed;
    int64_t nimg, ntgt;
    double Q[9], R[9], Rinv[9];
    const double* y;        // caller positions (n x d)
    const int* orig;        // per sorted source
    const double* pos;      // per sorted source (oriented, d)
    const int* leaf;        // per sorted source
    const double* center;   // per box (tree frame, d)
    const double* Cu;       // per box (caller frame, d)
    const int* tgt_of;      // per sorted target
    const int* tgt_orig;    // per sorted target
    const int* box_level;   // per box
    const double* self_w_level;  // W_{h_L}(0) per level
    void* src4;             // out: 4 T per sorted source
    float* src_lo;          // out (mixed): 4 per sorted source
    int* src_orig;          // out
    double* src_disp;       // out: caller-frame lattice vector per sorted source (d)
    void* tgt4;             // out
    float* tgt_lo;          // out (mixed)
    int* tgt_orig_out;      // out
    double* self_w;         // out: per sorted target
    int* tgt_leaf;          // out: per sorted target
};
void gpu_records(const RecordArgs& a, cudaStream_t s);
// caller-frame box centres Cu = Q^T c_b
void gpu_box_cu(int nb, int d, const double* Q, const double* center, double* Cu, cudaStream_t s);

// far-field layout: window starts, offsets and bins of every point, the points in bin order
// (stable), and the interpolation records of the targets
struct FarLayoutArgs {
    int d;
    int mixed;
    int64_t n, ntgt;
    int M[3], B[3], nbin[3];
    int w;
    int nbins_tot;
    const double* u;       // n x d
    const int* tgt_orig;   // per sorted target
    int4* pt_g0;           // out: per point in bin order
    void* pt_dq;           // out: 4 T per point in bin order
    int* sp_orig;          // out: point index per position in bin order
    int* bin_count;        // out: points per bin (nbins_tot)
    int4* t_g0;            // out: per sorted target
    DevicePool* pool;      // optional: temporary buffers from it, appended to *scratch (as GpuBuild)
    std::vector<std::pair<void*, size_t>>* scratch;
    void* t_dq;            // out
};
int gpu_far_layout(const FarLayoutArgs& a, cudaStream_t s, std::string* msg);

// near-field entries: per direct-list entry e of target leaf k (list_begin[k] <= e <
// list_begin[k + 1]), the source leaf's range and the shift Q (Cu_s + L n - Cu_t) of its
// centre into the target leaf's frame (hi / lo split in mixed precision), as the host build
struct EntryArgs {
    int d;
    int mixed;
    int64_t nlist;
    int ntleaf;
    double Q[9];
    double Ln[27 * 3];          // caller-frame lattice vector of every shift code
    const int* tleaf;           // target leaf boxes
    const long long* list_begin;  // ntleaf + 1
    const int* list;            // source leaf per entry
    const int* shift;           // shift code per entry
    const int* bsb;             // per box: first sorted source
    const int* bsc;             // per box: source count
    const double* Cu;           // per box: caller-frame centre (d)
    int2* ent;                  // out
    void* ent_sh;               // out: 4 T per entry (zeroed by the caller)
    float* ent_shlo;            // out (mixed; zeroed by the caller)
};
void gpu_near_entries(const EntryArgs& a, cudaStream_t s);

// ---- near-field lists on the device (after gpu_build_tree, from its box arrays) ----
// The direct lists and descriptors of the host build (build_direct_lists, the descriptor
// order of the near-field layout), identically: per target leaf (a leaf with targets, in box
// order) the sorted, unique (source leaf, shift code) pairs of its 3^d neighbourhood, where a
// missing same-level neighbour is covered by the colleague of the leaf's parent (one level
// up, a leaf, by the level restriction); descriptors of at most 32 targets when split32,
// ordered by decreasing pair count, ties in leaf order.
struct NearLists {
    int ntleaf = 0;                       // target leaves
    int64_t nlist = 0;                    // direct-list entries
    int64_t ndesc = 0;                    // descriptors
    int64_t pairs = 0;                    // source-target pairs of the lists
    int* d_tleaf = nullptr;               // target leaf boxes
    long long* d_list_begin = nullptr;    // ntleaf + 1
    int* d_shift = nullptr;               // per entry: shift code
    long long* d_nsrc = nullptr;          // per target leaf: sources of its list
    long long* d_desc_begin = nullptr;    // per target leaf: first descriptor (ntleaf + 1)
};
// counts (downloaded) and the lists' offsets; 0, or PDMK_ERR_CUDA, or PDMK_ERR_INTERNAL when a
// list outgrows its bound (the host build serves the inputs then)
int gpu_near_count(GpuBuild* b, const Geometry& g, bool split32, NearLists* nl, cudaStream_t s, std::string* msg);
// the entries' source leaves (d_list, nlist), the descriptors (d_desc, ndesc TLeaf records),
// the per-box source ranges (d_bsb, d_bsc: int, nb)
struct TLeaf;
int gpu_near_fill(GpuBuild* b, const Geometry& g, bool split32, NearLists* nl, int* d_list, TLeaf* d_desc,
                  int* d_bsb, int* d_bsc, cudaStream_t s, std::string* msg);

}  // namespace pdmk
