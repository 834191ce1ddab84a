// k_pw.cuh -- plane-wave passes of the difference kernels D_l (Sec. 2.3, Eq. (2.5)-(2.6);
// Sec. 3.5: the free-space DMK on the extended domain with the root W_0 step omitted):
// upward proxy charges, outgoing plane waves, colleague translation, incoming plane waves
// to local values, downward interpolation, and evaluation at leaf targets.
#pragma once
#include <cuda_runtime.h>

#include "dev_pool.h"

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "host_plan.h"

namespace pdmk {

struct PwPlan {
    int d = 3;
    int p = 0;   // Chebyshev proxy points per dimension
    int K = 0;   // plane-wave nodes -K..K per dimension
    bool mixed = false;
    bool active = false;  // the tree has levels below the root grid
    int nout = 0, nin = 0;
    int launches = 0;  // kernels launched by the last pw_eval
    int64_t moment_sources = 0, eval_targets = 0;
    int merge_parents = 0, down_parents = 0;
    int64_t device_bytes = 0;
    double* d_pot = nullptr;   // per sorted target
    double* d_grad = nullptr;  // d per sorted target
    const void* d_src4 = nullptr;  // borrowed from the plan (sorted sources, leaf-relative)
    const void* d_tgt4 = nullptr;  // borrowed (sorted targets, leaf-relative)
    int* h_err = nullptr;   // host-mapped flag: a bounded device wait expired (sticky)
    int* d_err = nullptr;   // its device address
    int wait_test = 0;      // test hook: make the first dependent downward item wait forever
    int nsm = 1;            // SMs of the plan's device (grid sizing)
    bool tensor_cores = true;  // 3D leaf evaluation of FP32 plans on tcgen05 (3xTF32)
    std::vector<int> lslot;  // per box: slot of its local expansion in the local array, or -1
    std::vector<unsigned char> local_full;  // per box: the slot holds its complete local expansion
                                            // after the downward pass (every receiving non-leaf box,
                                            // and the target leaves unless the 2D single-launch pass
                                            // keeps theirs in shared memory)
    std::vector<std::pair<void*, size_t>> allocs;  // (buffer, bytes)
    DevicePool* pool = nullptr;  // the plan's: buffers released by pw_free_sources go there
    void* impl = nullptr;
};

void pw_plan_create(PwPlan* pw, int d, double eps, double c, const KernelTables& kt, int n_proxy, int n_pw,
                    bool mixed);
bool pw_supported(const PwPlan* pw);
// leaf_of: the leaf of every sorted source on the host, or empty with d_leaf_of (nimg entries)
// on the device
int pw_set_sources(PwPlan* pw, const Tree& t, const SortedSources& s, const std::vector<int>& leaf_of,
                   const std::vector<int>& tgt_leaf, const Geometry& g, cudaStream_t stream,
                   const int* d_leaf_of, int64_t nimg);
// The same layout built on the device from the device tree's box arrays (3D plans; the
// lists equal pw_set_sources', box for box).  The host per-box slot tables (lslot,
// local_full) are then filled on demand by pw_host_slots.
struct PwTreeDev {
    int nb = 0;
    const int* level = nullptr;
    const int* child0 = nullptr;
    const long long* src_b = nullptr;
    const long long* src_e = nullptr;
    const long long* tgt_b = nullptr;
    const long long* tgt_e = nullptr;
    const int* colleague = nullptr;  // 27 per box
};
int pw_set_sources_device(PwPlan* pw, const PwTreeDev& dt, const std::vector<int>& level_start, int nlevels,
                          const Geometry& g, cudaStream_t stream);
// the host per-box slot tables of the layout (lslot, local_full), if not filled yet
void pw_host_slots(PwPlan* pw, const Tree& t);
// the layout's device lists and counts, as named byte arrays (the set-up comparison)
void pw_layout_snapshot(PwPlan* pw, std::vector<std::pair<std::string, std::vector<unsigned char>>>* out);
int pw_set_charges(PwPlan* pw, cudaStream_t stream);
// phase 0: leaf moments (in 2D compile-time orders: moments and outgoing waves straight
// from the sources); 1: upward merges; 2: outgoing plane waves; 3: translation + incoming;
// 4: downward pass; 5: evaluation at leaf targets
constexpr int kPwPhases = 6;
int pw_eval(PwPlan* pw, cudaStream_t stream, int phase);
// Evaluation of stored local expansions at arbitrary points (after phases 0-4 of pw_eval):
// list entries (local slot, first point, count, level of the box) over points given relative
// to their box's centre (d_pts4: 4 values of the plan's precision per point); writes pot (one
// per point) and grad (d per point).
int pw_eval_points(PwPlan* pw, cudaStream_t stream, const int4* d_list, int nlist, const void* d_pts4, double* pot,
                   double* grad);
void pw_free_sources(PwPlan* pw);
void pw_free(PwPlan* pw);

}  // namespace pdmk
