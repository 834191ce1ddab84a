// pw.cu -- plane-wave passes (placeholder: depth-0 trees need none).
#include "k_pw.cuh"
#include "pdmk.h"

namespace pdmk {

void pw_plan_create(PwPlan* pw, int d, double, double, const KernelTables&, int, int, bool mixed) {
    pw->d = d;
    pw->mixed = mixed;
}
bool pw_supported(const PwPlan*) { return false; }
int pw_set_sources(PwPlan* pw, const Tree& t, const SortedSources&, const std::vector<int>&,
                   const std::vector<int>&, const Geometry&, cudaStream_t) {
    pw->active = t.nlevels > 1;
    return pw->active ? PDMK_ERR_INTERNAL : PDMK_OK;
}
int pw_set_charges(PwPlan*, cudaStream_t) { return PDMK_OK; }
int pw_eval(PwPlan*, cudaStream_t) { return PDMK_OK; }
void pw_free_sources(PwPlan* pw) {
    for (void* p : pw->allocs) cudaFree(p);
    pw->allocs.clear();
    pw->active = false;
}
void pw_free(PwPlan* pw) { pw_free_sources(pw); }

}  // namespace pdmk
