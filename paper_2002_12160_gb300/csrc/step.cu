// step.cu -- the cold-started step kernels (every substep's solve starts from
// zero impulses) and the host entry points over all compiled shapes; the
// kernel itself is in step_kernel.cuh, its warm-started instances in
// step_warm.cu.
#include "step_kernel.cuh"

namespace ih {
// every shape holds any c_max <= IH_MAX_CONTACTS (contacts beyond its registers
// live in shared memory, and beyond the shape's staging capacity in the spill area)
int step_variant_max_contacts(const StepVariant &v) { return v.group > 0 ? IH_MAX_CONTACTS : 0; }

bool step_variant_supported(const StepVariant &v) {
    if (v.block != kBlock) return false;
#define IH_SUP(T, C) if (v.group == T && v.cpl == C) return true;
    IH_STEP_VARIANTS(IH_SUP)
#undef IH_SUP
    return false;
}

int step_variant_list(StepVariant *out, int cap) {
    int n = 0;
#define IH_LIST(T, C) if (n < cap) out[n] = StepVariant{T, C, kBlock}; ++n;
    IH_STEP_VARIANTS(IH_LIST)
#undef IH_LIST
    return n;
}

size_t step_smem_bytes(const StepVariant &v, int s_max, int c_max, bool warm, int clp_cap) {
    return warm ? step_smem_bytes_warm(v, s_max, c_max, clp_cap) : smem_bytes_w<false>(v, s_max, c_max, clp_cap);
}

cudaError_t step_prepare(const StepVariant &v, int s_max, int c_max, bool warm, int clp_cap, int *blocks_per_sm) {
    return warm ? step_prepare_warm(v, s_max, c_max, clp_cap, blocks_per_sm)
                : prepare_w<false>(v, s_max, c_max, clp_cap, blocks_per_sm);
}

int step_stage_capacity(const StepVariant &v, int c_max) {
    return stage_capacity(v.group * v.cpl, c_max, v.block / v.group);
}

cudaError_t launch_step(const StepArgs &a, const StepVariant &v, int grid, int s_max, cudaStream_t s) {
    return a.cfg.warm ? launch_step_warm(a, v, grid, s_max, s) : launch_w<false>(a, v, grid, s_max, s);
}

}  // namespace ih
