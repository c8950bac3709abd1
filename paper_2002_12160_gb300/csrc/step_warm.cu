// step_warm.cu -- the step kernels with the warm-started solver: each contact
// starts from the final impulse of the same (link, sphere) pair in the
// environment's previous substep, carried across launches in a per-environment
// cache (Sec. III-A's solver with the warm start of iterative contact solvers).
#include "step_kernel.cuh"

namespace ih {

size_t step_smem_bytes_warm(const StepVariant &v, int s_max, int c_max, int clp_cap) {
    return smem_bytes_w<true>(v, s_max, c_max, clp_cap);
}

cudaError_t step_prepare_warm(const StepVariant &v, int s_max, int c_max, int clp_cap, int *blocks_per_sm) {
    return prepare_w<true>(v, s_max, c_max, clp_cap, blocks_per_sm);
}

cudaError_t launch_step_warm(const StepArgs &a, const StepVariant &v, int grid, int s_max, cudaStream_t s) {
    return launch_w<true>(a, v, grid, s_max, s);
}

}  // namespace ih
