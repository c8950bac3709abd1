// noalloc.cu -- cost_eval_static: the cost-and-argmin step for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// allocator's callbacks, a real-time loop whose device memory was reserved
// up front, or a process that shares a GPU under a fixed memory budget. They
// can still hand us their own input and output buffers; what they cannot do
// is create a simulator handle (which allocates its state) or give us scratch.
// This entry point therefore keeps its scratch -- one partial (cost, index)
// per block and the last-block ticket -- in a file-scope __device__ array of
// fixed size that every GPU loading the library holds until the process exits.
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kNaBlock = 32;                        // environments per block
constexpr int kNaMaxBlocks = 4096;                  // => at most 131072 environments
constexpr int kNaMaxEnvs = kNaBlock * kNaMaxBlocks;

// Scratch: [0, kNaMaxBlocks) doubles of partial costs, then kNaMaxBlocks ints
// of partial indices, then the ticket. 48 KiB + 256 B per device.
struct NaScratch {
    double part_c[kNaMaxBlocks];
    int part_i[kNaMaxBlocks];
    unsigned int ticket;
};
static __device__ __align__(256) NaScratch g_na_scratch;

// Host code must not pass the symbol g_na_scratch itself to a kernel: on the
// host it only stands in for the array. Its device address is looked up on
// every call, in the current device's context (the lookup allocates nothing),
// so a device reset or a new primary context cannot leave a stale address.

__device__ __forceinline__ bool na_better(double ca, int ia, double cb, int ib) {
    return ca < cb || (ca == cb && ia < ib);
}

__device__ __forceinline__ void na_warp_min(double &c, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xffffffffu, c, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (na_better(oc, oi, c, i)) { c = oc; i = oi; }
    }
}

// Same arithmetic and order as cost_eval: FP64, no fused multiply-adds.
__global__ void __launch_bounds__(kNaBlock)
cost_static_kernel(const float *forces, const float *obs, const int *status, int N, int P, double tau,
                   double w_force, double w_contact, double *c_sum, int n_window, double *cost_mean,
                   int *argmin, NaScratch *scr) {
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double cm = INFINITY;
    int ci = 0x7fffffff;
    if (i < N) {
        double c = 0.0;
        if (status && (status[i] & kDiverged)) {
            c = INFINITY;
        } else {
            const float *f = forces + (size_t)i * P * 3;
            const double tau2 = __dmul_rn(tau, tau);
            for (int l = 0; l < P; ++l) {
                const double fx = f[3 * l], fy = f[3 * l + 1], fz = f[3 * l + 2];
                const double ox = obs[3 * l], oy = obs[3 * l + 1], oz = obs[3 * l + 2];
                const double dx = __dsub_rn(fx, ox), dy = __dsub_rn(fy, oy), dz = __dsub_rn(fz, oz);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                c = __dadd_rn(c, __dmul_rn(w_force, d2));
                const double ns = __dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz));
                const double no = __dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz));
                if ((ns > tau2) != (no > tau2)) c = __dadd_rn(c, w_contact);
            }
        }
        const double s = __dadd_rn(c_sum[i], c);
        c_sum[i] = s;
        cm = __ddiv_rn(s, (double)n_window);
        if (cost_mean) cost_mean[i] = cm;
        if (isnan(cm)) cm = INFINITY;
        ci = i;
    }
    na_warp_min(cm, ci);
    if (threadIdx.x == 0) {
        scr->part_c[blockIdx.x] = cm;
        scr->part_i[blockIdx.x] = ci;
        __threadfence();
        last = atomicAdd(&scr->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double bc = INFINITY;
    int bi = 0x7fffffff;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const double c = __ldcg(scr->part_c + b);
        const int ii = __ldcg(scr->part_i + b);
        if (na_better(c, ii, bc, bi)) { bc = c; bi = ii; }
    }
    na_warp_min(bc, bi);
    if (threadIdx.x == 0) {
        *argmin = (bi == 0x7fffffff) ? 0 : bi;
        scr->ticket = 0u;
    }
}

// The scratch's device address in the current device's context.
ih_status na_scratch(NaScratch **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) return IH_ERR_CUDA;
    *out = static_cast<NaScratch *>(p);
    return IH_OK;
}

}  // namespace
}  // namespace ih

using namespace ih;

extern "C" {

ih_status cost_eval_static(const float *forces, const float *obs, const int32_t *env_status, int32_t n_envs,
                           int32_t n_pads, float tau, float w_force, float w_contact, double *c_sum,
                           int32_t n_window, double *cost_mean, int32_t *argmin, void *stream) {
    if (!forces || !obs || !c_sum || !argmin) return IH_ERR_ARG;
    if (n_envs < 1 || n_pads < 1 || n_pads > IH_MAX_PADS || n_window < 1 || !(tau >= 0.0f)) return IH_ERR_ARG;
    if (n_envs > kNaMaxEnvs) return IH_ERR_OVERFLOW;   // beyond the fixed scratch
    NaScratch *scr = nullptr;
    ih_status r = na_scratch(&scr);
    if (r != IH_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero; the partials are written before they are read
    cudaError_t e = cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return IH_ERR_CUDA;
    const int blocks = (n_envs + kNaBlock - 1) / kNaBlock;
    cost_static_kernel<<<blocks, kNaBlock, 0, st>>>(forces, obs, env_status, n_envs, n_pads, (double)tau,
                                                    (double)w_force, (double)w_contact, c_sum, n_window,
                                                    cost_mean, argmin, scr);
    return cudaGetLastError() == cudaSuccess ? IH_OK : IH_ERR_CUDA;
}

}  // extern "C"
