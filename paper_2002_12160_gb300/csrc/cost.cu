// cost.cu -- per-environment cost against the observed sensor forces and the
// argmin estimate (Sec. III-C; Eqs. 1-2 with the running mean of Algorithm 1).
//
// One thread per environment accumulates, in FP64,
//   cost_i = sum_l [ w_force |c_il - o_l|^2 + w_contact ((|c_il| > tau) != (|o_l| > tau)) ]
// into the window sum, forms C_i = sum / n (n = frames in the window) and
// joins a block min-reduction on (C_i, i). Each block leaves its partial in
// scratch; the last block to finish (atomic ticket) reduces the partials,
// publishes i*, copies the pose of i*, advances the window count and resets
// the ticket for the next launch.
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kCostBlock = 256;

__device__ __forceinline__ bool better(double ca, int ia, double cb, int ib) {
    return ca < cb || (ca == cb && ia < ib);
}

__global__ void __launch_bounds__(kCostBlock) cost_kernel(const CostArgs a) {
    __shared__ double sc[kCostBlock];
    __shared__ int si[kCostBlock];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = *a.n_window + 1;
    double cm = INFINITY;
    int ci = 0x7fffffff;
    if (i < a.N) {
        double c = 0.0;
        if (a.status[i] & kDiverged) {
            c = INFINITY;
        } else {
            // evaluated in the order written, without fused multiply-adds
            const float *f = a.forces + (size_t)i * a.P * 3;
            const double tau = (double)a.cfg.tau, wf = (double)a.cfg.w_force;
            for (int l = 0; l < a.P; ++l) {
                const double fx = f[3 * l], fy = f[3 * l + 1], fz = f[3 * l + 2];
                const double ox = a.obs[3 * l], oy = a.obs[3 * l + 1], oz = a.obs[3 * l + 2];
                const double dx = __dsub_rn(fx, ox), dy = __dsub_rn(fy, oy), dz = __dsub_rn(fz, oz);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                c = __dadd_rn(c, __dmul_rn(wf, d2));
                const double ns = __dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz));
                const double no = __dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz));
                const bool on_sim = sqrt(ns) > tau;
                const bool on_obs = sqrt(no) > tau;
                if (on_sim != on_obs) c = __dadd_rn(c, (double)a.cfg.w_contact);
            }
        }
        const double s = __dadd_rn(a.c_sum[i], c);
        a.c_sum[i] = s;
        cm = __ddiv_rn(s, (double)n);
        if (a.cost_mean) a.cost_mean[i] = cm;
        if (isnan(cm)) cm = INFINITY;
        ci = i;
    }
    sc[threadIdx.x] = cm;
    si[threadIdx.x] = ci;
    __syncthreads();
    for (int o = kCostBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o && better(sc[threadIdx.x + o], si[threadIdx.x + o], sc[threadIdx.x], si[threadIdx.x])) {
            sc[threadIdx.x] = sc[threadIdx.x + o];
            si[threadIdx.x] = si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.part_c[blockIdx.x] = sc[0];
        a.part_i[blockIdx.x] = si[0];
        __threadfence();
        last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double bc = INFINITY;
    int bi = 0x7fffffff;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const double c = __ldcg(a.part_c + b);
        const int ii = __ldcg(a.part_i + b);
        if (better(c, ii, bc, bi)) { bc = c; bi = ii; }
    }
    sc[threadIdx.x] = bc;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = kCostBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o && better(sc[threadIdx.x + o], si[threadIdx.x + o], sc[threadIdx.x], si[threadIdx.x])) {
            sc[threadIdx.x] = sc[threadIdx.x + o];
            si[threadIdx.x] = si[threadIdx.x + o];
        }
        __syncthreads();
    }
    __shared__ int best_s;
    if (threadIdx.x == 0) {
        int best = si[0];
        if (best == 0x7fffffff) best = 0;
        *a.argmin_state = best;
        if (a.argmin_out) *a.argmin_out = best;
        *a.n_window = n;
        *a.done = 0u;
        best_s = best;
    }
    __syncthreads();
    if (a.est_pose_out && threadIdx.x < 8) {
        const float4 p = a.pose[2 * best_s + (threadIdx.x >> 2)];
        const float v[4] = {p.x, p.y, p.z, p.w};
        a.est_pose_out[threadIdx.x] = v[threadIdx.x & 3];
    }
}

}  // namespace

int cost_blocks(int N) { return (N + kCostBlock - 1) / kCostBlock; }

cudaError_t launch_cost(const CostArgs &a, cudaStream_t s) {
    cost_kernel<<<cost_blocks(a.N), kCostBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ih
