// cost.cu -- per-environment cost against the observed sensor forces and the
// argmin estimate (Sec. III-C; Eqs. 1-2 with the running mean of Algorithm 1).
//
// One thread per environment accumulates, in FP64,
//   cost_i = sum_l [ w_force |c_il - o_l|^2 + w_contact ((|c_il|^2 > tau^2) != (|o_l|^2 > tau^2)) ]
// into the window sum and forms C_i = sum / n (n = frames in the window).
// FP64 issue is scarce on this part, so blocks are one warp wide and spread
// over as many SMs as there are warps of environments. Each warp reduces
// (C_i, i) to its minimum with shuffles and leaves it in scratch; the last
// warp to finish (atomic ticket) reduces the partials, publishes i*, copies
// the pose of i*, advances the window count and re-arms the ticket.
#include "full_cost.cuh"
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kCostBlock = 32;

__device__ __forceinline__ bool better(double ca, int ia, double cb, int ib) {
    return ca < cb || (ca == cb && ia < ib);
}

__device__ __forceinline__ void warp_min(double &c, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xffffffffu, c, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(oc, oi, c, i)) { c = oc; i = oi; }
    }
}

// The full cost of the PD hand's observation (full_cost.cuh): the joints'
// term, then each pad's terms in pad order.
__device__ double frame_cost_full(const CostArgs &a, int i) {
    const int D = a.D, P = a.P;
    double w[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) w[k] = (double)a.cfg.w_full[k];
    double c = full_cost_joints(a.qj + (size_t)i * D, a.g_q, D, w[0]);
    for (int l = 0; l < P; ++l) {
        const size_t o = (size_t)i * P + l;
        c = __dadd_rn(c, full_cost_pad(w, (double)a.cfg.tau, a.pad_pose[2 * o], a.pad_pose[2 * o + 1], a.g_pose[2 * l],
                                       a.g_pose[2 * l + 1], a.forces + 3 * o, a.obs + 3 * l, a.slip[o], a.g_slip[l]));
    }
    return c;
}

__global__ void __launch_bounds__(kCostBlock) cost_kernel(const CostArgs a) {
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = *a.n_window + 1;
    double cm = INFINITY;
    int ci = 0x7fffffff;
    if (i < a.N) {
        double c = 0.0;
        if (a.status[i] & kDiverged) {
            c = INFINITY;
        } else if (a.qj) {
            c = frame_cost_full(a, i);
        } else {
            // evaluated in the order written, without fused multiply-adds
            const float *f = a.forces + (size_t)i * a.P * 3;
            const double tau = (double)a.cfg.tau, wf = (double)a.cfg.w_force;
            const double tau2 = __dmul_rn(tau, tau);
            for (int l = 0; l < a.P; ++l) {
                const double fx = f[3 * l], fy = f[3 * l + 1], fz = f[3 * l + 2];
                const double ox = a.obs[3 * l], oy = a.obs[3 * l + 1], oz = a.obs[3 * l + 2];
                const double dx = __dsub_rn(fx, ox), dy = __dsub_rn(fy, oy), dz = __dsub_rn(fz, oz);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                c = __dadd_rn(c, __dmul_rn(wf, d2));
                const double ns = __dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz));
                const double no = __dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz));
                if ((ns > tau2) != (no > tau2)) c = __dadd_rn(c, (double)a.cfg.w_contact);
            }
        }
        const double s = __dadd_rn(a.c_sum[i], c);
        a.c_sum[i] = s;
        cm = __ddiv_rn(s, (double)n);
        a.c_mean[i] = cm;
        if (a.cost_mean) a.cost_mean[i] = cm;
        if (isnan(cm)) cm = INFINITY;
        ci = i;
    }
    warp_min(cm, ci);
    if (threadIdx.x == 0) {
        a.part_c[blockIdx.x] = cm;
        a.part_i[blockIdx.x] = ci;
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
    warp_min(bc, bi);
    const int best = (bi == 0x7fffffff) ? 0 : bi;
    if (threadIdx.x == 0) {
        *a.argmin_state = best;
        if (a.argmin_out) *a.argmin_out = best;
        *a.n_window = n;
        *a.done = 0u;
    }
    if (a.est_pose_out && threadIdx.x < 8) {
        const float4 p = a.pose[2 * best + (threadIdx.x >> 2)];
        const float v[4] = {p.x, p.y, p.z, p.w};
        a.est_pose_out[threadIdx.x] = v[threadIdx.x & 3];
    }
}

}  // namespace

int cost_blocks(int N) { return (N + kCostBlock - 1) / kCostBlock; }

namespace {
// One thread per (frame, environment, term) of a PD window: term p < P is pad
// p's terms, term P the joints' term (skipped for an environment diverged by
// that frame, which scores +inf).
constexpr int kTermsBlock = 128;
__global__ void __launch_bounds__(kTermsBlock) frames_terms_kernel(const FramesCostArgs a) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int P1 = a.P + 1;
    if (k >= (size_t)a.T * a.N * P1) return;
    const int p = (int)(k % P1);
    const size_t ef = k / P1;   // frame * N + environment
    const int f = (int)(ef / a.N);
    if (a.fo_status[ef] & kDiverged) return;
    double w[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) w[q] = (double)a.cfg.w_full[q];
    double t;
    if (p == a.P) {
        t = full_cost_joints(a.fo_q + ef * a.D, a.g_q + (size_t)f * a.D, a.D, w[0]);
    } else {
        const size_t o = ef * a.P + p, g = (size_t)f * a.P + p;
        t = full_cost_pad(w, (double)a.cfg.tau, a.fo_pp[2 * o], a.fo_pp[2 * o + 1], a.g_pose[2 * g],
                          a.g_pose[2 * g + 1], a.fo_forces + 3 * o, a.g_forces + 3 * g, a.fo_slip[o], a.g_slip[g]);
    }
    a.terms[k] = t;
}

// One warp per environment, lane f for frame f (32 frames per round): each
// frame's cost (the joints' term, then the pads' in pad order, as
// frame_cost_full adds them) on its lane, the window sum in frame order (every
// lane runs the same chain of additions) and each frame's mean on its lane --
// the additions and divisions cost_kernel makes frame by frame.
constexpr int kMeanBlock = 128;
__global__ void __launch_bounds__(kMeanBlock) frames_mean_kernel(const FramesCostArgs a) {
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= a.N) return;   // whole warps
    const int n0 = *a.n_window, P1 = a.P + 1;
    double s = a.c_sum[i];
    for (int f0 = 0; f0 < a.T; f0 += 32) {
        const int f = f0 + lane;
        double c = INFINITY;
        if (f < a.T) {
            const size_t ef = (size_t)f * a.N + i;
            if (!(a.fo_status[ef] & kDiverged)) {
                const double *t = a.terms + ef * P1;
                c = t[a.P];
                for (int p = 0; p < a.P; ++p) c = __dadd_rn(c, t[p]);
            }
        }
        const int nf = min(32, a.T - f0);
        double sf = 0.0;   // the window sum after this lane's frame
        for (int k = 0; k < nf; ++k) {
            s = __dadd_rn(s, __shfl_sync(0xffffffffu, c, k));
            if (lane == k) sf = s;
        }
        if (f < a.T) {
            const double cm = __ddiv_rn(sf, (double)(n0 + f + 1));
            a.cm_frames[(size_t)f * a.N + i] = cm;
            if (f == a.T - 1) {
                a.c_sum[i] = sf;
                a.c_mean[i] = cm;
            }
        }
    }
}
}  // namespace

cudaError_t launch_frames_cost_full(const FramesCostArgs &a, cudaStream_t s) {
    if (a.N < 1 || a.T < 1) return cudaSuccess;
    const size_t total = (size_t)a.T * a.N * (a.P + 1);
    frames_terms_kernel<<<(unsigned)((total + kTermsBlock - 1) / kTermsBlock), kTermsBlock, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    frames_mean_kernel<<<(unsigned)(((size_t)a.N * 32 + kMeanBlock - 1) / kMeanBlock), kMeanBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cost(const CostArgs &a, cudaStream_t s) {
    cost_kernel<<<cost_blocks(a.N), kCostBlock, 0, s>>>(a);
    return cudaGetLastError();
}

namespace {
// One block per frame of a window-mode launch: the lowest (C_i, i) of that
// frame's window means (NaN = +inf), the pose of that environment after the
// frame, and -- for the window's last frame, when argmin_state is set -- the
// handle's i*.
__global__ void __launch_bounds__(1024) window_argmin_kernel(int N, int T, const double *cm_frames,
                                                              const float4 *pose_frames, const WinDesc *win,
                                                              int *argmin_out, float *est_out, int *argmin_state,
                                                              int *n_window) {
    __shared__ double sc[32];
    __shared__ int si[32];
    __shared__ int best_s;
    const int f = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    double bc = INFINITY;
    int bi = 0x7fffffff;
    for (int i = t; i < N; i += blockDim.x) {
        double c = cm_frames[(size_t)f * N + i];
        if (isnan(c)) c = INFINITY;
        if (c < bc || (c == bc && i < bi)) { bc = c; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oc < bc || (oc == bc && oi < bi)) { bc = oc; bi = oi; }
    }
    if (lane == 0) { sc[wid] = bc; si[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
        const int nw = (int)(blockDim.x >> 5);
        bc = lane < nw ? sc[lane] : INFINITY;
        bi = lane < nw ? si[lane] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) { bc = oc; bi = oi; }
        }
        if (lane == 0) {
            const int best = (bi == 0x7fffffff) ? 0 : bi;
            best_s = best;
            int *am = win ? win->argmin : argmin_out;
            if (am) am[f] = best;
            if (f == T - 1 && argmin_state) *argmin_state = best;
            if (f == 0 && n_window) *n_window += T;
        }
    }
    __syncthreads();
    float *est = win ? win->est : est_out;
    if (est && t < 8) {
        const float4 p = pose_frames[2 * ((size_t)f * N + best_s) + (t >> 2)];
        const float v[4] = {p.x, p.y, p.z, p.w};
        est[8 * f + t] = v[t & 3];
    }
}
}  // namespace

cudaError_t launch_window_argmin(int N, int T, const double *cm_frames, const float4 *pose_frames,
                                 const WinDesc *win, int *argmin_out, float *est_out, int *argmin_state,
                                 int *n_window, cudaStream_t s) {
    window_argmin_kernel<<<T, 1024, 0, s>>>(N, T, cm_frames, pose_frames, win, argmin_out, est_out, argmin_state,
                                            n_window);
    return cudaGetLastError();
}

}  // namespace ih
