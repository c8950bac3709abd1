// internal.cuh -- device-side records and FP32 helpers shared by the kernels
// of libinhand.so. Nothing here is part of the public ABI (include/inhand.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/inhand.h"

namespace ih {

constexpr int kDiverged = IH_ENV_NONFINITE | IH_ENV_ESCAPED | IH_ENV_OVERFLOW | IH_ENV_INVALID;
constexpr int kLinkStride = 3;  // float4 per link pose: (a, 0), (axis, 0), (quat wxyz)
constexpr int kCluster = 8;     // spheres per culling cluster (consecutive in the shape)

// Scene as seen by the kernels (device pointers, fixed at create).
struct DevScene {
    int n_shapes, n_fingers, n_links, n_pads, n_joints;
    float palm_hx, palm_hy, palm_hz;
    float link_len, link_rad;
    const float4 *spheres;      // [total] centroid-frame centre xyz, radius
    const int *shape_first;     // [n_shapes]
    const int *shape_count;     // [n_shapes]
    const float *shape_jinv;    // [n_shapes][6] inverse unit inertia xx yy zz xy xz yz
    const float *shape_bound;   // [n_shapes] bounding radius about the centroid
    const int *cl_first;        // [n_shapes] first cluster of each shape
    const float4 *clusters;     // [total clusters] centre (centroid frame), enclosing radius
    const float4 *finger_root;  // [F] x y z yaw
    const int *pad_link;        // [P]
    const float *pad_s0, *pad_s1;
};

struct DevConfig {
    float h;            // substep length
    int substeps;
    int iters;
    float margin, beta, slop, vmax;
    float gx, gy, gz;
    float tau, w_force, w_contact;
    int c_max;
    float escape_radius;
    int warm;           // warm-started solver (impulse cache per environment)
    int hand;           // 0: kinematic hand, 1: PD-driven joints
    float kp, kd, armature;   // joint PD gains and joint inertia
    float v_slip, w_slip;     // translational / rotational slip thresholds
    float w_full[10];         // weights of the full cost (PD hand)
};

// ---------------------------------------------------------------- FP32 math
struct V3 { float x, y, z; };
struct Q4 { float w, x, y, z; };

__host__ __device__ __forceinline__ V3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 xyz(float4 v) { return {v.x, v.y, v.z}; }

__device__ __forceinline__ Q4 qmul(Q4 a, Q4 b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
            a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
            a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ Q4 qnorm(Q4 q) {
    float s = rsqrtf(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
    return {q.w * s, q.x * s, q.y * s, q.z * s};
}
// rotate v by unit quaternion q: v + 2 w (u x v) + 2 u x (u x v)
__device__ __forceinline__ V3 qrot(Q4 q, V3 v) {
    V3 u = {q.x, q.y, q.z};
    V3 t = cross(u, v) * 2.0f;
    return v + t * q.w + cross(u, t);
}
__device__ __forceinline__ V3 qrot_inv(Q4 q, V3 v) { return qrot({q.w, -q.x, -q.y, -q.z}, v); }

// symmetric 3x3 stored as xx yy zz xy xz yz
struct S6 { float xx, yy, zz, xy, xz, yz; };
__device__ __forceinline__ V3 smul(const S6 &A, V3 v) {
    return {A.xx * v.x + A.xy * v.y + A.xz * v.z,
            A.xy * v.x + A.yy * v.y + A.yz * v.z,
            A.xz * v.x + A.yz * v.y + A.zz * v.z};
}
// columns of the rotation matrix of q
struct M3 { V3 c0, c1, c2; };
__device__ __forceinline__ M3 qmat(Q4 q) {
    M3 R;
    R.c0 = {1 - 2 * (q.y * q.y + q.z * q.z), 2 * (q.x * q.y + q.w * q.z), 2 * (q.x * q.z - q.w * q.y)};
    R.c1 = {2 * (q.x * q.y - q.w * q.z), 1 - 2 * (q.x * q.x + q.z * q.z), 2 * (q.y * q.z + q.w * q.x)};
    R.c2 = {2 * (q.x * q.z + q.w * q.y), 2 * (q.y * q.z - q.w * q.x), 1 - 2 * (q.x * q.x + q.y * q.y)};
    return R;
}
__device__ __forceinline__ V3 mmul(const M3 &R, V3 v) { return R.c0 * v.x + R.c1 * v.y + R.c2 * v.z; }
__device__ __forceinline__ V3 mtmul(const M3 &R, V3 v) { return {dot(R.c0, v), dot(R.c1, v), dot(R.c2, v)}; }

// W = R J^-1 R^T / m for symmetric J^-1 (body frame)
__device__ __forceinline__ S6 world_inv_inertia(const M3 &R, const S6 &Jb, float inv_m) {
    // columns of J R^T: rows of R are (c0.x, c1.x, c2.x) etc.
    V3 r0 = {R.c0.x, R.c1.x, R.c2.x}, r1 = {R.c0.y, R.c1.y, R.c2.y}, r2 = {R.c0.z, R.c1.z, R.c2.z};
    V3 a0 = smul(Jb, r0), a1 = smul(Jb, r1), a2 = smul(Jb, r2);
    S6 W;
    W.xx = dot(r0, a0) * inv_m; W.yy = dot(r1, a1) * inv_m; W.zz = dot(r2, a2) * inv_m;
    W.xy = dot(r0, a1) * inv_m; W.xz = dot(r0, a2) * inv_m; W.yz = dot(r1, a2) * inv_m;
    return W;
}

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al., "Parallel random numbers: as easy
// as 1, 2, 3" (SC'11): 10 rounds of a multiply-xor bijection on four 32-bit
// words, keyed by two 32-bit words bumped by the golden-ratio Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
__device__ __forceinline__ uint4 rng_words(uint64_t seed, uint32_t stream, uint32_t index,
                                           uint32_t env, uint32_t block) {
    return philox4x32_10(make_uint4(stream, index, env, block),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}
// uniform in (0, 1) from the top 53 bits of (hi, lo)
__device__ __forceinline__ double unit53(uint32_t hi, uint32_t lo) {
    const uint64_t b = ((uint64_t)hi << 21) | (lo >> 11);
    return ((double)b + 0.5) * 0x1.0p-53;
}
// two standard normals (Box-Muller, FP64) from one block
__device__ __forceinline__ void gauss2(uint4 w, double &z0, double &z1) {
    const double a = unit53(w.x, w.y), b = unit53(w.z, w.w);
    const double rad = sqrt(-2.0 * log(a));
    double s, c;
    sincospi(2.0 * b, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

// FP64 so(3) maps on (w, x, y, z) quaternions. FP64 instructions are scarce
// on this part (each warp instruction holds the pipe for many cycles), so the
// maps keep their count down: below a rotation of 1 rad the exponential's two
// factors come from their Taylor series, and each map divides once at most.
struct Q4d { double w, x, y, z; };
__device__ __forceinline__ Q4d qexp_d(double x, double y, double z) {
    const double t2 = x * x + y * y + z * z;
    if (t2 < 1.0) {
        // with u = (th / 2)^2 <= 1/4: cos(th / 2) = sum_n (-u)^n / (2n)! and
        // sin(th / 2) / th = (1/2) sum_n (-u)^n / (2n + 1)!, n <= 8 (the first
        // omitted terms are below 1e-18 of the sums)
        const double u = 0.25 * t2;
        double c = 1.0 / 20922789888000.0, sk = 1.0 / 355687428096000.0;   // 1/16!, 1/17!
        c = fma(c, -u, 1.0 / 87178291200.0);   sk = fma(sk, -u, 1.0 / 1307674368000.0);   // 1/14!, 1/15!
        c = fma(c, -u, 1.0 / 479001600.0);     sk = fma(sk, -u, 1.0 / 6227020800.0);      // 1/12!, 1/13!
        c = fma(c, -u, 1.0 / 3628800.0);       sk = fma(sk, -u, 1.0 / 39916800.0);        // 1/10!, 1/11!
        c = fma(c, -u, 1.0 / 40320.0);         sk = fma(sk, -u, 1.0 / 362880.0);          // 1/8!, 1/9!
        c = fma(c, -u, 1.0 / 720.0);           sk = fma(sk, -u, 1.0 / 5040.0);            // 1/6!, 1/7!
        c = fma(c, -u, 1.0 / 24.0);            sk = fma(sk, -u, 1.0 / 120.0);             // 1/4!, 1/5!
        c = fma(c, -u, 0.5);                   sk = fma(sk, -u, 1.0 / 6.0);               // 1/2!, 1/3!
        c = fma(c, -u, 1.0);                   sk = fma(sk, -u, 1.0);
        const double k = 0.5 * sk;
        return {c, x * k, y * k, z * k};
    }
    const double th = sqrt(t2);
    double s, c;
    sincos(0.5 * th, &s, &c);
    const double k = s / th;
    return {c, x * k, y * k, z * k};
}
__device__ __forceinline__ Q4d qmul_d(Q4d a, Q4d b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
            a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
            a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ Q4d qnorm_d(Q4d q) {
    const double r = rsqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
    return {q.w * r, q.x * r, q.y * r, q.z * r};
}
__device__ __forceinline__ void qlog_d(Q4d q, double out[3]) {
    if (q.w < 0) { q.w = -q.w; q.x = -q.x; q.y = -q.y; q.z = -q.z; }
    const double s = sqrt(q.x * q.x + q.y * q.y + q.z * q.z);
    if (s < 1e-300) { out[0] = out[1] = out[2] = 0.0; return; }
    const double k = 2.0 * atan2(s, q.w) / s;
    out[0] = q.x * k; out[1] = q.y * k; out[2] = q.z * k;
}

// ---------------------------------------------------------------- launches
// Declared here, defined in the kernel translation units.
cudaError_t launch_shape_setup(const float4 *spheres_in, float4 *spheres_out, const int *first,
                               const int *count, int n_shapes, float *jinv, float *bound,
                               const int *cl_first, float4 *clusters, cudaStream_t s);
cudaError_t launch_lpt_order(int N, const int *shape_count, const int *shape, const int *iters, int *scratch,
                             int *order, cudaStream_t s);
cudaError_t launch_fk(const DevScene &sc, const float *q, int n_frames, int substeps,
                      float4 *link_tab_out, cudaStream_t s);
cudaError_t launch_sample_initial(int N, float4 pose0, float4 quat0, float sigma_p, float sigma_r,
                                  float m_lo, float m_hi, float mu_lo, float mu_hi, uint64_t seed,
                                  float4 *pose, float4 *vel, float2 *params, int *status,
                                  cudaStream_t s);
cudaError_t launch_set_state(int N, int n_shapes, const float *pose, const float *vel,
                             const float *params, const int *shape_in, const int *iters_in,
                             float4 *pose_out, float4 *vel_out, float2 *params_out, int *shape,
                             int *iters, int *status, cudaStream_t s);

// Per-window arguments of a replayed tracking window, read by the kernels
// of the captured graph (written by a one-thread kernel before each replay).
struct WinDesc {
    int frame0;
    uint32_t update_index;
    const float *obs;     // [T][P][3]
    float *est;           // [T][8] or null
    int *argmin;          // [T] or null
};

struct StepArgs {
    DevScene sc;
    DevConfig cfg;
    int N;
    const float4 *link_tab;   // [frames][ns+1][Lk][3]
    int frame0, n_frames;
    float4 *pose, *vel;       // [N][2]
    const float2 *params;
    const int *shape, *iters;
    const int *order;         // [N] environment of each work slot (most work first), or null
    int *status;
    float *forces;            // [N][P][3]
    unsigned long long *work; // [6]
    // scoring fused at the end of the (single) frame; obs == null and win == null: no scoring
    const float *obs;         // [P][3]
    const WinDesc *win;       // when set: frame0, obs and outputs come from win (+ win_k)
    int win_k;
    double *c_sum, *c_mean;   // [N]
    int *n_window;
    double *cost_mean;        // [N] caller copy or null
    int *argmin_state, *argmin_out;
    float *est_pose_out;
    double *part_c;           // [grid] scratch
    int *part_i;              // [grid] scratch
    unsigned int *done;       // ticket
    // window mode (cm_frames != null): n_frames scored frames in one launch; each
    // environment writes its window mean and pose after every frame, and
    // launch_window_argmin takes each frame's argmin afterwards
    double *cm_frames;        // [n_frames][N]
    float4 *pose_frames;      // [n_frames][N][2]
    // warm start (cfg.warm): per environment the last substep's contacts
    float4 *cache;            // [N][c_max]: final impulse xyz, pair id (link << 8 | sphere) in w
    int *cache_n;             // [N]
    // contact staging: the first stage_cap contacts of an environment's substep
    // in shared memory, the rest (up to c_max) in a global spill area of
    // (c_max - stage_cap) x 4 float4 per resident group
    int stage_cap;
    float4 *spill;            // [grid * groups per block][c_max - stage_cap][4] or null
    int clp_cap;              // (link, cluster) pairs a group can hold
    int *queue;               // [2] work queue head, finished blocks (zero between launches) or null
};
// The step with the PD-driven hand (step_pd.cu): the joints are state.
struct PdArgs {
    DevScene sc;
    DevConfig cfg;
    int N;
    const float *cmd;         // [frames + 1][D] desired joint positions at frame boundaries
    int frame0, n_frames;
    float4 *pose, *vel;       // [N][2]
    const float2 *params;
    const int *shape, *iters;
    const int *order;         // [N] or null
    int *status;
    float *qj, *qdj;          // [N][D] joint angles and velocities
    float *forces;            // [N][P][3]
    float4 *pad_pose;         // [N][P][2]: (position, 0), (quaternion w x y z)
    float4 *slip;             // [N][P]: (d_x, d_y, flag bits, 0)
    unsigned long long *work; // [6]
    // window mode (pose_frames != null): n_frames frames, each frame's
    // observation, status and pose written out for the frames' cost launches
    float *fo_q;              // [n_frames][N][D]
    float4 *fo_pp;            // [n_frames][N][P][2]
    float *fo_forces;         // [n_frames][N][P][3]
    float4 *fo_slip;          // [n_frames][N][P]
    int *fo_status;           // [n_frames][N]
    float4 *pose_frames;      // [n_frames][N][2]
};
// The full cost of every frame of a PD window launch against the truth's
// observation of that frame: one thread per (frame, environment, term) forms
// a pad's terms (or the joints' term), then one thread per environment adds
// each frame's terms (joints first, pads in order) and the window sum and mean
// in frame order -- the cost kernel's functions in the cost kernel's order.
struct FramesCostArgs {
    int N, P, D, T;
    DevConfig cfg;
    const float *fo_q;        // [T][N][D]
    const float4 *fo_pp;      // [T][N][P][2]
    const float *fo_forces;   // [T][N][P][3]
    const float4 *fo_slip;    // [T][N][P]
    const int *fo_status;     // [T][N]
    const float *g_q;         // [T][D]
    const float4 *g_pose;     // [T][P][2]
    const float *g_forces;    // [T][P][3]
    const float4 *g_slip;     // [T][P]
    double *terms;            // [T][N][P + 1] scratch
    double *c_sum, *c_mean;   // [N]
    const int *n_window;
    double *cm_frames;        // [T][N]
};
cudaError_t launch_frames_cost_full(const FramesCostArgs &a, cudaStream_t s);
size_t pd_step_smem_bytes(int s_max, int c_max);
cudaError_t pd_step_prepare(int s_max, int c_max);
int pd_step_grid(int N, int sms);
cudaError_t launch_pd_step(const PdArgs &a, int grid, int s_max, cudaStream_t s);
cudaError_t launch_hand_rest(int N, int D, const float *q0, float *qj, float *qdj, cudaStream_t s);

struct StepVariant {
    int group;        // lanes per environment
    int cpl;          // register-resident contacts per lane
    int block;        // threads per CTA
};
cudaError_t launch_step(const StepArgs &a, const StepVariant &v, int grid, int s_max, cudaStream_t s);
int step_variant_max_contacts(const StepVariant &v);
bool step_variant_supported(const StepVariant &v);
size_t step_smem_bytes(const StepVariant &v, int s_max, int c_max, bool warm, int clp_cap);
// contacts a shape stages in shared memory (the rest of c_max spill to global memory)
int step_stage_capacity(const StepVariant &v, int c_max);
int step_variant_list(StepVariant *out, int cap);

struct CostArgs {
    int N, P;
    DevConfig cfg;
    const float *forces;     // [N][P][3]
    const float *obs;        // [P][3]
    const int *status;
    double *c_sum;           // [N] window sums
    double *c_mean;          // [N] window means (handle-owned, read by the optimizer)
    int *n_window;           // device counter
    double *cost_mean;       // [N] caller copy or null
    const float4 *pose;      // for est_pose
    int *argmin_state;       // handle's i*
    int *argmin_out;         // user or null
    float *est_pose_out;     // user float[8] or null
    double *part_c;          // [blocks] scratch
    int *part_i;             // [blocks] scratch
    unsigned int *done;      // scratch ticket (zero between launches)
    // full cost (qj non-null, PD hand): the environments' observation against
    // the ground truth's (obs holds its forces)
    const float *qj;         // [N][D]
    const float4 *pad_pose;  // [N][P][2]
    const float4 *slip;      // [N][P]
    const float *g_q;        // [D]
    const float4 *g_pose;    // [P][2]
    const float4 *g_slip;    // [P]
    int D;
};
cudaError_t launch_cost(const CostArgs &a, cudaStream_t s);
int cost_blocks(int N);
// argmin and estimate of every frame of a window-mode step launch (outputs from
// win when set, else argmin_out [T] / est_out [T][8], either may be null);
// advances the window counter by T and sets the handle's i* to the last frame's
// (each skipped when its pointer is null)
cudaError_t launch_window_argmin(int N, int T, const double *cm_frames, const float4 *pose_frames,
                                 const WinDesc *win, int *argmin_out, float *est_out, int *argmin_state,
                                 int *n_window, cudaStream_t s);

constexpr int kOptBlock = 32;   // elites / environments per block in the grid kernels
constexpr int kMoments = 45;    // sum w, sum w d (8), sum w d d^T (36, lower triangle)

struct OptArgs {
    int N;
    float elite_frac;
    double floor_var[8];
    float m_lo, m_hi, mu_lo, mu_hi;
    uint64_t seed;
    uint32_t update_index;
    const double *c_mean;     // [N] window means
    double *c_sum;            // [N] reset by apply
    int *n_window;            // reset by apply
    float4 *pose, *vel;
    float2 *params;
    int *status;
    // scratch
    unsigned char *is_elite;  // [N]
    int *rank;                // [N] rank among elites or among non-elites
    int *elite_env;           // [N] elites in index order (first k used)
    double *elite_w;          // [N] unnormalised weights, then inclusive prefix within its block
    double *block_w;          // [blocks] weight sum per block, then exclusive offsets
    double *moments;          // [blocks][kMoments]
    double *misc;             // [80]: L (64), k, u, i*, ok, wsum, cmin, sd, nfin, nblocks
    int *argmin_state;
    int *argmin_out;
    int *parent_out;
    const WinDesc *win;       // when set, update_index comes from win
    // WRS / REPS (kind 1 / 2): PMF over all simulations, draws with replacement
    int kind;
    double wrs_lambda, reps_epsilon;
    float sigma_pose[6], sigma_theta[2], sigma_vel[6];
    int explore_velocity;
    float4 *sn_pose, *sn_vel; // [N][2] state before the update
    float2 *sn_params;        // [N]
    int *sn_status;           // [N]
    int *cache_n;             // warm-start cache counts, or null: a replaced environment starts cold
    // PD-driven hand: a replaced environment takes its parent's joints (null: kinematic hand)
    float *qj, *qdj;          // [N][D]
    int D;
    float *sn_qj, *sn_qdj;    // [N][D] joints before the update (WRS / REPS)
};
int opt_blocks(int N);

// One step of the refinement of the elites (sim_refine_elites), taken by the
// adjoint launch that evaluated the step's trial.
struct RefineArgs {
    int k;
    const int *elite;             // [k] environments
    float4 *tr_pose;              // [N][2] trial states (elites' entries)
    float2 *tr_params;            // [N]
    float4 *best_pose;            // [k][2]
    float2 *best_params;          // [k]
    float *best_grad;             // [k][8]
    double *best_c, *c0;          // [k] best cost so far, cost of the unrefined state
    float *scale;                 // [k] step multiplier (halved on a rejected trial)
    const double *cost;           // [k] cost at the trial
    const float *grad;            // [k][8] gradient at the trial
    const float4 *end_pose, *end_vel;    // [k][2] end state of the trial's window
    float4 *best_end_pose, *best_end_vel;  // [k][2] end state of the best trial
    unsigned long long *accepted; // [k] bit j set when evaluation j was kept
    float eta[8];                 // step length per coordinate
    float m_lo, m_hi, mu_lo, mu_hi;
    int step;                     // 0: the first evaluation (of the unrefined state)
    int last;                     // 1: restore the best state instead of stepping, then commit
    const float4 *ws_pose;        // [N][2] window-start states: the first evaluation's trial
    const float2 *ws_params;      // [N]
    // the commit: an improved elite's live end state, parameters and window cost
    float4 *pose, *vel;           // [N][2]
    float2 *params;               // [N]
    double *c_sum, *c_mean;       // [N]
    const int *n_window;
};

// Reverse-mode derivative of the tracking cost over a horizon (adjoint.cu).
struct AdjArgs {
    DevScene sc;
    DevConfig cfg;
    int N;                    // environments in the handle
    int n;                    // environments differentiated (slots)
    const int *envs;          // [n] environment of each slot, or null: slot = environment
    const float4 *link_tab;   // [frames][ns+1][Lk][3]
    int frame0, H, K;         // first frame, horizon, checkpoint interval (frames)
    const float4 *pose, *vel; // [N][2] state at the start of frame0 (read only)
    const float2 *params;
    const int *shape, *iters, *status;
    const float *obs;         // [H][P][3]
    float beta_s;             // slope of the smoothed normal clamp (1 / (N s))
    float width;              // relative width of the smoothed friction-disk clamp
    double *cost;             // [n] or null
    float *grad;              // [n][8]: position, rotation vector (world frame, left), m, mu
    float *grad_quat;         // [n][4] derivative w.r.t. the quaternion's components, or null
    float *scratch;           // [n][stride] floats
    size_t stride;
    int iters_max;
    int forward_only;         // 1: cost (and end state) only, no reverse sweep
    int seg_tape;             // 1: tape every substep of a segment (else re-run each substep to tape it)
    int zero;                 // always 0: combined with the forward substep's flags so that they are
                              // run-time values and the substep is compiled once for every pass
    int gw, pl;               // kernel shape: warps per environment, register contacts per thread (0, 0: automatic)
    int s_max;                // most spheres in one shape of the scene
    int refine;               // 1: each slot's group then takes the refinement step rf for its elite
    RefineArgs rf;
    float4 *out_pose, *out_vel;   // [n][2] end state of each slot, or null
};

// Gradient refinement of the elites (adjoint.cu): accept or reject the last
// trial of every elite, then step from its best state.
// copy refined elites (end state [k][2], parameters, window cost) into the live state
size_t adjoint_scratch_floats(int H, int K, int substeps, int n_pads, int c_max, int iters_max, bool seg_tape);
cudaError_t launch_adjoint(const AdjArgs &a, cudaStream_t s);
bool adjoint_variant_supported(int gw, int pl);   // (0, 0) = automatic
cudaError_t launch_adjoint_iters_max(int n, int N, const int *envs, const int *iters, int *out, cudaStream_t s);
cudaError_t launch_win_desc(WinDesc *d, WinDesc v, cudaStream_t s);
// shared-memory opt-in of a shape; blocks_per_sm (may be null) receives its occupancy
cudaError_t step_prepare(const StepVariant &v, int s_max, int c_max, bool warm, int clp_cap, int *blocks_per_sm);
// the warm-started instances (step_warm.cu)
size_t step_smem_bytes_warm(const StepVariant &v, int s_max, int c_max, int clp_cap);
cudaError_t step_prepare_warm(const StepVariant &v, int s_max, int c_max, int clp_cap, int *blocks_per_sm);
cudaError_t launch_step_warm(const StepArgs &a, const StepVariant &v, int grid, int s_max, cudaStream_t s);
cudaError_t launch_optimizer(const OptArgs &a, cudaStream_t s);
// the optimizer's first stage alone: elite flags, ranks and elite_env (index order), i*
cudaError_t launch_select(const OptArgs &a, cudaStream_t s);

}  // namespace ih
