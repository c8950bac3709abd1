// api.cu -- host side of the C ABI declared in include/inhand.h: argument
// checks, device allocations owned by the handle, and kernel launches on the
// handle's stream. No arithmetic of the method runs here.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace ih;

struct ih_sim {
    // scene
    int n_shapes = 0, n_fingers = 0, n_links = 0, n_pads = 0, n_joints = 0, total_spheres = 0;
    float palm_half[3] = {0, 0, 0};
    float link_len = 0, link_rad = 0;
    // config
    ih_config cfg{};
    DevConfig dcfg{};
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    StepVariant variant{32, 4, 128};
    int step_grid = 0;
    int s_max = 1;   // most spheres in one shape
    int sms = 1;     // SMs of the device
    int stage_cap = 0, clp_cap = 0;   // the step shape's shared-memory staging; (link, cluster) pair capacity
    float4 *spill = nullptr;          // contacts beyond the staging capacity, per resident group
    size_t spill_f4 = 0;              // its size in float4
    int *queue = nullptr;             // the step's work queue (head, finished blocks)
    // device buffers
    float4 *spheres_raw = nullptr, *spheres = nullptr, *finger_root = nullptr;
    int *shape_first = nullptr, *shape_count = nullptr, *pad_link = nullptr;
    float *shape_jinv = nullptr, *shape_bound = nullptr, *pad_s0 = nullptr, *pad_s1 = nullptr;
    int *cl_first = nullptr;
    float4 *clusters = nullptr;
    float4 *link_tab = nullptr;
    float4 *pose = nullptr, *vel = nullptr;
    float2 *params = nullptr;
    int *shape = nullptr, *iters = nullptr, *status = nullptr;
    int *order = nullptr, *lpt_scratch = nullptr;
    float *forces = nullptr;
    double *c_sum = nullptr, *c_mean = nullptr;
    int *n_window = nullptr, *argmin = nullptr;
    double *part_c = nullptr;
    int *part_i = nullptr;
    unsigned int *done = nullptr;
    unsigned long long *work = nullptr;
    unsigned char *is_elite = nullptr;
    int *rank = nullptr, *elite_env = nullptr;
    double *elite_w = nullptr, *block_w = nullptr, *moments = nullptr, *misc = nullptr;
    WinDesc *win = nullptr;
    std::vector<void *> owned;
    // adjoint scratch (grown on demand, freed in sim_destroy)
    float *adj_scratch = nullptr;
    size_t adj_floats = 0;
    size_t adj_budget = (size_t)16 << 30;   // bytes of adjoint scratch for whole-segment taping
    bool adj_seg = false;
    int adj_gw = 0, adj_pl = 0;   // the adjoint kernel's shape (0, 0: automatic)
    int iters_max_all = -1;       // the largest iteration count of any environment (-1: to be read)
    int *adj_word = nullptr;
    // gradient refinement: window-start snapshot, trial, best and end states (allocated on first use)
    bool rf_alloc = false, ws_valid = false;
    int ws_frames = 0;
    float4 *ws_pose = nullptr, *ws_vel = nullptr, *tr_pose = nullptr, *end_pose = nullptr, *end_vel = nullptr,
           *best_pose = nullptr, *best_end_pose = nullptr, *best_end_vel = nullptr;
    float2 *ws_params = nullptr, *tr_params = nullptr, *best_params = nullptr;
    float *best_grad = nullptr, *scale = nullptr, *r_grad = nullptr;
    double *best_c = nullptr, *c0 = nullptr, *r_cost = nullptr;
    unsigned long long *r_acc = nullptr;
    // WRS / REPS: the state before an update
    float4 *sn_pose = nullptr, *sn_vel = nullptr;
    float2 *sn_params = nullptr;
    int *sn_status = nullptr;
    // warm-started solver: per environment the last substep's contacts (impulse, pair id)
    float4 *cache = nullptr;
    int *cache_n = nullptr;
    // PD-driven hand: commands, joints, the full observation
    bool pd = false;
    float *cmd = nullptr;               // [max_frames + 1][D] desired joint positions
    float *qj = nullptr, *qdj = nullptr; // [N][D]
    float4 *pad_pose = nullptr;         // [N][P][2]
    float4 *slip = nullptr;             // [N][P]
    float *sn_qj = nullptr, *sn_qdj = nullptr;
    int pd_grid = 0;
    // captured tracking window (replayed by sim_track_window)
    cudaGraphExec_t win_exec = nullptr;
    cudaStream_t cap_stream = nullptr;          // private stream: capture and replay
    cudaStream_t cap_side = nullptr;            // the window graph's second branch (capture only)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
    int win_T = 0;
    double *wf_cm = nullptr;        // [T][N] window means of every frame (window-mode launches)
    float4 *wf_pose = nullptr;      // [T][N][2] poses of every frame
    int wf_T = 0;
    // PD window launches: every frame's observation and status, the cost terms
    float *fo_q = nullptr, *fo_forces = nullptr;
    float4 *fo_pp = nullptr, *fo_slip = nullptr;
    int *fo_status = nullptr;
    double *fo_terms = nullptr;
    int fo_T = 0;
    int frames_T = 0;               // frames of the last sim_step_frames call, not yet scored
    StepVariant win_variant{0, 0, 0};
    ih_opt_config win_opt{};
    // host bookkeeping
    std::vector<char> frame_ready;   // commands uploaded for frame f
    int window_frames = 0;           // frames scored since the last reset
    bool stepped = false;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

ih_status fail(ih_sim *s, ih_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf; else g_create_err = buf;
    return code;
}

ih_status cuda_fail(ih_sim *s, cudaError_t e, const char *what) {
    return fail(s, e == cudaErrorMemoryAllocation ? IH_ERR_OOM : IH_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

ih_status refuse_pd(ih_sim *s, const char *what) {
    return fail(s, IH_ERR_ARG, "%s is not available with the PD-driven hand (use sim_step and cost_eval_full)", what);
}

// frames scored by sim_step_frames wait for sim_frames_argmin (which advances
// the window counter); no other scored call may come in between
ih_status check_no_pending(ih_sim *s) {
    if (s->frames_T > 0)
        return fail(s, IH_ERR_STATE, "sim_frames_argmin must follow sim_step_frames before further scoring");
    return IH_OK;
}

template <typename T>
cudaError_t dalloc(ih_sim *s, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    s->owned.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

DevScene dev_scene(const ih_sim *s) {
    DevScene d;
    d.n_shapes = s->n_shapes; d.n_fingers = s->n_fingers; d.n_links = s->n_links;
    d.n_pads = s->n_pads; d.n_joints = s->n_joints;
    d.palm_hx = s->palm_half[0]; d.palm_hy = s->palm_half[1]; d.palm_hz = s->palm_half[2];
    d.link_len = s->link_len; d.link_rad = s->link_rad;
    d.spheres = s->spheres; d.shape_first = s->shape_first; d.shape_count = s->shape_count;
    d.shape_jinv = s->shape_jinv; d.shape_bound = s->shape_bound; d.finger_root = s->finger_root;
    d.cl_first = s->cl_first; d.clusters = s->clusters;
    d.pad_link = s->pad_link; d.pad_s0 = s->pad_s0; d.pad_s1 = s->pad_s1;
    return d;
}

// Default step-kernel shape before any autotuning: few environments get a
// whole CTA each (latency bound), many get one warp each (issue bound); the
// register-resident contacts per thread must cover c_max.
StepVariant default_variant(int N, int c_max) {
    (void)c_max;   // every shape holds any c_max
    return N <= 4096 ? StepVariant{64, 2, 128} : StepVariant{32, 2, 128};
}

int grid_for(const StepVariant &v, int N) {
    const int groups_per_block = v.block / v.group;
    const int need = (N + groups_per_block - 1) / groups_per_block;
    return need > 0 ? need : 1;
}

// Make v the step shape: shared-memory opt-in, a persistent grid of at most the
// blocks that fit on the device at once (the groups take environments from the
// launch's work queue), and a spill area for the contacts beyond the shape's
// shared-memory staging, grown when needed (cudaFree synchronises the device,
// so no launch still uses the old one).
cudaError_t use_variant(ih_sim *s, const StepVariant &v) {
    int bps = 0;
    cudaError_t e = step_prepare(v, s->s_max, s->cfg.c_max, s->dcfg.warm != 0, s->clp_cap, &bps);
    if (e != cudaSuccess) return e;
    const int resident = std::max(1, bps) * std::max(1, s->sms);
    const int grid = std::min(grid_for(v, s->cfg.n_envs), resident);
    const int sc = step_stage_capacity(v, s->cfg.c_max);
    const size_t need = (size_t)grid * (v.block / v.group) * (size_t)(s->cfg.c_max - sc) * 4;
    if (need > s->spill_f4) {
        // a captured window graph holds the old spill pointer: let it finish, capture again
        if (s->cap_stream) cudaStreamSynchronize(s->cap_stream);
        cudaStreamSynchronize(s->stream);
        if (s->win_exec) { cudaGraphExecDestroy(s->win_exec); s->win_exec = nullptr; }
        if (s->spill) cudaFree(s->spill);
        s->spill = nullptr;
        s->spill_f4 = 0;
        e = cudaMalloc(&s->spill, need * sizeof(float4));
        if (e != cudaSuccess) { s->spill = nullptr; return e; }
        s->spill_f4 = need;
    }
    s->variant = v;
    s->step_grid = grid;
    s->stage_cap = sc;
    return cudaSuccess;
}

}  // namespace

extern "C" {

ih_status sim_create(const ih_scene *sc, const ih_config *cfg, uint64_t seed, void *stream,
                     ih_sim **out) {
    if (!sc || !cfg || !out) return fail(nullptr, IH_ERR_ARG, "null argument");
    *out = nullptr;
    if (sc->n_shapes < 1 || !sc->shape_first || !sc->shape_count || !sc->spheres)
        return fail(nullptr, IH_ERR_ARG, "scene needs at least one shape");
    if (sc->n_fingers < 0 || sc->n_fingers > IH_MAX_FINGERS)
        return fail(nullptr, IH_ERR_ARG, "n_fingers must be in [0, %d]", IH_MAX_FINGERS);
    if (sc->n_fingers > 0 && !sc->finger_root) return fail(nullptr, IH_ERR_ARG, "finger_root is null");
    if (sc->n_pads < 1 || sc->n_pads > IH_MAX_PADS || !sc->pad_link || !sc->pad_s0 || !sc->pad_s1)
        return fail(nullptr, IH_ERR_ARG, "n_pads must be in [1, %d] with pad arrays", IH_MAX_PADS);
    if (!finite_pos(sc->palm_half[0]) || !finite_pos(sc->palm_half[1]) || !finite_pos(sc->palm_half[2]) ||
        !finite_pos(sc->link_len) || !(sc->link_rad >= 0.0f))
        return fail(nullptr, IH_ERR_ARG, "palm and link dimensions must be positive");
    const int n_links = 1 + 4 * sc->n_fingers;
    int total = 0, s_max_scene = 1;
    for (int k = 0; k < sc->n_shapes; ++k) {
        const int f = sc->shape_first[k], c = sc->shape_count[k];
        if (c < 1 || c > IH_MAX_SPHERES || f < 0)
            return fail(nullptr, IH_ERR_ARG, "shape %d: count must be in [1, %d]", k, IH_MAX_SPHERES);
        total = std::max(total, f + c);
        s_max_scene = std::max(s_max_scene, c);
    }
    for (int j = 0; j < total; ++j)
        if (!(sc->spheres[4 * j + 3] > 0.0f) || !std::isfinite(sc->spheres[4 * j]) ||
            !std::isfinite(sc->spheres[4 * j + 1]) || !std::isfinite(sc->spheres[4 * j + 2]))
            return fail(nullptr, IH_ERR_ARG, "sphere %d is invalid", j);
    for (int p = 0; p < sc->n_pads; ++p) {
        if (sc->pad_link[p] < 0 || sc->pad_link[p] >= n_links || !(sc->pad_s0[p] <= sc->pad_s1[p]))
            return fail(nullptr, IH_ERR_ARG, "pad %d is invalid", p);
        int same = 0;
        for (int k = 0; k < sc->n_pads; ++k) same += sc->pad_link[k] == sc->pad_link[p];
        if (same > 4) return fail(nullptr, IH_ERR_ARG, "more than 4 pads on link %d", sc->pad_link[p]);
    }
    if (cfg->n_envs < 1 || cfg->max_frames < 1 || cfg->substeps < 1 || cfg->iters < 0 ||
        !finite_pos(cfg->frame_dt) || !(cfg->margin >= 0.0f) || !(cfg->beta >= 0.0f) ||
        !(cfg->slop >= 0.0f) || !(cfg->vmax >= 0.0f) || !(cfg->tau >= 0.0f) ||
        cfg->c_max < 1 || cfg->c_max > IH_MAX_CONTACTS || !finite_pos(cfg->escape_radius) ||
        (cfg->warm_start != 0 && cfg->warm_start != 1))
        return fail(nullptr, IH_ERR_ARG, "invalid config");
    if (cfg->hand != IH_HAND_KINEMATIC && cfg->hand != IH_HAND_PD) return fail(nullptr, IH_ERR_ARG, "unknown hand");
    if (cfg->hand == IH_HAND_PD) {
        if (!(cfg->kp >= 0.0f) || !(cfg->kd >= 0.0f) || !finite_pos(cfg->armature) || !std::isfinite(cfg->kp) ||
            !std::isfinite(cfg->kd) || !(cfg->v_slip >= 0.0f) || !(cfg->w_slip >= 0.0f))
            return fail(nullptr, IH_ERR_ARG, "invalid PD hand constants");
        if (cfg->warm_start) return fail(nullptr, IH_ERR_ARG, "warm_start is not available with the PD-driven hand");
        for (int k = 0; k < 10; ++k)
            if (!(cfg->w_full[k] >= 0.0f) || !std::isfinite(cfg->w_full[k]))
                return fail(nullptr, IH_ERR_ARG, "w_full[%d] is invalid", k);
    }

    ih_sim *s = new ih_sim();
    s->n_shapes = sc->n_shapes; s->n_fingers = sc->n_fingers; s->n_links = n_links;
    s->n_pads = sc->n_pads; s->n_joints = 4 * sc->n_fingers; s->total_spheres = total;
    s->s_max = s_max_scene;
    for (int k = 0; k < 3; ++k) s->palm_half[k] = sc->palm_half[k];
    s->link_len = sc->link_len; s->link_rad = sc->link_rad;
    s->cfg = *cfg;
    s->seed = seed;
    s->stream = static_cast<cudaStream_t>(stream);
    DevConfig &d = s->dcfg;
    d.h = cfg->frame_dt / (float)cfg->substeps;
    d.substeps = cfg->substeps; d.iters = cfg->iters;
    d.margin = cfg->margin; d.beta = cfg->beta; d.slop = cfg->slop; d.vmax = cfg->vmax;
    d.gx = cfg->gravity[0]; d.gy = cfg->gravity[1]; d.gz = cfg->gravity[2];
    d.tau = cfg->tau; d.w_force = cfg->w_force; d.w_contact = cfg->w_contact;
    d.c_max = cfg->c_max; d.escape_radius = cfg->escape_radius;
    d.warm = cfg->warm_start;
    d.hand = cfg->hand;
    d.kp = cfg->kp; d.kd = cfg->kd; d.armature = cfg->armature; d.v_slip = cfg->v_slip; d.w_slip = cfg->w_slip;
    for (int k = 0; k < 10; ++k) d.w_full[k] = cfg->w_full[k];
    s->pd = cfg->hand == IH_HAND_PD;
    s->variant = default_variant(cfg->n_envs, cfg->c_max);
    const int N = cfg->n_envs, P = sc->n_pads, F = sc->n_fingers;

    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(s, &s->spheres_raw, total)); A(dalloc(s, &s->spheres, total));
    A(dalloc(s, &s->shape_first, sc->n_shapes)); A(dalloc(s, &s->shape_count, sc->n_shapes));
    A(dalloc(s, &s->shape_jinv, 6 * sc->n_shapes)); A(dalloc(s, &s->shape_bound, sc->n_shapes));
    std::vector<int> cl_first(sc->n_shapes);
    int n_clusters = 0;
    for (int k = 0; k < sc->n_shapes; ++k) {
        cl_first[k] = n_clusters;
        n_clusters += (sc->shape_count[k] + kCluster - 1) / kCluster;
    }
    A(dalloc(s, &s->cl_first, sc->n_shapes)); A(dalloc(s, &s->clusters, n_clusters));
    A(dalloc(s, &s->finger_root, F > 0 ? F : 1));
    A(dalloc(s, &s->pad_link, P)); A(dalloc(s, &s->pad_s0, P)); A(dalloc(s, &s->pad_s1, P));
    A(dalloc(s, &s->link_tab, (size_t)cfg->max_frames * (cfg->substeps + 1) * n_links * kLinkStride));
    A(dalloc(s, &s->pose, 2 * (size_t)N)); A(dalloc(s, &s->vel, 2 * (size_t)N));
    A(dalloc(s, &s->params, N)); A(dalloc(s, &s->shape, N)); A(dalloc(s, &s->iters, N));
    A(dalloc(s, &s->status, N)); A(dalloc(s, &s->forces, (size_t)N * P * 3));
    A(dalloc(s, &s->order, N)); A(dalloc(s, &s->lpt_scratch, 64));
    A(dalloc(s, &s->c_sum, N)); A(dalloc(s, &s->c_mean, N));
    A(dalloc(s, &s->n_window, 1)); A(dalloc(s, &s->argmin, 1));
    A(dalloc(s, &s->part_c, std::max(N, cost_blocks(N)))); A(dalloc(s, &s->part_i, std::max(N, cost_blocks(N))));
    A(dalloc(s, &s->win, 1));
    A(dalloc(s, &s->done, 1)); A(dalloc(s, &s->work, 6)); A(dalloc(s, &s->adj_word, 1));
    A(dalloc(s, &s->queue, 2));
    A(dalloc(s, &s->is_elite, N)); A(dalloc(s, &s->rank, N)); A(dalloc(s, &s->elite_env, N));
    A(dalloc(s, &s->elite_w, N)); A(dalloc(s, &s->block_w, opt_blocks(N)));
    A(dalloc(s, &s->moments, (size_t)opt_blocks(N) * kMoments)); A(dalloc(s, &s->misc, 80));
    if (d.warm) { A(dalloc(s, &s->cache, (size_t)N * cfg->c_max)); A(dalloc(s, &s->cache_n, N)); }
    if (s->pd) {
        const size_t Dj = 4 * (size_t)sc->n_fingers;
        A(dalloc(s, &s->cmd, ((size_t)cfg->max_frames + 1) * Dj)); A(dalloc(s, &s->qj, (size_t)N * Dj));
        A(dalloc(s, &s->qdj, (size_t)N * Dj)); A(dalloc(s, &s->pad_pose, 2 * (size_t)N * P));
        A(dalloc(s, &s->slip, (size_t)N * P));
    }
    if (e != cudaSuccess) {
        ih_status st = cuda_fail(nullptr, e, "sim_create allocation");
        sim_destroy(s);
        return st;
    }
    std::vector<float4> sph(total);
    for (int j = 0; j < total; ++j)
        sph[j] = make_float4(sc->spheres[4 * j], sc->spheres[4 * j + 1], sc->spheres[4 * j + 2], sc->spheres[4 * j + 3]);
    std::vector<float4> roots(F > 0 ? F : 1, make_float4(0, 0, 0, 0));
    for (int f = 0; f < F; ++f)
        roots[f] = make_float4(sc->finger_root[4 * f], sc->finger_root[4 * f + 1], sc->finger_root[4 * f + 2],
                               sc->finger_root[4 * f + 3]);
    std::vector<int> shp0(N, 0), it0(N, cfg->iters);
    cudaStream_t st = s->stream;
    A(cudaMemcpyAsync(s->spheres_raw, sph.data(), total * sizeof(float4), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->shape_first, sc->shape_first, sc->n_shapes * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->shape_count, sc->shape_count, sc->n_shapes * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->cl_first, cl_first.data(), sc->n_shapes * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->finger_root, roots.data(), roots.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->pad_link, sc->pad_link, P * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->pad_s0, sc->pad_s0, P * sizeof(float), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->pad_s1, sc->pad_s1, P * sizeof(float), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->shape, shp0.data(), N * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(s->iters, it0.data(), N * sizeof(int), cudaMemcpyHostToDevice, st));
    s->iters_max_all = cfg->iters;
    A(cudaMemsetAsync(s->pose, 0, 2 * (size_t)N * sizeof(float4), st));
    A(cudaMemsetAsync(s->vel, 0, 2 * (size_t)N * sizeof(float4), st));
    A(cudaMemsetAsync(s->params, 0, (size_t)N * sizeof(float2), st));
    A(cudaMemsetAsync(s->status, 0, (size_t)N * sizeof(int), st));
    A(cudaMemsetAsync(s->forces, 0, (size_t)N * P * 3 * sizeof(float), st));
    A(cudaMemsetAsync(s->c_sum, 0, (size_t)N * sizeof(double), st));
    A(cudaMemsetAsync(s->c_mean, 0, (size_t)N * sizeof(double), st));
    A(cudaMemsetAsync(s->n_window, 0, sizeof(int), st));
    A(cudaMemsetAsync(s->argmin, 0, sizeof(int), st));
    A(cudaMemsetAsync(s->done, 0, sizeof(unsigned int), st));
    A(cudaMemsetAsync(s->queue, 0, 2 * sizeof(int), st));
    A(cudaMemsetAsync(s->work, 0, 6 * sizeof(unsigned long long), st));
    if (d.warm) A(cudaMemsetAsync(s->cache_n, 0, (size_t)N * sizeof(int), st));
    if (s->pd) {
        A(launch_hand_rest(N, 4 * sc->n_fingers, nullptr, s->qj, s->qdj, st));
        A(cudaMemsetAsync(s->pad_pose, 0, 2 * (size_t)N * P * sizeof(float4), st));
        A(cudaMemsetAsync(s->slip, 0, (size_t)N * P * sizeof(float4), st));
    }
    A(launch_shape_setup(s->spheres_raw, s->spheres, s->shape_first, s->shape_count, sc->n_shapes,
                         s->shape_jinv, s->shape_bound, s->cl_first, s->clusters, st));
    A(launch_lpt_order(N, s->shape_count, s->shape, s->iters, s->lpt_scratch, s->order, st));
    A(cudaStreamSynchronize(st));   // host vectors above go out of scope
    if (e != cudaSuccess) {
        ih_status r = cuda_fail(nullptr, e, "sim_create upload");
        sim_destroy(s);
        return r;
    }
    s->frame_ready.assign(cfg->max_frames, 0);
    {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        s->sms = sms > 0 ? sms : 1;
    }
    s->clp_cap = (1 + 4 * sc->n_fingers) * ((s->s_max + 7) / 8);
    if (e == cudaSuccess) e = use_variant(s, s->variant);
    if (e == cudaSuccess && s->pd) {
        e = pd_step_prepare(s->s_max, s->cfg.c_max);
        s->pd_grid = pd_step_grid(N, s->sms);
    }
    if (e != cudaSuccess) {
        ih_status r = cuda_fail(nullptr, e, "sim_create step setup");
        sim_destroy(s);
        return r;
    }
    *out = s;
    return IH_OK;
}

ih_status sim_destroy(ih_sim *s) {
    if (!s) return IH_OK;
    cudaStreamSynchronize(s->stream);
    if (s->win_exec) cudaGraphExecDestroy(s->win_exec);
    if (s->cap_stream) { cudaStreamSynchronize(s->cap_stream); cudaStreamDestroy(s->cap_stream); }
    if (s->cap_side) cudaStreamDestroy(s->cap_side);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    for (void *p : s->owned) cudaFree(p);
    if (s->adj_scratch) cudaFree(s->adj_scratch);
    if (s->spill) cudaFree(s->spill);
    if (s->wf_cm) cudaFree(s->wf_cm);
    if (s->wf_pose) cudaFree(s->wf_pose);
    for (void *q : {(void *)s->fo_q, (void *)s->fo_forces, (void *)s->fo_pp, (void *)s->fo_slip, (void *)s->fo_status,
                    (void *)s->fo_terms})
        if (q) cudaFree(q);
    delete s;
    return IH_OK;
}

ih_status sim_set_stream(ih_sim *s, void *stream) {
    if (!s) return IH_ERR_ARG;
    s->stream = static_cast<cudaStream_t>(stream);
    return IH_OK;
}

ih_status sim_set_commands(ih_sim *s, int32_t frame0, int32_t n_frames, const float *q) {
    if (!s) return IH_ERR_ARG;
    if ((!q && s->n_joints > 0) || n_frames < 1 || frame0 < 0 || frame0 + n_frames > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "frames [%d, %d) outside the table of %d", frame0, frame0 + n_frames,
                    s->cfg.max_frames);
    float4 *tab = s->link_tab + (size_t)frame0 * (s->cfg.substeps + 1) * s->n_links * kLinkStride;
    cudaError_t e = launch_fk(dev_scene(s), q, n_frames, s->cfg.substeps, tab, s->stream);
    if (e == cudaSuccess && s->pd && s->n_joints > 0)
        e = cudaMemcpyAsync(s->cmd + (size_t)frame0 * s->n_joints, q, ((size_t)n_frames + 1) * s->n_joints * sizeof(float),
                            cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "fk launch");
    for (int f = frame0; f < frame0 + n_frames; ++f) s->frame_ready[f] = 1;
    return IH_OK;
}

ih_status sim_sample_initial(ih_sim *s, const float *nominal, float sigma_p, float sigma_r, float m_lo,
                             float m_hi, float mu_lo, float mu_hi) {
    if (!s) return IH_ERR_ARG;
    if (!nominal || !(sigma_p >= 0.0f) || !(sigma_r >= 0.0f) || !(m_lo > 0.0f) || !(m_hi >= m_lo) ||
        !(mu_lo >= 0.0f) || !(mu_hi >= mu_lo))
        return fail(s, IH_ERR_ARG, "invalid sampling parameters");
    const float4 x0 = make_float4(nominal[0], nominal[1], nominal[2], 0.0f);
    const float4 q0 = make_float4(nominal[4], nominal[5], nominal[6], nominal[7]);
    cudaError_t e = launch_sample_initial(s->cfg.n_envs, x0, q0, sigma_p, sigma_r, m_lo, m_hi, mu_lo, mu_hi,
                                          s->seed, s->pose, s->vel, s->params, s->status, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->c_sum, 0, s->cfg.n_envs * sizeof(double), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->n_window, 0, sizeof(int), s->stream);
    if (e == cudaSuccess && s->cache_n) e = cudaMemsetAsync(s->cache_n, 0, s->cfg.n_envs * sizeof(int), s->stream);
    if (e == cudaSuccess && s->pd)
        e = launch_hand_rest(s->cfg.n_envs, s->n_joints, s->frame_ready[0] ? s->cmd : nullptr, s->qj, s->qdj, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "sample_initial");
    s->window_frames = 0;
    s->ws_valid = false;
    return IH_OK;
}

ih_status sim_set_state(ih_sim *s, const float *pose, const float *vel, const float *params,
                        const int32_t *shape_id, const int32_t *iters) {
    if (!s) return IH_ERR_ARG;
    if (!pose || !vel || !params) return fail(s, IH_ERR_ARG, "pose, vel and params are required");
    if (!aligned16(pose) || !aligned16(vel) || (reinterpret_cast<uintptr_t>(params) & 7u))
        return fail(s, IH_ERR_ARG, "pose/vel must be 16-byte aligned, params 8-byte aligned");
    cudaError_t e = launch_set_state(s->cfg.n_envs, s->n_shapes, pose, vel, params, shape_id, iters,
                                     s->pose, s->vel, s->params, s->shape, s->iters, s->status, s->stream);
    if (e == cudaSuccess && (shape_id || iters))
        e = launch_lpt_order(s->cfg.n_envs, s->shape_count, s->shape, s->iters, s->lpt_scratch, s->order, s->stream);
    if (e == cudaSuccess && s->cache_n) e = cudaMemsetAsync(s->cache_n, 0, s->cfg.n_envs * sizeof(int), s->stream);
    if (e == cudaSuccess && s->pd)
        e = launch_hand_rest(s->cfg.n_envs, s->n_joints, s->frame_ready[0] ? s->cmd : nullptr, s->qj, s->qdj, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "set_state");
    s->ws_valid = false;
    if (iters) s->iters_max_all = -1;
    return IH_OK;
}

ih_status sim_get_state(ih_sim *s, float *pose, float *vel, float *params, int32_t *env_status) {
    if (!s) return IH_ERR_ARG;
    const size_t N = s->cfg.n_envs;
    cudaError_t e = cudaSuccess;
    if (pose) e = cudaMemcpyAsync(pose, s->pose, N * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && vel)
        e = cudaMemcpyAsync(vel, s->vel, N * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && params)
        e = cudaMemcpyAsync(params, s->params, N * sizeof(float2), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && env_status)
        e = cudaMemcpyAsync(env_status, s->status, N * sizeof(int), cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "get_state");
    return IH_OK;
}

ih_status sim_get_warm_cache(ih_sim *s, int32_t *count, float *entries) {
    if (!s) return IH_ERR_ARG;
    if (!s->cache) return fail(s, IH_ERR_ARG, "the handle was created without warm_start");
    if (!count || !entries || !aligned16(entries)) return fail(s, IH_ERR_ARG, "count and 16-byte aligned entries are required");
    const size_t N = s->cfg.n_envs;
    cudaError_t e = cudaMemcpyAsync(count, s->cache_n, N * sizeof(int), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(entries, s->cache, N * s->cfg.c_max * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "get_warm_cache");
    return IH_OK;
}

ih_status sim_step(ih_sim *s, int32_t frame0, int32_t n_frames) {
    if (!s) return IH_ERR_ARG;
    if (n_frames < 1 || frame0 < 0 || frame0 + n_frames > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "frames [%d, %d) outside the table", frame0, frame0 + n_frames);
    for (int f = frame0; f < frame0 + n_frames; ++f)
        if (!s->frame_ready[f]) return fail(s, IH_ERR_ARG, "no commands for frame %d", f);
    if (s->pd) {
        PdArgs p;
        p.sc = dev_scene(s); p.cfg = s->dcfg; p.N = s->cfg.n_envs; p.cmd = s->cmd;
        p.frame0 = frame0; p.n_frames = n_frames; p.pose = s->pose; p.vel = s->vel; p.params = s->params;
        p.shape = s->shape; p.iters = s->iters; p.order = s->order; p.status = s->status;
        p.qj = s->qj; p.qdj = s->qdj; p.forces = s->forces; p.pad_pose = s->pad_pose; p.slip = s->slip;
        p.work = s->work;
        p.fo_q = nullptr; p.fo_pp = nullptr; p.fo_forces = nullptr; p.fo_slip = nullptr; p.fo_status = nullptr;
        p.pose_frames = nullptr;
        cudaError_t e = launch_pd_step(p, s->pd_grid, s->s_max, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "PD step launch");
        s->stepped = true;
        return IH_OK;
    }
    StepArgs a;
    a.sc = dev_scene(s); a.cfg = s->dcfg; a.N = s->cfg.n_envs; a.link_tab = s->link_tab;
    a.frame0 = frame0; a.n_frames = n_frames; a.pose = s->pose; a.vel = s->vel; a.params = s->params;
    a.shape = s->shape; a.iters = s->iters; a.status = s->status; a.forces = s->forces; a.work = s->work;
    a.order = s->order;
    a.obs = nullptr; a.win = nullptr; a.win_k = 0;
    a.c_sum = s->c_sum; a.c_mean = s->c_mean; a.n_window = s->n_window; a.cost_mean = nullptr;
    a.argmin_state = s->argmin; a.argmin_out = nullptr; a.est_pose_out = nullptr;
    a.part_c = s->part_c; a.part_i = s->part_i; a.done = s->done;
    a.cm_frames = nullptr; a.pose_frames = nullptr;
    a.cache = s->cache; a.cache_n = s->cache_n;
    a.stage_cap = s->stage_cap; a.spill = s->spill; a.clp_cap = s->clp_cap;
    // the work queue only when the grid's groups are fewer than the environments
    a.queue = (size_t)s->step_grid * (s->variant.block / s->variant.group) < (size_t)s->cfg.n_envs ? s->queue : nullptr;
    cudaError_t e = launch_step(a, s->variant, s->step_grid, s->s_max, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    s->stepped = true;
    return IH_OK;
}

namespace {
StepArgs scored_args(ih_sim *s, int frame, const float *obs, double *cost_mean, int32_t *argmin, float *est) {
    StepArgs a;
    a.sc = dev_scene(s); a.cfg = s->dcfg; a.N = s->cfg.n_envs; a.link_tab = s->link_tab;
    a.frame0 = frame; a.n_frames = 1; a.pose = s->pose; a.vel = s->vel; a.params = s->params;
    a.shape = s->shape; a.iters = s->iters; a.status = s->status; a.forces = s->forces; a.work = s->work;
    a.order = s->order;
    a.obs = obs; a.win = nullptr; a.win_k = 0;
    a.c_sum = s->c_sum; a.c_mean = s->c_mean; a.n_window = s->n_window; a.cost_mean = cost_mean;
    a.argmin_state = s->argmin; a.argmin_out = argmin; a.est_pose_out = est;
    a.part_c = s->part_c; a.part_i = s->part_i; a.done = s->done;
    a.cm_frames = nullptr; a.pose_frames = nullptr;
    a.cache = s->cache; a.cache_n = s->cache_n;
    a.stage_cap = s->stage_cap; a.spill = s->spill; a.clp_cap = s->clp_cap;
    // the work queue only when the grid's groups are fewer than the environments
    a.queue = (size_t)s->step_grid * (s->variant.block / s->variant.group) < (size_t)s->cfg.n_envs ? s->queue : nullptr;
    return a;
}

OptArgs opt_args(ih_sim *s, const ih_opt_config *opt, uint32_t update_index, int32_t *argmin, int32_t *parent) {
    OptArgs a;
    a.N = s->cfg.n_envs; a.elite_frac = opt->elite_frac;
    for (int k = 0; k < 8; ++k) a.floor_var[k] = (double)opt->floor_std[k] * (double)opt->floor_std[k];
    a.m_lo = opt->m_lo; a.m_hi = opt->m_hi; a.mu_lo = opt->mu_lo; a.mu_hi = opt->mu_hi;
    a.seed = s->seed; a.update_index = update_index; a.c_mean = s->c_mean; a.c_sum = s->c_sum;
    a.n_window = s->n_window; a.pose = s->pose; a.vel = s->vel; a.params = s->params;
    a.status = s->status; a.is_elite = s->is_elite; a.rank = s->rank; a.elite_env = s->elite_env;
    a.elite_w = s->elite_w; a.block_w = s->block_w; a.moments = s->moments; a.misc = s->misc;
    a.argmin_state = s->argmin; a.argmin_out = argmin; a.parent_out = parent; a.win = nullptr;
    a.kind = opt->kind; a.wrs_lambda = opt->wrs_lambda; a.reps_epsilon = opt->reps_epsilon;
    for (int k = 0; k < 6; ++k) { a.sigma_pose[k] = opt->sigma_pose[k]; a.sigma_vel[k] = opt->sigma_vel[k]; }
    a.sigma_theta[0] = opt->sigma_theta[0]; a.sigma_theta[1] = opt->sigma_theta[1];
    a.explore_velocity = opt->explore_velocity;
    a.sn_pose = s->sn_pose; a.sn_vel = s->sn_vel; a.sn_params = s->sn_params; a.sn_status = s->sn_status;
    a.cache_n = s->cache_n;
    a.qj = s->qj; a.qdj = s->qdj; a.D = s->n_joints; a.sn_qj = s->sn_qj; a.sn_qdj = s->sn_qdj;
    return a;
}

ih_status check_opt(ih_sim *s, const ih_opt_config *opt) {
    if (!opt || !(opt->elite_frac > 0.0f) || !(opt->elite_frac <= 1.0f) || !(opt->m_lo > 0.0f) ||
        !(opt->m_hi >= opt->m_lo) || !(opt->mu_lo >= 0.0f) || !(opt->mu_hi >= opt->mu_lo))
        return fail(s, IH_ERR_ARG, "invalid optimizer config");
    for (int k = 0; k < 8; ++k)
        if (!(opt->floor_std[k] >= 0.0f) || !std::isfinite(opt->floor_std[k]))
            return fail(s, IH_ERR_ARG, "floor_std[%d] is invalid", k);
    if (opt->kind < IH_OPT_ELITE || opt->kind > IH_OPT_REPS) return fail(s, IH_ERR_ARG, "unknown optimizer kind");
    if (opt->kind != IH_OPT_ELITE) {
        if (opt->kind == IH_OPT_WRS && !(opt->wrs_lambda > 0.0f && std::isfinite(opt->wrs_lambda)))
            return fail(s, IH_ERR_ARG, "wrs_lambda must be positive");
        if (opt->kind == IH_OPT_REPS && !(opt->reps_epsilon > 0.0f && std::isfinite(opt->reps_epsilon)))
            return fail(s, IH_ERR_ARG, "reps_epsilon must be positive");
        for (int k = 0; k < 6; ++k)
            if (!(opt->sigma_pose[k] >= 0.0f) || !std::isfinite(opt->sigma_pose[k]) || !(opt->sigma_vel[k] >= 0.0f) ||
                !std::isfinite(opt->sigma_vel[k]))
                return fail(s, IH_ERR_ARG, "exploration sigma %d is invalid", k);
        if (!(opt->sigma_theta[0] >= 0.0f) || !(opt->sigma_theta[1] >= 0.0f) || !std::isfinite(opt->sigma_theta[0]) ||
            !std::isfinite(opt->sigma_theta[1]))
            return fail(s, IH_ERR_ARG, "sigma_theta is invalid");
        // the state before the update, for draws with replacement (allocated once, outside any capture)
        if (!s->sn_pose) {
            const size_t N = s->cfg.n_envs;
            cudaError_t e = cudaSuccess;
            auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
            A(dalloc(s, &s->sn_pose, 2 * N)); A(dalloc(s, &s->sn_vel, 2 * N));
            A(dalloc(s, &s->sn_params, N)); A(dalloc(s, &s->sn_status, N));
            if (s->pd) { A(dalloc(s, &s->sn_qj, N * s->n_joints)); A(dalloc(s, &s->sn_qdj, N * s->n_joints)); }
            if (e != cudaSuccess) return cuda_fail(s, e, "optimizer snapshot");
        }
    }
    return IH_OK;
}
}  // namespace

ih_status sim_step_track(ih_sim *s, int32_t frame, const float *obs, double *cost_mean, int32_t *argmin,
                         float *est_pose) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_step_track");
    if (ih_status rp = check_no_pending(s)) return rp;
    if (!obs) return fail(s, IH_ERR_ARG, "obs is required");
    if (frame < 0 || frame >= s->cfg.max_frames || !s->frame_ready[frame])
        return fail(s, IH_ERR_ARG, "no commands for frame %d", frame);
    StepArgs a = scored_args(s, frame, obs, cost_mean, argmin, est_pose);
    cudaError_t e = launch_step(a, s->variant, s->step_grid, s->s_max, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    s->stepped = true;
    s->window_frames += 1;
    return IH_OK;
}

namespace {
// per-frame window means and poses of a window-mode launch, grown to T frames
cudaError_t window_buffers(ih_sim *s, int T) {
    if (T <= s->wf_T) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (s->cap_stream && e == cudaSuccess) e = cudaStreamSynchronize(s->cap_stream);
    if (e != cudaSuccess) return e;
    if (s->wf_cm) cudaFree(s->wf_cm);
    if (s->wf_pose) cudaFree(s->wf_pose);
    s->wf_cm = nullptr; s->wf_pose = nullptr; s->wf_T = 0;
    void *p1 = nullptr, *p2 = nullptr;
    e = cudaMalloc(&p1, (size_t)T * s->cfg.n_envs * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p2, (size_t)T * s->cfg.n_envs * 2 * sizeof(float4));
    if (e != cudaSuccess) { if (p1) cudaFree(p1); return e; }
    s->wf_cm = static_cast<double *>(p1);
    s->wf_pose = static_cast<float4 *>(p2);
    s->wf_T = T;
    return cudaSuccess;
}

// the PD window's per-frame observation, status and cost-term buffers, grown to T frames
cudaError_t pd_frame_buffers(ih_sim *s, int T) {
    if (T <= s->fo_T) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return e;
    void **bufs[6] = {(void **)&s->fo_q, (void **)&s->fo_forces, (void **)&s->fo_pp, (void **)&s->fo_slip,
                      (void **)&s->fo_status, (void **)&s->fo_terms};
    for (void **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    s->fo_T = 0;
    const size_t ef = (size_t)T * s->cfg.n_envs, P = (size_t)s->n_pads, D = (size_t)s->n_joints;
    const size_t bytes[6] = {ef * D * sizeof(float), ef * P * 3 * sizeof(float), ef * P * 2 * sizeof(float4),
                             ef * P * sizeof(float4), ef * sizeof(int), ef * (P + 1) * sizeof(double)};
    for (int k = 0; k < 6; ++k) {
        e = cudaMalloc(bufs[k], bytes[k] > 0 ? bytes[k] : 16);
        if (e != cudaSuccess) return e;   // what was allocated is freed with the handle
    }
    s->fo_T = T;
    return cudaSuccess;
}
}  // namespace

ih_status sim_step_frames(ih_sim *s, int32_t frame0, int32_t T, const float *obs) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_step_frames");
    if (ih_status rp = check_no_pending(s)) return rp;
    if (!obs) return fail(s, IH_ERR_ARG, "obs is required");
    if (T < 1 || frame0 < 0 || frame0 + T > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "frames [%d, %d) outside the table", frame0, frame0 + T);
    for (int f = frame0; f < frame0 + T; ++f)
        if (!s->frame_ready[f]) return fail(s, IH_ERR_ARG, "no commands for frame %d", f);
    cudaError_t e = window_buffers(s, T);
    if (e != cudaSuccess) return cuda_fail(s, e, "window buffers");
    StepArgs a = scored_args(s, frame0, obs, nullptr, nullptr, nullptr);
    a.n_frames = T;
    a.cm_frames = s->wf_cm;
    a.pose_frames = s->wf_pose;
    e = launch_step(a, s->variant, s->step_grid, s->s_max, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    s->stepped = true;
    s->frames_T = T;
    return IH_OK;
}

ih_status sim_step_frames_full(ih_sim *s, int32_t frame0, int32_t T, const float *q, const float *pad_pose,
                               const float *forces, const float *slip) {
    if (!s) return IH_ERR_ARG;
    if (!s->pd) return fail(s, IH_ERR_ARG, "sim_step_frames_full needs the PD-driven hand");
    if (ih_status rp = check_no_pending(s)) return rp;
    if ((!q && s->n_joints > 0) || !pad_pose || !forces || !slip)
        return fail(s, IH_ERR_ARG, "the ground truth's q, pad_pose, forces and slip are required");
    if (!aligned16(pad_pose) || !aligned16(slip)) return fail(s, IH_ERR_ARG, "pad_pose and slip must be 16-byte aligned");
    if (T < 1 || frame0 < 0 || frame0 + T > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "frames [%d, %d) outside the table", frame0, frame0 + T);
    for (int f = frame0; f < frame0 + T; ++f)
        if (!s->frame_ready[f]) return fail(s, IH_ERR_ARG, "no commands for frame %d", f);
    cudaError_t e = window_buffers(s, T);
    if (e == cudaSuccess) e = pd_frame_buffers(s, T);
    if (e != cudaSuccess) return cuda_fail(s, e, "window buffers");
    PdArgs p;
    p.sc = dev_scene(s); p.cfg = s->dcfg; p.N = s->cfg.n_envs; p.cmd = s->cmd;
    p.frame0 = frame0; p.n_frames = T; p.pose = s->pose; p.vel = s->vel; p.params = s->params;
    p.shape = s->shape; p.iters = s->iters; p.order = s->order; p.status = s->status;
    p.qj = s->qj; p.qdj = s->qdj; p.forces = s->forces; p.pad_pose = s->pad_pose; p.slip = s->slip;
    p.work = s->work;
    p.fo_q = s->fo_q; p.fo_pp = s->fo_pp; p.fo_forces = s->fo_forces; p.fo_slip = s->fo_slip;
    p.fo_status = s->fo_status; p.pose_frames = s->wf_pose;
    e = launch_pd_step(p, s->pd_grid, s->s_max, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "PD step launch");
    FramesCostArgs c;
    c.N = s->cfg.n_envs; c.P = s->n_pads; c.D = s->n_joints; c.T = T; c.cfg = s->dcfg;
    c.fo_q = s->fo_q; c.fo_pp = s->fo_pp; c.fo_forces = s->fo_forces; c.fo_slip = s->fo_slip;
    c.fo_status = s->fo_status;
    c.g_q = q; c.g_pose = reinterpret_cast<const float4 *>(pad_pose); c.g_forces = forces;
    c.g_slip = reinterpret_cast<const float4 *>(slip);
    c.terms = s->fo_terms; c.c_sum = s->c_sum; c.c_mean = s->c_mean; c.n_window = s->n_window;
    c.cm_frames = s->wf_cm;
    e = launch_frames_cost_full(c, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "frames cost launch");
    s->stepped = true;
    s->frames_T = T;
    return IH_OK;
}

ih_status sim_frames_argmin(ih_sim *s, float *est_pose, int32_t *argmin) {
    if (!s) return IH_ERR_ARG;
    if (s->frames_T < 1) return fail(s, IH_ERR_STATE, "no sim_step_frames call to score");
    cudaError_t e = launch_window_argmin(s->cfg.n_envs, s->frames_T, s->wf_cm, s->wf_pose, nullptr, argmin, est_pose,
                                         s->argmin, s->n_window, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "argmin launch");
    s->window_frames += s->frames_T;
    s->frames_T = 0;
    return IH_OK;
}

ih_status sim_track_window(ih_sim *s, int32_t frame0, int32_t T, const float *obs, const ih_opt_config *opt,
                           uint32_t update_index, float *est_pose, int32_t *argmin) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_track_window");
    if (ih_status rp = check_no_pending(s)) return rp;
    if (!obs) return fail(s, IH_ERR_ARG, "obs is required");
    if (T < 1 || frame0 < 0 || frame0 + T > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "window [%d, %d) outside the table", frame0, frame0 + T);
    for (int f = frame0; f < frame0 + T; ++f)
        if (!s->frame_ready[f]) return fail(s, IH_ERR_ARG, "no commands for frame %d", f);
    ih_status r = check_opt(s, opt);
    if (r != IH_OK) return r;
    cudaError_t e = cudaSuccess;
    if (!s->cap_stream) {
        e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(s, e, "window stream");
    }
    // the caller's stream -> private stream -> back, so ordering follows the caller's stream
    WinDesc v{frame0, update_index, obs, est_pose, argmin};
    e = launch_win_desc(s->win, v, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_in, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cap_stream, s->ev_in, 0);
    if (e != cudaSuccess) return cuda_fail(s, e, "window descriptor");
    cudaStream_t st = s->cap_stream;
    const bool same = s->win_exec && s->win_T == T && s->win_variant.group == s->variant.group &&
                      s->win_variant.cpl == s->variant.cpl && std::memcmp(&s->win_opt, opt, sizeof *opt) == 0;
    if (!same) {
        if (s->win_exec) { cudaGraphExecDestroy(s->win_exec); s->win_exec = nullptr; }
        e = window_buffers(s, T);   // outside the capture
        if (e != cudaSuccess) return cuda_fail(s, e, "window buffers");
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(s, e, "begin capture");
        cudaError_t le = cudaSuccess;
        {   // the window's T frames in one launch
            StepArgs a = scored_args(s, frame0, nullptr, nullptr, nullptr, nullptr);
            a.win = s->win;
            a.win_k = 0;
            a.n_frames = T;
            a.cm_frames = s->wf_cm;
            a.pose_frames = s->wf_pose;
            le = launch_step(a, s->variant, s->step_grid, s->s_max, st);
        }
        // then two branches: every frame's argmin and estimate (from the frame
        // buffers, which nothing else writes) beside the optimizer update; the
        // update sets the handle's i* and restarts the window count, so the
        // argmin branch leaves both alone
        if (le == cudaSuccess) le = cudaEventRecord(s->ev_fork, st);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(s->cap_side, s->ev_fork, 0);
        if (le == cudaSuccess)
            le = launch_window_argmin(s->cfg.n_envs, T, s->wf_cm, s->wf_pose, s->win, nullptr, nullptr, nullptr,
                                      nullptr, s->cap_side);
        if (le == cudaSuccess) {
            OptArgs oa = opt_args(s, opt, update_index, nullptr, nullptr);
            oa.win = s->win;
            le = launch_optimizer(oa, st);
        }
        if (le == cudaSuccess) le = cudaEventRecord(s->ev_join, s->cap_side);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(st, s->ev_join, 0);
        e = cudaStreamEndCapture(st, &g);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(s, le != cudaSuccess ? le : e, "window capture");
        }
        e = cudaGraphInstantiate(&s->win_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { s->win_exec = nullptr; return cuda_fail(s, e, "window instantiate"); }
        s->win_T = T;
        s->win_variant = s->variant;
        s->win_opt = *opt;
    }
    e = cudaGraphLaunch(s->win_exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_out, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_out, 0);
    if (e != cudaSuccess) return cuda_fail(s, e, "window launch");
    s->stepped = true;
    s->window_frames = 0;
    s->ws_valid = false;
    return IH_OK;
}

ih_status sim_read_sensors(ih_sim *s, float *forces, int32_t *env_status) {
    if (!s) return IH_ERR_ARG;
    const size_t N = s->cfg.n_envs;
    cudaError_t e = cudaSuccess;
    if (forces)
        e = cudaMemcpyAsync(forces, s->forces, N * s->n_pads * 3 * sizeof(float), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && env_status)
        e = cudaMemcpyAsync(env_status, s->status, N * sizeof(int), cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "read_sensors");
    return IH_OK;
}

ih_status cost_eval(ih_sim *s, const float *obs, double *cost_mean, int32_t *argmin, float *est_pose) {
    if (!s) return IH_ERR_ARG;
    if (ih_status rp = check_no_pending(s)) return rp;
    if (!obs) return fail(s, IH_ERR_ARG, "obs is required");
    CostArgs a;
    a.N = s->cfg.n_envs; a.P = s->n_pads; a.cfg = s->dcfg; a.forces = s->forces; a.obs = obs;
    a.status = s->status; a.c_sum = s->c_sum; a.c_mean = s->c_mean; a.n_window = s->n_window;
    a.cost_mean = cost_mean;
    a.pose = s->pose; a.argmin_state = s->argmin; a.argmin_out = argmin; a.est_pose_out = est_pose;
    a.part_c = s->part_c; a.part_i = s->part_i; a.done = s->done;
    a.qj = nullptr; a.pad_pose = nullptr; a.slip = nullptr; a.g_q = nullptr; a.g_pose = nullptr; a.g_slip = nullptr;
    a.D = 0;
    cudaError_t e = launch_cost(a, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "cost launch");
    s->window_frames += 1;
    return IH_OK;
}

ih_status cost_eval_full(ih_sim *s, const float *q, const float *pad_pose, const float *forces, const float *slip,
                         double *cost_mean, int32_t *argmin, float *est_pose) {
    if (!s) return IH_ERR_ARG;
    if (!s->pd) return fail(s, IH_ERR_ARG, "cost_eval_full needs the PD-driven hand");
    if (ih_status rp = check_no_pending(s)) return rp;
    if ((!q && s->n_joints > 0) || !pad_pose || !forces || !slip)
        return fail(s, IH_ERR_ARG, "the ground truth's q, pad_pose, forces and slip are required");
    if (!aligned16(pad_pose) || !aligned16(slip)) return fail(s, IH_ERR_ARG, "pad_pose and slip must be 16-byte aligned");
    CostArgs a;
    a.N = s->cfg.n_envs; a.P = s->n_pads; a.cfg = s->dcfg; a.forces = s->forces; a.obs = forces;
    a.status = s->status; a.c_sum = s->c_sum; a.c_mean = s->c_mean; a.n_window = s->n_window;
    a.cost_mean = cost_mean;
    a.pose = s->pose; a.argmin_state = s->argmin; a.argmin_out = argmin; a.est_pose_out = est_pose;
    a.part_c = s->part_c; a.part_i = s->part_i; a.done = s->done;
    a.qj = s->qj; a.pad_pose = s->pad_pose; a.slip = s->slip; a.D = s->n_joints;
    a.g_q = q; a.g_pose = reinterpret_cast<const float4 *>(pad_pose); a.g_slip = reinterpret_cast<const float4 *>(slip);
    cudaError_t e = launch_cost(a, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "cost launch");
    s->window_frames += 1;
    return IH_OK;
}

ih_status sim_read_observation(ih_sim *s, float *q, float *pad_pose, float *slip) {
    if (!s) return IH_ERR_ARG;
    if (!s->pd) return fail(s, IH_ERR_ARG, "the full observation needs the PD-driven hand");
    if ((pad_pose && !aligned16(pad_pose)) || (slip && !aligned16(slip)))
        return fail(s, IH_ERR_ARG, "pad_pose and slip must be 16-byte aligned");
    const size_t N = s->cfg.n_envs, P = s->n_pads, D = s->n_joints;
    cudaError_t e = cudaSuccess;
    if (q && D > 0) e = cudaMemcpyAsync(q, s->qj, N * D * sizeof(float), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && pad_pose)
        e = cudaMemcpyAsync(pad_pose, s->pad_pose, 2 * N * P * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && slip)
        e = cudaMemcpyAsync(slip, s->slip, N * P * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "read_observation");
    return IH_OK;
}

ih_status sim_set_hand(ih_sim *s, const float *q, const float *qd) {
    if (!s) return IH_ERR_ARG;
    if (!s->pd) return fail(s, IH_ERR_ARG, "the hand's joints are state only with the PD-driven hand");
    const size_t bytes = (size_t)s->cfg.n_envs * s->n_joints * sizeof(float);
    if (bytes == 0) return IH_OK;
    if (!q) return fail(s, IH_ERR_ARG, "q is required");
    cudaError_t e = cudaMemcpyAsync(s->qj, q, bytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess)
        e = qd ? cudaMemcpyAsync(s->qdj, qd, bytes, cudaMemcpyDeviceToDevice, s->stream)
               : cudaMemsetAsync(s->qdj, 0, bytes, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "set_hand");
    return IH_OK;
}

ih_status sim_get_hand(ih_sim *s, float *q, float *qd) {
    if (!s) return IH_ERR_ARG;
    if (!s->pd) return fail(s, IH_ERR_ARG, "the hand's joints are state only with the PD-driven hand");
    const size_t bytes = (size_t)s->cfg.n_envs * s->n_joints * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (q && bytes) e = cudaMemcpyAsync(q, s->qj, bytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && qd && bytes) e = cudaMemcpyAsync(qd, s->qdj, bytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "get_hand");
    return IH_OK;
}

ih_status optimizer_update(ih_sim *s, const ih_opt_config *opt, uint32_t update_index, int32_t *argmin,
                           int32_t *parent) {
    if (!s) return IH_ERR_ARG;
    if (ih_status rp = check_no_pending(s)) return rp;
    ih_status r = check_opt(s, opt);
    if (r != IH_OK) return r;
    if (s->window_frames < 1) return fail(s, IH_ERR_STATE, "no frame scored since the last update");
    OptArgs a = opt_args(s, opt, update_index, argmin, parent);
    cudaError_t e = launch_optimizer(a, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "optimizer launch");
    s->window_frames = 0;
    s->ws_valid = false;
    return IH_OK;
}

ih_status sim_work_counters(ih_sim *s, uint64_t *out, int32_t reset) {
    if (!s || !out) return IH_ERR_ARG;
    unsigned long long w[6];
    cudaError_t e = cudaMemcpyAsync(w, s->work, sizeof w, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(s->work, 0, sizeof w, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "work counters");
    for (int k = 0; k < 6; ++k) out[k] = w[k];
    return IH_OK;
}

ih_status sim_set_variant(ih_sim *s, int32_t tpe, int32_t cpl) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_set_variant");
    StepVariant v{tpe, cpl, 128};
    if (!step_variant_supported(v)) return fail(s, IH_ERR_ARG, "unsupported step shape %d x %d", tpe, cpl);
    if (step_variant_max_contacts(v) < s->cfg.c_max)
        return fail(s, IH_ERR_ARG, "shape %d x %d holds fewer than c_max = %d contacts", tpe, cpl, s->cfg.c_max);
    cudaError_t e = use_variant(s, v);
    if (e != cudaSuccess) return cuda_fail(s, e, "set_variant");
    return IH_OK;
}

int32_t sim_step_variants(int32_t *out, int32_t cap) {
    StepVariant v[32];
    const int n = step_variant_list(v, 32);
    for (int k = 0; k < n && k < cap && out; ++k) { out[2 * k] = v[k].group; out[2 * k + 1] = v[k].cpl; }
    return n;
}

ih_status sim_autotune(ih_sim *s, int32_t frame0, int32_t n_frames, int32_t *chosen, float *ms_out) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_autotune");
    if (n_frames < 1 || frame0 < 0 || frame0 + n_frames > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "frames [%d, %d) outside the table", frame0, frame0 + n_frames);
    for (int f = frame0; f < frame0 + n_frames; ++f)
        if (!s->frame_ready[f]) return fail(s, IH_ERR_ARG, "no commands for frame %d", f);
    const size_t N = s->cfg.n_envs, P = s->n_pads;
    // scratch copy of everything a step writes
    void *bp = nullptr, *bv = nullptr, *bs = nullptr, *bf = nullptr, *bc = nullptr, *bn = nullptr;
    unsigned long long wsave[6];
    const size_t cache_bytes = s->cache ? N * s->cfg.c_max * sizeof(float4) : 0;
    cudaError_t e = cudaMalloc(&bp, N * 2 * sizeof(float4));
    if (e == cudaSuccess && s->cache) e = cudaMalloc(&bc, cache_bytes);
    if (e == cudaSuccess && s->cache) e = cudaMalloc(&bn, N * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&bv, N * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&bs, N * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&bf, N * P * 3 * sizeof(float));
    cudaStream_t st = s->stream;
    auto save = [&]() {
        cudaMemcpyAsync(bp, s->pose, N * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(bv, s->vel, N * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(bs, s->status, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(bf, s->forces, N * P * 3 * sizeof(float), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(wsave, s->work, sizeof wsave, cudaMemcpyDeviceToHost, st);
        if (bc) {
            cudaMemcpyAsync(bc, s->cache, cache_bytes, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(bn, s->cache_n, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
        }
    };
    auto restore = [&]() {
        cudaMemcpyAsync(s->pose, bp, N * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s->vel, bv, N * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s->status, bs, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s->forces, bf, N * P * 3 * sizeof(float), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s->work, wsave, sizeof wsave, cudaMemcpyHostToDevice, st);
        if (bc) {
            cudaMemcpyAsync(s->cache, bc, cache_bytes, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(s->cache_n, bn, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
        }
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    StepVariant cand[32];
    const int nv = step_variant_list(cand, 32);
    const StepVariant keep = s->variant;
    StepVariant best = keep;
    float best_ms = INFINITY;
    if (e == cudaSuccess) { save(); e = cudaStreamSynchronize(st); }
    for (int k = 0; k < nv && e == cudaSuccess; ++k) {
        float ms = NAN;
        if (step_variant_max_contacts(cand[k]) >= s->cfg.c_max && use_variant(s, cand[k]) == cudaSuccess) {
            ih_status r = sim_step(s, frame0, n_frames);   // warm-up (and first-use setup)
            restore();
            for (int rep = 0; rep < 3 && r == IH_OK && e == cudaSuccess; ++rep) {
                float t = NAN;
                cudaEventRecord(e0, st);
                r = sim_step(s, frame0, n_frames);
                cudaEventRecord(e1, st);
                restore();
                e = cudaStreamSynchronize(st);
                if (e == cudaSuccess && r == IH_OK) cudaEventElapsedTime(&t, e0, e1);
                if (!(ms <= t)) ms = t;   // best of three
            }
            if (r != IH_OK && e == cudaSuccess) e = cudaErrorLaunchFailure;
            if (ms < best_ms) { best_ms = ms; best = cand[k]; }
        }
        if (ms_out && k < 16) ms_out[k] = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(bp); cudaFree(bv); cudaFree(bs); cudaFree(bf);
    if (bc) cudaFree(bc);
    if (bn) cudaFree(bn);
    if (e != cudaSuccess) {
        use_variant(s, keep);
        return cuda_fail(s, e, "autotune");
    }
    e = use_variant(s, best);
    if (e != cudaSuccess) return cuda_fail(s, e, "autotune");
    if (chosen) { chosen[0] = best.group; chosen[1] = best.cpl; }
    return IH_OK;
}

namespace {
// Size (and grow) the adjoint scratch for n slots: reads back the largest
// iteration count among the selected environments (synchronises the stream).
ih_status adjoint_prepare(ih_sim *s, int n, const int32_t *envs, int horizon, int K, size_t *stride, int *imax) {
    (void)envs;
    cudaStream_t st = s->stream;
    cudaError_t e = cudaSuccess;
    // the tape holds the iterations of the largest count of any environment
    // (it bounds every selection's); read back only after sim_set_state set
    // new counts, so that the calls in between need no synchronisation
    if (s->iters_max_all < 0) {
        int m = 0;
        e = launch_adjoint_iters_max(s->cfg.n_envs, s->cfg.n_envs, nullptr, s->iters, s->adj_word, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&m, s->adj_word, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(s, e, "adjoint sizing");
        s->iters_max_all = m;
    }
    const int m = s->iters_max_all;
    // tape whole segments when that fits the handle's budget, else substep by substep
    size_t str = adjoint_scratch_floats(horizon, K, s->cfg.substeps, s->n_pads, s->cfg.c_max, m, true);
    bool seg = str * (size_t)n * sizeof(float) <= s->adj_budget;
    if (!seg) str = adjoint_scratch_floats(horizon, K, s->cfg.substeps, s->n_pads, s->cfg.c_max, m, false);
    const size_t need = str * (size_t)n;
    if (need > s->adj_floats) {
        e = cudaStreamSynchronize(st);   // the old scratch may still be in use
        if (e != cudaSuccess) return cuda_fail(s, e, "adjoint sizing");
        if (s->adj_scratch) cudaFree(s->adj_scratch);
        s->adj_scratch = nullptr;
        s->adj_floats = 0;
        void *p = nullptr;
        e = cudaMalloc(&p, need * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(s, e, "adjoint scratch");
        s->adj_scratch = static_cast<float *>(p);
        s->adj_floats = need;
    }
    *stride = str;
    *imax = m;
    s->adj_seg = seg;
    return IH_OK;
}

ih_status check_horizon(ih_sim *s, int32_t frame0, int32_t horizon) {
    if (horizon < 1 || frame0 < 0 || frame0 + horizon > s->cfg.max_frames)
        return fail(s, IH_ERR_ARG, "horizon [%d, %d) outside the table", frame0, frame0 + horizon);
    for (int f = frame0; f < frame0 + horizon; ++f)
        if (!s->frame_ready[f]) return fail(s, IH_ERR_ARG, "no commands for frame %d", f);
    return IH_OK;
}

AdjArgs adjoint_args(ih_sim *s, int32_t frame0, int32_t horizon, int K, const float *obs, float beta, float width) {
    AdjArgs a;
    a.sc = dev_scene(s); a.cfg = s->dcfg; a.N = s->cfg.n_envs; a.n = 0; a.envs = nullptr;
    a.link_tab = s->link_tab; a.frame0 = frame0; a.H = horizon; a.K = K;
    a.pose = s->pose; a.vel = s->vel; a.params = s->params; a.shape = s->shape; a.iters = s->iters;
    a.status = s->status; a.obs = obs; a.beta_s = beta; a.width = width;
    a.cost = nullptr; a.grad = nullptr; a.grad_quat = nullptr;
    a.scratch = s->adj_scratch; a.stride = 0; a.iters_max = 0;
    a.forward_only = 0; a.out_pose = nullptr; a.out_vel = nullptr; a.seg_tape = 0; a.zero = 0;
    a.gw = s->adj_gw; a.pl = s->adj_pl; a.s_max = s->s_max;
    a.refine = 0;
    a.rf = RefineArgs{};
    return a;
}
}  // namespace

ih_status sim_adjoint(ih_sim *s, int32_t frame0, int32_t horizon, int32_t checkpoint_every, const float *obs,
                      const int32_t *envs, int32_t n, float beta, float width, double *cost, float *grad,
                      float *grad_quat) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_adjoint");
    if (s->dcfg.warm) return fail(s, IH_ERR_ARG, "the adjoint differentiates the cold-started solver only");
    if (!obs || !grad) return fail(s, IH_ERR_ARG, "obs and grad are required");
    ih_status r = check_horizon(s, frame0, horizon);
    if (r != IH_OK) return r;
    if (checkpoint_every < 1) return fail(s, IH_ERR_ARG, "checkpoint_every must be >= 1");
    if (n < 1 || n > s->cfg.n_envs) return fail(s, IH_ERR_ARG, "n must be in [1, %d]", s->cfg.n_envs);
    if (!(beta > 0.0f) || !std::isfinite(beta) || !(width > 0.0f) || !std::isfinite(width))
        return fail(s, IH_ERR_ARG, "beta and width must be positive");
    const int K = std::min(checkpoint_every, horizon);
    size_t stride = 0;
    int imax = 0;
    r = adjoint_prepare(s, n, envs, horizon, K, &stride, &imax);
    if (r != IH_OK) return r;
    AdjArgs a = adjoint_args(s, frame0, horizon, K, obs, beta, width);
    a.n = n; a.envs = envs; a.cost = cost; a.grad = grad; a.grad_quat = grad_quat;
    a.scratch = s->adj_scratch; a.stride = stride; a.iters_max = imax; a.seg_tape = s->adj_seg ? 1 : 0;
    cudaError_t e = launch_adjoint(a, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "adjoint launch");
    return IH_OK;
}

namespace {
cudaError_t refine_alloc(ih_sim *s) {
    if (s->rf_alloc) return cudaSuccess;
    const size_t N = s->cfg.n_envs;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(s, &s->ws_pose, 2 * N)); A(dalloc(s, &s->ws_vel, 2 * N)); A(dalloc(s, &s->ws_params, N));
    A(dalloc(s, &s->tr_pose, 2 * N)); A(dalloc(s, &s->tr_params, N));
    A(dalloc(s, &s->end_pose, 2 * N)); A(dalloc(s, &s->end_vel, 2 * N));
    A(dalloc(s, &s->best_end_pose, 2 * N)); A(dalloc(s, &s->best_end_vel, 2 * N));
    A(dalloc(s, &s->best_pose, 2 * N)); A(dalloc(s, &s->best_params, N)); A(dalloc(s, &s->best_grad, 8 * N));
    A(dalloc(s, &s->scale, N)); A(dalloc(s, &s->r_grad, 8 * N));
    A(dalloc(s, &s->best_c, N)); A(dalloc(s, &s->c0, N)); A(dalloc(s, &s->r_cost, N));
    A(dalloc(s, &s->r_acc, N));
    if (e == cudaSuccess) s->rf_alloc = true;
    return e;
}
}  // namespace

ih_status sim_set_adjoint_memory(ih_sim *s, uint64_t bytes) {
    if (!s) return IH_ERR_ARG;
    s->adj_budget = (size_t)bytes;
    return IH_OK;
}

ih_status sim_set_adjoint_variant(ih_sim *s, int32_t gw, int32_t pl) {
    if (!s) return IH_ERR_ARG;
    if (!adjoint_variant_supported(gw, pl))
        return fail(s, IH_ERR_ARG, "unsupported adjoint shape %d warps x %d contacts", gw, pl);
    s->adj_gw = gw;
    s->adj_pl = pl;
    return IH_OK;
}

ih_status sim_mark_window(ih_sim *s) {
    if (!s) return IH_ERR_ARG;
    cudaError_t e = refine_alloc(s);
    const size_t N = s->cfg.n_envs;
    cudaStream_t st = s->stream;
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->ws_pose, s->pose, 2 * N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->ws_vel, s->vel, 2 * N * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->ws_params, s->params, N * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "mark_window");
    s->ws_valid = true;
    s->ws_frames = s->window_frames;
    return IH_OK;
}

ih_status sim_refine_elites(ih_sim *s, int32_t frame0, int32_t T, const float *obs, const ih_opt_config *opt,
                            int32_t steps, float step_scale, float beta, float width, int32_t *elite_out,
                            double *cost_before, double *cost_after, uint64_t *accepted_out, float *start_pose_out,
                            float *start_params_out) {
    if (!s) return IH_ERR_ARG;
    if (s->pd) return refuse_pd(s, "sim_refine_elites");
    if (s->dcfg.warm) return fail(s, IH_ERR_ARG, "the adjoint differentiates the cold-started solver only");
    if (!obs) return fail(s, IH_ERR_ARG, "obs is required");
    ih_status r = check_opt(s, opt);
    if (r != IH_OK) return r;
    r = check_horizon(s, frame0, T);
    if (r != IH_OK) return r;
    if (steps < 0 || steps > 63 || !(step_scale > 0.0f) || !std::isfinite(step_scale))
        return fail(s, IH_ERR_ARG, "steps must be in [0, 63] and step_scale positive");
    if (!(beta > 0.0f) || !std::isfinite(beta) || !(width > 0.0f) || !std::isfinite(width))
        return fail(s, IH_ERR_ARG, "beta and width must be positive");
    if (!s->ws_valid) return fail(s, IH_ERR_STATE, "no window start marked (sim_mark_window)");
    if (s->window_frames - s->ws_frames != T)
        return fail(s, IH_ERR_STATE, "%d frames scored since the window start, expected %d",
                    s->window_frames - s->ws_frames, T);
    const int N = s->cfg.n_envs;
    int k = (int)std::floor((double)opt->elite_frac * (double)N);
    k = std::max(1, std::min(k, N));
    cudaStream_t st = s->stream;
    // elites of the window (the optimizer's own selection); the first trial is
    // the window start itself
    OptArgs oa = opt_args(s, opt, 0, nullptr, nullptr);
    cudaError_t e = launch_select(oa, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "refine select");
    size_t stride = 0;
    int imax = 0;
    r = adjoint_prepare(s, k, s->elite_env, T, T, &stride, &imax);
    if (r != IH_OK) return r;
    AdjArgs a = adjoint_args(s, frame0, T, T, obs, beta, width);
    a.n = k; a.envs = s->elite_env; a.vel = s->ws_vel;
    a.cost = s->r_cost; a.grad = s->r_grad; a.scratch = s->adj_scratch; a.stride = stride; a.iters_max = imax;
    a.out_pose = s->end_pose; a.out_vel = s->end_vel; a.seg_tape = s->adj_seg ? 1 : 0;
    RefineArgs ra;
    ra.k = k; ra.elite = s->elite_env; ra.tr_pose = s->tr_pose; ra.tr_params = s->tr_params;
    ra.best_pose = s->best_pose; ra.best_params = s->best_params; ra.best_grad = s->best_grad;
    ra.best_c = s->best_c; ra.c0 = s->c0; ra.scale = s->scale; ra.cost = s->r_cost; ra.grad = s->r_grad;
    ra.end_pose = s->end_pose; ra.end_vel = s->end_vel;
    ra.best_end_pose = s->best_end_pose; ra.best_end_vel = s->best_end_vel; ra.accepted = s->r_acc;
    for (int d = 0; d < 8; ++d) ra.eta[d] = step_scale * opt->floor_std[d];
    ra.m_lo = opt->m_lo; ra.m_hi = opt->m_hi; ra.mu_lo = opt->mu_lo; ra.mu_hi = opt->mu_hi;
    ra.ws_pose = s->ws_pose; ra.ws_params = s->ws_params;
    ra.pose = s->pose; ra.vel = s->vel; ra.params = s->params;
    ra.c_sum = s->c_sum; ra.c_mean = s->c_mean; ra.n_window = s->n_window;
    // each launch evaluates the elites' trials, and each elite's group then
    // takes its refinement step; after the last trial (its cost only) the
    // groups restore the best states and commit the improved elites' windows
    a.refine = 1;
    for (int it = 0; it <= steps && e == cudaSuccess; ++it) {
        a.forward_only = it == steps ? 1 : 0;
        a.pose = it == 0 ? s->ws_pose : s->tr_pose;
        a.params = it == 0 ? s->ws_params : s->tr_params;
        ra.step = it;
        ra.last = it == steps ? 1 : 0;
        a.rf = ra;
        e = launch_adjoint(a, st);
    }
    if (e == cudaSuccess && elite_out)
        e = cudaMemcpyAsync(elite_out, s->elite_env, k * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && cost_before)
        e = cudaMemcpyAsync(cost_before, s->c0, k * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && cost_after)
        e = cudaMemcpyAsync(cost_after, s->best_c, k * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && accepted_out)
        e = cudaMemcpyAsync(accepted_out, s->r_acc, k * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && start_pose_out)
        e = cudaMemcpyAsync(start_pose_out, s->best_pose, 2 * (size_t)k * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && start_params_out)
        e = cudaMemcpyAsync(start_params_out, s->best_params, (size_t)k * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "refine");
    return IH_OK;
}

ih_status sim_sync(ih_sim *s) {
    if (!s) return IH_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "sync");
    return IH_OK;
}

const char *sim_last_error(const ih_sim *s) {
    if (!s) return g_create_err.c_str();
    return s->err.c_str();
}

}  // extern "C"
