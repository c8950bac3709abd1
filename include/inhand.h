/*
 * inhand.h -- C ABI of libinhand.so, the GB300 (sm_103a) hot path of
 * sim-in-the-loop in-hand object pose tracking (arXiv 2002.12160).
 *
 * The library steps N independent hand-plus-object simulations (the forward
 * model s_{t+1} = f(s_t, u_t, theta) of Sec. III-A), reads the contact-sensor
 * forces c_t^(l) (Sec. III-A), scores every environment against the observed
 * forces and tracks i* = argmin_i C_i (Eqs. 1-2, Sec. III-C), and runs the
 * periodic resample-and-perturb update of pose, mass and friction
 * (Sec. III-D, Algorithm 1). Every computation runs in CUDA kernels.
 *
 * Conventions, shared by every entry point:
 *  - Units are SI (m, kg, s, N, rad). The palm is at the origin, its top face
 *    at z = +palm_half[2], gravity is `gravity` (normally (0, 0, -9.81)).
 *  - Array arguments documented "device" are device pointers owned by the
 *    caller; "host" arguments are read during the call and may be freed after
 *    it returns. Nothing here takes ownership of a caller's buffer.
 *  - Per-environment layouts (row-major, N rows):
 *      pose   float[N][8]: position x y z, 0, quaternion w x y z (world frame)
 *      vel    float[N][8]: linear x y z, 0, angular x y z (world frame), 0
 *      params float[N][2]: mass (kg), friction coefficient mu
 *      forces float[N][P][3]: force on each sensor pad by the object (N)
 *  - Every call is asynchronous on the handle's CUDA stream (sim_create,
 *    sim_set_stream). Host-detectable errors (bad arguments) return at once
 *    and change nothing; device-side conditions are reported per environment
 *    through the env_status bits below and never stop the batch.
 *  - A handle is not thread safe; different handles are independent.
 *  - No call throws; every call returns an ih_status. sim_last_error() gives
 *    a message for the last non-IH_OK status of that handle.
 */
#ifndef INHAND_H
#define INHAND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ih_sim ih_sim;

typedef enum {
    IH_OK = 0,
    IH_ERR_ARG = 1,      /* invalid argument (nothing was launched) */
    IH_ERR_CUDA = 2,     /* a CUDA runtime call or launch failed */
    IH_ERR_OOM = 3,      /* device allocation failed */
    IH_ERR_TIMEOUT = 4,  /* reserved: no kernel here waits on another */
    IH_ERR_STATE = 5,    /* call not valid in the handle's current state */
    IH_ERR_OVERFLOW = 6  /* a size exceeds a fixed capacity */
} ih_status;

/* per-environment status bits (sticky until the optimizer replaces the env) */
#define IH_ENV_NONFINITE 1   /* a pose or velocity component is not finite */
#define IH_ENV_ESCAPED   2   /* object farther than escape_radius from the palm */
#define IH_ENV_OVERFLOW  4   /* more contacts than c_max in one substep */
#define IH_ENV_INVALID   8   /* sim_set_state received an invalid value */

/* Fixed geometry shared by all environments (host arrays, copied at create).
 * Link 0 is the palm box; finger f has links 1+4f+j, j = 0..3, each a capsule
 * of length link_len and radius link_rad along its frame's +x axis:
 *   T_0 = Trans(root_f) Rz(yaw_f + q_{4f}) Ry(-pi/2),
 *   T_j = T_{j-1} Trans(link_len, 0, 0) Ry(-q_{4f+j}), j = 1..3.
 * Object shapes are clusters of spheres in the body frame; the library takes
 * the centroid of the sphere centres as the body origin. A contact on link l
 * at axial fraction t belongs to the first pad k with pad_link[k] == l and
 * pad_s0[k] <= t < pad_s1[k] (t <= 1 when pad_s1[k] >= 1); palm contacts
 * belong to the first pad whose link is 0. */
typedef struct {
    int32_t n_shapes;             /* >= 1 */
    const int32_t *shape_first;   /* host [n_shapes] first row in `spheres` */
    const int32_t *shape_count;   /* host [n_shapes] spheres, 1..IH_MAX_SPHERES */
    const float *spheres;         /* host [total][4] centre x y z, radius */
    float palm_half[3];           /* palm box half extents */
    int32_t n_fingers;            /* 0..IH_MAX_FINGERS */
    const float *finger_root;     /* host [F][4] root x y z, yaw */
    float link_len, link_rad;
    int32_t n_pads;               /* 1..IH_MAX_PADS */
    const int32_t *pad_link;      /* host [P] */
    const float *pad_s0, *pad_s1; /* host [P] */
} ih_scene;

#define IH_MAX_SPHERES 256
#define IH_MAX_FINGERS 7
#define IH_MAX_PADS 32
#define IH_MAX_CONTACTS 256

/* Step, sensor and cost constants. */
typedef struct {
    int32_t n_envs;        /* N >= 1 */
    int32_t max_frames;    /* capacity of the commanded-trajectory table */
    float frame_dt;        /* 1/30 s */
    int32_t substeps;      /* ns >= 1, h = frame_dt / ns */
    int32_t iters;         /* Jacobi iterations when no per-env count is set */
    float margin;          /* pair is a contact when its gap d < margin */
    float beta, slop, vmax;/* bias: d/h if d > 0 else max(beta min(d+slop,0)/h, -vmax) */
    float gravity[3];
    float tau;             /* sensor on/off threshold on |c| (N) */
    float w_force;         /* weight of sum_l |c_sim - c_obs|^2 */
    float w_contact;       /* weight of each on/off mismatch */
    int32_t c_max;         /* contacts per env per substep, <= IH_MAX_CONTACTS */
    float escape_radius;   /* |x| beyond this marks the env escaped */
    int32_t warm_start;    /* 0: every substep's solve starts from zero impulses;
                              1: each contact starts from the final impulse of the
                              same (link, sphere) pair in the environment's
                              previous substep (cache per environment, carried
                              across launches; emptied by sim_sample_initial,
                              sim_set_state and when the optimizer replaces the
                              environment). sim_adjoint and sim_refine_elites
                              refuse a warm-started handle (IH_ERR_ARG). */
    /* The hand (Sec. III-A: s_t holds the joint angles of articulated bodies;
     * u_t are desired joint positions; Sec. IV: a joint-angle PD controller).
     * hand = IH_HAND_KINEMATIC: the joints follow u_t exactly (shared by all
     * environments). hand = IH_HAND_PD: each environment's joints are state,
     * each a revolute joint of inertia `armature` driven toward u_t by
     * kp (u - q) - kd qd, integrated implicitly per substep, and pushed back
     * by the contacts (the solve updates the object and the joints together);
     * the handle then also reports the full observation (sim_read_observation)
     * and scores it with all ten cost terms (cost_eval_full). With IH_HAND_PD,
     * warm_start must be 0, and sim_step_track, sim_step_frames,
     * sim_track_window, sim_autotune, sim_set_variant, sim_adjoint and
     * sim_refine_elites return IH_ERR_ARG. */
    int32_t hand;
    float kp, kd, armature;  /* N m/rad, N m s/rad, kg m^2 (armature > 0) */
    float v_slip, w_slip;    /* a pad slips when its mean relative tangential
                                speed exceeds v_slip (m/s); it slips rotationally
                                when its relative spin about the normal exceeds
                                w_slip (rad/s) */
    float w_full[10];        /* w1..w10 of the full cost (cost_eval_full) */
} ih_config;

enum { IH_HAND_KINEMATIC = 0, IH_HAND_PD = 1 };

/* Optimizer kinds (Sec. III-D). */
enum { IH_OPT_ELITE = 0, IH_OPT_WRS = 1, IH_OPT_REPS = 2 };

/* Optimizer constants. IH_OPT_ELITE: elite-weighted Gaussian resample (uses
 * elite_frac, floor_std and the clamps). IH_OPT_WRS / IH_OPT_REPS: a PMF over
 * all simulations, N draws with replacement and isotropic exploration of every
 * simulation (uses wrs_lambda or reps_epsilon, the sigma_* fields and the
 * clamps). */
typedef struct {
    float elite_frac;      /* k = max(1, floor(elite_frac N)) elites */
    float floor_std[8];    /* exploration floor: x y z (m), rotation (rad) x3, m (kg), mu */
    float m_lo, m_hi;      /* clamp of the perturbed mass */
    float mu_lo, mu_hi;    /* clamp of the perturbed friction */
    int32_t kind;          /* IH_OPT_ELITE, IH_OPT_WRS or IH_OPT_REPS */
    float wrs_lambda;      /* WRS temperature lambda > 0 */
    float reps_epsilon;    /* REPS bound epsilon > 0 on KL(P || uniform) */
    float sigma_pose[6];   /* exploration of the pose: x y z (m), rotation (rad) x3 */
    float sigma_theta[2];  /* exploration of m (kg) and mu */
    int32_t explore_velocity;  /* 1: explore the velocity by sigma_vel instead of the pose */
    float sigma_vel[6];    /* linear (m/s) x3, angular (rad/s) x3 */
} ih_opt_config;

/* Create a simulator for cfg->n_envs environments on the current device.
 * Copies the scene, allocates the handle's device state (poses, velocities,
 * parameters, forces, cost sums, link-pose table, optimizer scratch) and
 * derives each shape's centroid frame, unit inertia and bounding radius on
 * the GPU. `seed` keys every random stream (Philox4x32-10). `stream` is a
 * cudaStream_t (NULL = legacy default stream). Errors: IH_ERR_ARG for a bad
 * scene or config, IH_ERR_OOM, IH_ERR_CUDA. Passage: Sec. III-B (K
 * concurrent simulations initialised from s_0). */
ih_status sim_create(const ih_scene *scene, const ih_config *cfg, uint64_t seed,
                     void *stream, ih_sim **out);

/* Free the handle and everything it allocated (synchronises its stream). */
ih_status sim_destroy(ih_sim *sim);

/* Use another cudaStream_t for subsequent calls. */
ih_status sim_set_stream(ih_sim *sim, void *stream);

/* Upload commanded joint angles u_t (desired joint positions, Sec. III-A) for
 * frames [frame0, frame0 + n_frames) and compute the kinematic hand's link
 * poses at every substep boundary of those frames. q is device
 * float[n_frames + 1][4F]: row k holds the command at the start of frame
 * frame0 + k (the last row closes the last frame); it may be NULL when the
 * hand has no fingers. Within a frame the hand moves linearly in joint
 * space. Errors: IH_ERR_ARG if the range exceeds max_frames. The same
 * command goes to every environment (Sec. III-B). */
ih_status sim_set_commands(ih_sim *sim, int32_t frame0, int32_t n_frames, const float *q);

/* Initial sampling (Sec. III-D, Algorithm 1 initialisation): for every env i,
 *   x = x0 + sigma_p n_{0..2},  R = exp([sigma_r n_{3..5}]x) R0,
 *   m ~ U[m_lo, m_hi], mu ~ U[mu_lo, mu_hi], velocities 0, status 0,
 * with n standard normals (Box-Muller, FP64) of Philox4x32-10 counter
 * (0, 0, i, block 0..2) and the uniforms from block 3, key = seed.
 * nominal_pose is host float[8] (layout of `pose`). Also clears the cost
 * window. Errors: IH_ERR_ARG for negative sigmas or empty ranges. */
ih_status sim_sample_initial(ih_sim *sim, const float *nominal_pose, float sigma_p, float sigma_r,
                             float m_lo, float m_hi, float mu_lo, float mu_hi);

/* Overwrite the state of all N environments from device arrays (pose, vel,
 * params as above; shape_id int32[N] and iters int32[N] may be NULL to keep
 * the current values). Values are checked on the GPU: a non-finite number,
 * mass <= 0, mu < 0, a shape id outside [0, n_shapes) or an iteration count
 * outside [0, 4096] sets IH_ENV_INVALID for that env (which then costs +inf
 * and is not stepped). Other status bits are cleared. */
ih_status sim_set_state(ih_sim *sim, const float *pose, const float *vel, const float *params,
                        const int32_t *shape_id, const int32_t *iters);

/* Copy the state out to device arrays; any pointer may be NULL. */
ih_status sim_get_state(ih_sim *sim, float *pose, float *vel, float *params, int32_t *env_status);

/* Copy the warm-start cache out (a handle created with warm_start = 1; any
 * other handle gives IH_ERR_ARG) to device arrays: count int32[N], the number
 * of contacts of each environment's last stepped substep, and entries
 * float[N][c_max][4], per contact in pair order its final impulse (x, y, z, in
 * N s) and, in the fourth float, the bits of its int32 pair id
 * (link << 8 | sphere). Entries past count are unspecified. entries must be
 * 16-byte aligned. Asynchronous on the handle's stream. */
ih_status sim_get_warm_cache(ih_sim *sim, int32_t *count, float *entries);

/* Advance every environment over frames [frame0, frame0 + n_frames) with the
 * commands set by sim_set_commands (Algorithm 1, "step simulation"). Per
 * substep: gravity prediction, object spheres to world, bounding-sphere cull,
 * sphere-capsule / sphere-box narrowphase (a pair is a contact when its gap
 * d < margin), per-contact effective masses and bias, `iters` Jacobi
 * projected-impulse iterations with Coulomb friction and 1/n_c relaxation,
 * symplectic Euler with the exact rotation update, and sensor-pad sums.
 * Environments with IH_ENV_NONFINITE/ESCAPED/OVERFLOW/INVALID are skipped.
 * The pad forces of the last frame stepped stay in the handle for
 * sim_read_sensors and cost_eval. Errors: IH_ERR_ARG for a frame range
 * without commands. */
ih_status sim_step(ih_sim *sim, int32_t frame0, int32_t n_frames);

/* One frame of Algorithm 1 in one kernel: sim_step(frame, 1) followed by
 * cost_eval(obs, ...), with the frame's cost computed from the same FP32 pad
 * forces in the same FP64 order, so results equal the two separate calls bit
 * for bit. obs is device float[P][3]; cost_mean (double[N]), argmin
 * (int32[1]) and est_pose (float[8]) are device outputs and may be NULL.
 * Passages: Sec. III-A (step, observation), Sec. III-C and Eqs. 1-2 (cost,
 * i*). */
ih_status sim_step_track(ih_sim *sim, int32_t frame, const float *obs, double *cost_mean,
                         int32_t *argmin, float *est_pose);

/* T scored frames [frame0, frame0 + T) in one kernel launch: for every
 * environment, T frames of sim_step, each followed by its frame cost, window
 * sum and window mean as in sim_step_track (same arithmetic, same order); the
 * mean and the pose after every frame are kept in the handle for
 * sim_frames_argmin. The environments need no argmin to advance, so the T
 * frames run without a grid-wide step in between. obs is device
 * float[T][P][3]. sim_frames_argmin must follow before any other scored call
 * (sim_step_track, sim_step_frames, cost_eval, optimizer_update,
 * sim_track_window), which return IH_ERR_STATE until it has. Passages:
 * Sec. III-A, Sec. III-C, Algorithm 1. */
ih_status sim_step_frames(ih_sim *sim, int32_t frame0, int32_t T, const float *obs);

/* The argmin i*_f (NaN = +inf, ties to the lowest index) and the pose of i*_f
 * after frame f, for each frame of the last sim_step_frames call; outputs
 * (device, may be NULL): est_pose float[T][8], argmin int32[T]. Results equal
 * T calls of sim_step_track bit for bit. IH_ERR_STATE without a preceding
 * sim_step_frames. */
ih_status sim_frames_argmin(ih_sim *sim, float *est_pose, int32_t *argmin);

/* One tracking window of Algorithm 1: for k = 0..T-1, sim_step_track(frame0
 * + k, obs + k P 3, ...) writing est_pose[k] and argmin[k], then
 * optimizer_update(opt, update_index), launched as sim_step_frames, then
 * sim_frames_argmin's kernel and the optimizer's kernels side by side (two
 * branches of the graph: the argmin reads only the frames' buffers, the
 * update sets i* and the window count itself). obs is device float[T][P][3];
 * est_pose (float[T][8]) and argmin (int32[T]) are device outputs (may be
 * NULL). The window's launches are captured once into a CUDA graph and
 * replayed on later calls with the same T, step shape and optimizer
 * constants; per-window arguments reach the graph through a device
 * descriptor, so pointers may change between calls. The first call (and any
 * call after a change) captures, so it must not itself be made while the
 * stream is being captured. Results equal the separate calls bit for bit. */
ih_status sim_track_window(ih_sim *sim, int32_t frame0, int32_t T, const float *obs,
                           const ih_opt_config *opt, uint32_t update_index, float *est_pose,
                           int32_t *argmin);

/* Copy the last frame's pad forces (device float[N][P][3], world frame,
 * averaged over the frame's substeps: the observation c_t^(l) of Sec. III-A)
 * and the status bits (device int32[N]); either may be NULL. */
ih_status sim_read_sensors(ih_sim *sim, float *forces, int32_t *env_status);

/* PD hand only (IH_HAND_PD; IH_ERR_ARG otherwise): the last frame's full
 * observation o_t of Sec. III-A besides the forces, to device arrays (any may
 * be NULL):
 *   q        float[N][D]      joint angles q_t (D = 4 n_fingers)
 *   pad_pose float[N][P][8]   each pad's position (x y z, 0) -- the link's
 *                             origin plus the middle of the pad's axial interval
 *                             along the capsule, or the palm's top centre --
 *                             and the link's rotation (w x y z): P_t, R_t
 *   slip     float[N][P][4]   (d_x, d_y, flags, 0): flags are int32 bits stored
 *                             in the float (bit 0: translational slip, bit 1:
 *                             rotational slip, bit 2: spin about the normal is
 *                             positive); d is the unit slip direction in the
 *                             pad's contact plane (first axis: the link's axis
 *                             projected into the plane; second: normal x
 *                             first), zero without translational slip. The slip
 *                             is the normal-impulse-weighted mean of the
 *                             object's velocity relative to the link at the
 *                             pad's contacts over the frame's substeps.
 * pad_pose and slip must be 16-byte aligned. */
ih_status sim_read_observation(ih_sim *sim, float *q, float *pad_pose, float *slip);

/* PD hand only: set (q, qd device float[N][D], qd may be NULL for rest) or
 * read (either may be NULL) every environment's joint angles and velocities.
 * sim_sample_initial and sim_set_state put each hand at rest at the frame-0
 * command when commands for frame 0 have been uploaded, else at q = 0. */
ih_status sim_set_hand(ih_sim *sim, const float *q, const float *qd);
ih_status sim_get_hand(ih_sim *sim, float *q, float *qd);

/* PD hand only: score the last stepped frame with the full cost of Sec. III-C
 * against the ground truth's observation (device arrays in the layouts of
 * sim_read_observation for one environment: q float[D], pad_pose float[P][8],
 * forces float[P][3], slip float[P][4]):
 *   cost_i = w1 |q - q_gt| + sum_l [ w2 |P - P_gt| + w3 angle(R^-1 R_gt)
 *            + w4 (1 - alpha) + alpha (w5 | |c| - |c_gt| | + w6 angle(c, c_gt))
 *            + w7 (1 - beta) + beta w8 angle(d, d_gt)
 *            + w9 (1 - gamma) + gamma w10 |r - r_gt| ]
 * alpha, beta, gamma = 1 when the pads agree on contact (|c| > tau), on
 * translational and on rotational slip; the force angle counts only when both
 * are in contact, the slip angle only when both slip, |r - r_gt| only when
 * both slip rotationally. FP64; window mean, argmin and outputs as cost_eval. */
ih_status cost_eval_full(ih_sim *sim, const float *q, const float *pad_pose, const float *forces,
                         const float *slip, double *cost_mean, int32_t *argmin, float *est_pose);

/* PD hand only: T frames from frame0 in one step launch, each frame's
 * observation kept and then scored with the full cost (as cost_eval_full)
 * against the ground truth's observation of that frame by two further
 * launches (the pads' and joints' terms in parallel, then each environment's
 * sums and window means): q float[T][D], pad_pose float[T][P][8], forces float[T][P][3], slip
 * float[T][P][4] (device; pad_pose and slip 16-byte aligned). As with
 * sim_step_frames, sim_frames_argmin must follow (IH_ERR_STATE otherwise) and
 * gives every frame's argmin and estimate; results equal T calls of sim_step
 * and cost_eval_full. The handle allocates (on the first call, or for a larger
 * T, after synchronising its stream) device buffers of about
 * T x N x (4 D + 60 P + 44 + 8 (P + 1)) bytes for the frames' observations,
 * statuses, poses, window means and cost terms; they are freed with the
 * handle. */
ih_status sim_step_frames_full(ih_sim *sim, int32_t frame0, int32_t T, const float *q, const float *pad_pose,
                               const float *forces, const float *slip);

/* Score the last stepped frame against the observation (Sec. III-C, force and
 * contact-state terms; Eqs. 1-2 with the running mean of Algorithm 1):
 *   cost_i = sum_l [ w_force |c_il - o_l|^2 + w_contact ((|c_il| > tau) != (|o_l| > tau)) ]
 * in FP64 (+inf for a skipped env), C_i = (sum of costs since the window
 * start) / (frames in the window), i* = argmin C_i (NaN = +inf, ties to the
 * lowest index). obs is device float[P][3]. Outputs (device, any may be
 * NULL): cost_mean double[N], argmin int32[1], est_pose float[8] (pose of
 * i*). */
ih_status cost_eval(ih_sim *sim, const float *obs, double *cost_mean, int32_t *argmin,
                    float *est_pose);

/* Optimizer update (Sec. III-D, population-based variant with elite-weighted
 * Gaussian exploration; Algorithm 1, "update simulations"), on the current
 * window means C_i:
 *  1. rank by (C_i, i); the first k = max(1, floor(elite_frac N)) are elites;
 *  2. w_j = exp(-(C_j - C_min) / s) over the elites, s = standard deviation of
 *     their finite costs (uniform when s < 1e-12), normalised (FP64);
 *  3. z = [x, log(R R_{i*}^T), m, mu]; weighted mean and covariance Sigma_w
 *     over the elites; L = chol(Sigma_w + diag(floor_std^2)) (FP64);
 *  4. non-elites, in index order r = 0..N-k-1, draw parents by systematic
 *     resampling over the elites in index order at (u + r)/(N - k), u from
 *     Philox counter (2, update_index, 0, 0);
 *  5. each non-elite copies its parent's pose, velocity, parameters and
 *     status and adds L eps (eps from counter (1, update_index, i, 0..3)):
 *     x += d_0..2, R <- exp([d_3..5]x) R, m += d_6, mu += d_7, then clamps.
 * Elites are unchanged. The cost window is reset.
 * With opt->kind IH_OPT_WRS or IH_OPT_REPS instead (Sec. III-D, WRS and REPS):
 *  1. over the simulations with a finite C_i (the others get weight 0; all
 *     of them when none is finite), WRS P(i) ~ exp(-lambda (C_i - C_min));
 *     REPS P(i) ~ exp(R_i / eta*), R_i = C_max + C_min - C_i, eta* the
 *     minimiser of the dual eta eps + eta log((1/K) sum exp(R_i / eta)) (K
 *     finite simulations), by Newton steps on log eta inside a shrinking
 *     bracket, in FP64 (equal costs: uniform; eps >= log(K / #minima): the
 *     minima only);
 *  2. every simulation i takes the parent at the inverse CDF (index order) of
 *     u_i from Philox counter (3, update_index, i, 0) -- N draws with
 *     replacement -- and copies its state as it was before the update;
 *  3. explores with eps from counter (1, update_index, i, 0..3): m, mu +=
 *     sigma_theta eps_6,7 (clamped), and x += sigma_pose eps_0..2, R <-
 *     exp([sigma_pose eps_3..5]x) R, or with explore_velocity v, w +=
 *     sigma_vel eps_0..5 (the pose then changes only through the dynamics).
 * Outputs (device, may be NULL): argmin int32[1] = i*, parent int32[N]
 * (self for elites).
 * Errors: IH_ERR_ARG for elite_frac outside (0, 1] or bad clamps;
 * IH_ERR_STATE when no frame has been scored since the last reset. */
ih_status optimizer_update(ih_sim *sim, const ih_opt_config *opt, uint32_t update_index,
                           int32_t *argmin, int32_t *parent);

/* Work done by the step kernel since the last call with reset != 0:
 * out[0] = sphere-link tests after culling, out[1] = contacts, out[2] =
 * contact-iterations, out[3] = env-substeps stepped, out[4] = solver
 * iterations summed over env-substeps with contacts, out[5] = cluster-link
 * culling tests (host uint64[6]; synchronises the stream). */
ih_status sim_work_counters(ih_sim *sim, uint64_t *out, int32_t reset);

/* Choose the step kernel's shape -- threads per environment (16, 32, 64 or
 * 128) and register-resident contacts per thread -- by timing every
 * supported shape whose capacity covers c_max on frames [frame0, frame0 +
 * n_frames) of the current state (one warm-up run, then the best of three).
 * The state, forces and work counters are
 * restored after every trial, so the call leaves the simulation unchanged.
 * Results of different shapes agree up to FP32 summation order. chosen
 * (host int32[2], may be NULL) receives the shape; ms (host float[16], may be
 * NULL) the time of each tried shape in the order of sim_step_variants.
 * Synchronises the stream. Not a passage of the paper: the batching of
 * environments onto the GPU is this library's. */
ih_status sim_autotune(ih_sim *sim, int32_t frame0, int32_t n_frames, int32_t *chosen, float *ms);

/* Force the step kernel's shape (threads per env, contacts per thread);
 * IH_ERR_ARG if unsupported or below c_max. */
ih_status sim_set_variant(ih_sim *sim, int32_t threads_per_env, int32_t contacts_per_thread);

/* The supported shapes as pairs (threads per env, contacts per thread):
 * writes up to `cap` pairs into out (host int32[2 * cap]) and returns how
 * many exist. */
int32_t sim_step_variants(int32_t *out, int32_t cap);

/* Measured FP32 throughput of the current device: the denominator of the
 * step kernels' ALU roofline (their work is FP32 issue, not a dense
 * contraction). Runs `reps` launches (after two warm-up launches) of a kernel
 * in which every thread carries 8 independent FMA chains of 16 x iters FMAs,
 * with 2048 threads on each SM (the SM count is read from the device), timed
 * with CUDA events on `stream` (NULL = legacy default stream); an FMA counts
 * as 2 flop. tflops (host double, required) receives the measured TFLOP/s,
 * ms_per_launch and sm_count (host, may be NULL) the mean launch time and the
 * SM count. Allocates and frees a small output buffer; synchronises the
 * stream. Not a passage of the paper: a measurement of this GPU.
 * Errors: IH_ERR_ARG (iters or reps < 1, null tflops), IH_ERR_OOM,
 * IH_ERR_CUDA. */
ih_status ih_fp32_peak(int32_t iters, int32_t reps, void *stream, double *tflops, double *ms_per_launch,
                       int32_t *sm_count);

/* cost_eval for callers that cannot allocate device memory.
 *
 * Some callers may not call cudaMalloc at all: code running inside another
 * allocator's callbacks, a real-time loop that reserved all its device memory
 * up front, or a process held to a fixed memory budget on a shared GPU. Such a
 * caller cannot create a simulator handle (sim_create allocates) and cannot
 * hand us scratch space, but it can pass its own inputs and outputs. This
 * entry point computes the same per-environment cost, window mean and argmin
 * as cost_eval -- same FP64 arithmetic, same order, same tie rule -- from
 * caller buffers only, and allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *
 * The paper has no counterpart to this call; it exists for such callers.
 *
 * forces  device float[n_envs][n_pads][3]   pad forces of the frame
 * obs     device float[n_pads][3]           observed forces
 * env_status device int32[n_envs] or NULL   envs with IH_ENV_NONFINITE,
 *                                           ESCAPED, OVERFLOW or INVALID cost +inf
 * c_sum   device double[n_envs], in/out     window sums; the frame's cost is added
 * n_window frames in the window including this one (divides c_sum)
 * cost_mean device double[n_envs] or NULL   window means C_i
 * argmin  device int32[1]                   i* (NaN = +inf, ties to the lowest index)
 * stream  cudaStream_t (NULL = legacy default stream)
 *
 * Limits: n_envs <= 131072 (IH_ERR_OVERFLOW beyond it), n_pads <= IH_MAX_PADS.
 * Its scratch -- one partial per 32 environments and a counter, about 48 KiB --
 * is a fixed __device__ array that every GPU which loads this library holds
 * until the process exits. Every call looks up that array's device address in
 * the current device's context (so a device reset cannot leave a stale one);
 * the first lookup on a device may load the library's device code, so make
 * the first call on each device before any stream capture.
 * Every call shares the one array (each call re-zeroes its counter on the
 * stream), so calls that may overlap on the GPU -- on different streams, or
 * from different threads -- race and must be serialised by the caller.
 * Errors: IH_ERR_ARG (null or out-of-range argument), IH_ERR_OVERFLOW (too many
 * environments), IH_ERR_CUDA (device lookup or launch failed). */
ih_status cost_eval_static(const float *forces, const float *obs, const int32_t *env_status,
                           int32_t n_envs, int32_t n_pads, float tau, float w_force,
                           float w_contact, double *c_sum, int32_t n_window, double *cost_mean,
                           int32_t *argmin, void *stream);

/* Gradient of the tracking cost over a horizon, by reverse mode (the
 * derivative that the gradient-based refinement of the estimate needs; the
 * paper optimises without it, Sec. III-D, and this call adds it).
 *
 * For each selected environment i, from its current state (the state at the
 * start of frame0; left unchanged), the horizon's cost
 *   L_i = sum_{f = frame0}^{frame0 + horizon - 1} sum_l [ w_force |c_il,f - o_l,f|^2
 *                                                         + w_contact (contact-state mismatch) ]
 * (Sec. III-C on the frame step of Sec. III-A) and its derivatives with respect
 * to the initial position, the initial rotation (as a world-frame rotation
 * vector d applied on the left, q -> exp(d) q, at d = 0), the mass and the
 * friction coefficient. The contact-state terms are piecewise constant and
 * contribute no derivative. Derivatives of the two projections of the Jacobi
 * update are smoothed (the forward values stay exact): max(0, z) takes
 * sigmoid(beta z), and the radial clamp of a tangential impulse z onto the
 * Coulomb disk of radius L takes the derivative of z smin(|z|, L)/|z| with
 * smin(a, b) = (a + b - sqrt((a - b)^2 + (width b)^2)) / 2. Contact
 * membership, capsule end clamps, palm face choice and bias regimes are held
 * fixed. The state after every checkpoint_every-th frame is kept; the
 * reverse sweep recomputes the forward between checkpoints and, per substep,
 * once more with a record of the Jacobi iterations.
 *
 * obs        device float[horizon][P][3]  observed pad forces of each frame
 * envs       device int32[n] or NULL      environments to differentiate
 *                                         (NULL: environments 0..n-1)
 * n          1..N
 * beta       > 0, slope of the smoothed normal clamp (1 / (N s))
 * width      > 0, relative width of the smoothed disk clamp
 * cost       device double[n] or NULL     L_i (FP64, as the scored step; +inf
 *                                         for an environment that diverges or
 *                                         is invalid, NaN for an index outside
 *                                         [0, N))
 * grad       device float[n][8]           dL/d(x, y, z, rx, ry, rz, m, mu)
 *                                         (zero where the cost is not finite)
 * grad_quat  device float[n][4] or NULL   dL/d(q_w, q_x, q_y, q_z) of the
 *                                         initial quaternion's components
 *
 * Scratch: the handle grows a buffer of about (16 c_max (iters + 6) + 16
 * (horizon / checkpoint_every + 2 checkpoint_every substeps)) floats per
 * selected environment and keeps it until sim_destroy. Synchronises the stream
 * once to size it (the largest iteration count among the selected
 * environments is read back), so the call cannot be captured in a graph.
 * Errors: IH_ERR_ARG (frames without commands, n or a constant out of range,
 * null obs or grad), IH_ERR_OOM. */
ih_status sim_adjoint(ih_sim *sim, int32_t frame0, int32_t horizon, int32_t checkpoint_every,
                      const float *obs, const int32_t *envs, int32_t n, float beta, float width,
                      double *cost, float *grad, float *grad_quat);

/* Memory the adjoint may use to keep the tape (the Jacobi impulses of every
 * iteration) of all substeps of a checkpoint segment at once, in bytes
 * (default 16 GiB). Within the budget each substep of the forward is run twice
 * per gradient (the pass that computes the cost and checkpoints, and the
 * segment's recomputation, which records the tape); beyond it the tape of a
 * single substep is kept and each substep runs a third time just before its
 * reverse sweep. Results are the same bit for bit. 0 always takes the
 * smaller mode. Not a passage of the paper: a memory/time trade of this
 * library's checkpointing. */
ih_status sim_set_adjoint_memory(ih_sim *sim, uint64_t bytes);

/* The adjoint kernel's shape for sim_adjoint and sim_refine_elites: warps
 * per environment and contacts per thread held in registers over the Jacobi
 * iterations and their reverse; a substep's contacts beyond those (up to
 * c_max) run from the environment's scratch memory, in the same per-thread
 * order. Supported: (4, 1), (1, 1), (1, 2); (0, 0) restores the automatic
 * choice: (4, 1) while the environments are at most two per SM, else (1, 1)
 * when no shape has more than 32 spheres and (1, 2) otherwise.
 * Results of different shapes agree up to FP32 summation order.
 * IH_ERR_ARG for another pair. Not a passage of the paper: a tuning choice of
 * this library. */
ih_status sim_set_adjoint_variant(ih_sim *sim, int32_t warps_per_env, int32_t contacts_per_thread);

/* Snapshot every environment's state (pose, velocity, parameters) into the
 * handle: the start of a tracking window, for sim_refine_elites. */
ih_status sim_mark_window(ih_sim *sim);

/* Gradient refinement of the elite samples (an addition to the paper's
 * derivative-free update of Sec. III-D, run between the window's last scored
 * frame and optimizer_update).
 *
 * The window is frames [frame0, frame0 + T), all scored since the last
 * sim_mark_window; obs is device float[T][P][3], those frames' observations.
 * The elites are the optimizer's (the k = max(1, floor(elite_frac N)) lowest
 * window means, ties to the lowest index). Each elite's window-start state
 * z = (position, rotation, m, mu) is refined by `steps` steps
 *   s = eta g, z <- z - scale eta s / |s|,  eta = step_scale floor_std,
 * with g the gradient of the window's cost (sim_adjoint's, horizon T, same
 * smoothing beta and width; the rotation step is exp([dz]x) on the left, m and
 * mu are clamped to the optimizer's ranges). A step is kept when it lowers the
 * cost, otherwise the elite's scale halves and the next step starts from its
 * best state. An elite whose cost went down is then simulated from its best
 * window-start state to the window's end, and that end state, its parameters
 * and its window cost (sum and mean) replace the scored ones; the others keep
 * theirs. optimizer_update then resamples around the refined elites.
 * Outputs (device, k entries each, any may be NULL): elite_out int32 (the
 * elites, index order), cost_before double (window cost of the unrefined
 * state, as the adjoint's forward computes it), cost_after double (the best
 * cost found; <= cost_before), accepted_out uint64 (bit j set when evaluation
 * j was kept: bit 0, the unrefined state, always; bit j >= 1, the j-th
 * step), start_pose_out float[k][8] and start_params_out float[k][2] (the
 * best window-start pose and parameters found, the unrefined ones when no
 * step was kept).
 * Synchronises the stream once (adjoint scratch sizing).
 * Errors: IH_ERR_ARG (bad range or constant; steps must be in [0, 63]),
 * IH_ERR_STATE (no mark, or not exactly T frames scored since it),
 * IH_ERR_OOM. */
ih_status sim_refine_elites(ih_sim *sim, int32_t frame0, int32_t T, const float *obs,
                            const ih_opt_config *opt, int32_t steps, float step_scale, float beta,
                            float width, int32_t *elite_out, double *cost_before, double *cost_after,
                            uint64_t *accepted_out, float *start_pose_out, float *start_params_out);

/* Wait for the handle's stream; IH_ERR_CUDA if a kernel failed. */
ih_status sim_sync(ih_sim *sim);

/* Message for the handle's last error (never NULL, valid until the next
 * call on that handle). */
const char *sim_last_error(const ih_sim *sim);

#ifdef __cplusplus
}
#endif

#endif /* INHAND_H */
