"""Seeded synthetic inputs for the in-hand tracking hot path.

This module builds the *inputs* only: object sphere clusters, the hand's fixed
geometry, sensor-pad layout, the commanded joint trajectory u_t, the nominal
initial pose and the per-configuration constants. It contains none of the
method's arithmetic (no kinematics, contact, solver, cost or optimizer step),
so that the FP64 oracle and the CUDA path can both be fed from it without
sharing any computation.

The paper's own inputs (YCB meshes and point clouds, 24 teleoperated
trajectories, BioTac recordings; Sec. IV) are not available; the objects and
trajectories here stand in for them:

* objects are clusters of spheres (box of 27, cylinder of 64, Fibonacci
  sphere of 16, L-shaped composite of 256, mug of 128), each generated with
  its sphere centres already centred on their mean;
* the hand is a palm box (8 x 8 x 2 cm, top face at z = +0.01 m) plus 4 or 5
  fingers of 4 capsule links (3 cm long, 8 mm radius) rooted on the palm top
  around the object; the commanded joint angles u_t (desired joint positions,
  Sec. III-A) are seeded sinusoids that open and close the grasp.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------
# objects (body-frame sphere clusters: rows of x, y, z, radius in metres)
# ----------------------------------------------------------------------------


def _centred(rows: np.ndarray) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.float64).copy()
    rows[:, :3] -= rows[:, :3].mean(axis=0)
    return rows


def box27(side: float = 0.05, radius: float = 0.0083) -> np.ndarray:
    """A cube of the given side as a 3x3x3 grid of equal spheres."""
    half = side / 2 - radius
    g = np.linspace(-half, half, 3)
    pts = np.array([(x, y, z) for z in g for y in g for x in g])
    return _centred(np.column_stack([pts, np.full(len(pts), radius)]))


def cylinder64(radius: float = 0.03, height: float = 0.08, r_s: float = 0.008,
               layers: int = 4, per_ring: int = 16) -> np.ndarray:
    """Upright cylinder: `layers` rings of `per_ring` spheres on radius R - r_s."""
    ring = radius - r_s
    zs = np.linspace(-(height / 2 - r_s), height / 2 - r_s, layers)
    rows = []
    for li, z in enumerate(zs):
        off = 0.5 * (li % 2) * 2 * math.pi / per_ring  # stagger alternate rings
        for k in range(per_ring):
            a = off + 2 * math.pi * k / per_ring
            rows.append((ring * math.cos(a), ring * math.sin(a), z, r_s))
    return _centred(np.array(rows))


def sphere16(outer: float = 0.025, r_s: float = 0.009) -> np.ndarray:
    """Fibonacci shell of 16 spheres whose outer envelope has radius `outer`."""
    n = 16
    shell = outer - r_s
    golden = math.pi * (3 - math.sqrt(5))
    rows = []
    for k in range(n):
        z = 1 - 2 * (k + 0.5) / n
        rr = math.sqrt(max(0.0, 1 - z * z))
        a = golden * k
        rows.append((shell * rr * math.cos(a), shell * rr * math.sin(a), shell * z, r_s))
    return _centred(np.array(rows))


def l_composite256(r_s: float = 0.003) -> np.ndarray:
    """Two 4x4x8 blocks of spheres joined into an L (one upright, one lying)."""
    sp = 2 * r_s
    rows = []
    for iz in range(8):          # upright block: 4 (x) x 4 (y) x 8 (z)
        for iy in range(4):
            for ix in range(4):
                rows.append((ix * sp, iy * sp, iz * sp, r_s))
    for iz in range(4):          # lying block: 8 (x) x 4 (y) x 4 (z), beside it
        for iy in range(4):
            for ix in range(8):
                rows.append(((4 + ix) * sp, iy * sp, iz * sp, r_s))
    return _centred(np.array(rows))


def mug128(radius: float = 0.03, height: float = 0.08, r_s: float = 0.006,
           handle_r_s: float = 0.005, handle_yaw: float = math.radians(36.0)) -> np.ndarray:
    """Mug-like composite: a 7 x 16 cylindrical shell plus a 16-sphere handle arc."""
    ring = radius - r_s
    rows = []
    zs = np.linspace(-(height / 2 - r_s), height / 2 - r_s, 7)
    for li, z in enumerate(zs):
        off = 0.5 * (li % 2) * 2 * math.pi / 16
        for k in range(16):
            a = off + 2 * math.pi * k / 16
            rows.append((ring * math.cos(a), ring * math.sin(a), z, r_s))
    # handle: a half ring in the vertical plane through `handle_yaw`
    hc = radius          # arc centre on the outer wall
    hr = 0.022           # arc radius
    cy, sy = math.cos(handle_yaw), math.sin(handle_yaw)
    for k in range(16):
        a = math.radians(-80.0 + 160.0 * k / 15)
        rad = hc + hr * math.cos(a)
        rows.append((rad * cy, rad * sy, hr * math.sin(a), handle_r_s))
    return _centred(np.array(rows))


OBJECTS = {
    "box27": box27,
    "cylinder64": cylinder64,
    "sphere16": sphere16,
    "l256": l_composite256,
    "mug128": mug128,
}


def horizontal_halfwidth(rows: np.ndarray) -> float:
    """Largest horizontal distance of the cluster's envelope from its centre."""
    return float(np.max(np.hypot(rows[:, 0], rows[:, 1]) + rows[:, 3]))


def bottom_depth(rows: np.ndarray) -> float:
    """Distance from the cluster centre down to its lowest sphere surface."""
    return float(-np.min(rows[:, 2] - rows[:, 3]))


# ----------------------------------------------------------------------------
# scene and configuration records
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Scene:
    """Fixed geometry shared by every environment.

    shapes       list of (S, 4) float64 arrays (body-frame sphere centre, radius)
    palm_half    half extents of the palm box (link 0, at the origin)
    finger_root  (F, 4): root position x, y, z and yaw (rad) of each finger
    link_len     capsule length of every finger link
    link_rad     capsule radius of every finger link
    pad_link     (P,) int32 link index of each sensor pad (0 = palm)
    pad_s0/s1    (P,) axial interval of the pad along the capsule, in [0, 1]
    """

    shapes: list
    palm_half: np.ndarray
    finger_root: np.ndarray
    link_len: float
    link_rad: float
    pad_link: np.ndarray
    pad_s0: np.ndarray
    pad_s1: np.ndarray

    @property
    def n_fingers(self) -> int:
        return int(self.finger_root.shape[0])

    @property
    def n_links(self) -> int:
        return 1 + 4 * self.n_fingers

    @property
    def n_joints(self) -> int:
        return 4 * self.n_fingers

    @property
    def n_pads(self) -> int:
        return int(self.pad_link.shape[0])

    def flat_spheres(self):
        """(first, count, rows) arrays of the concatenated shape table."""
        counts = np.array([len(s) for s in self.shapes], dtype=np.int32)
        first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int32)
        rows = np.concatenate(self.shapes, axis=0).astype(np.float64)
        return first, counts, rows


@dataclasses.dataclass
class SimConfig:
    """Per-configuration constants of the step, the sensors and the cost."""

    frame_dt: float = 1.0 / 30.0
    substeps: int = 2
    iters: int = 20
    margin: float = 0.002        # speculative contact margin (m)
    beta: float = 0.2            # penetration-recovery factor
    slop: float = 0.0005         # allowed penetration (m)
    vmax: float = 1.0            # cap on the recovery speed (m/s)
    gravity: tuple = (0.0, 0.0, -9.81)
    tau: float = 0.02            # contact-sensor on/off threshold (N)
    w_force: float = 1.0         # weight of the force-difference term (1/N^2)
    w_contact: float = 1.0       # weight of the contact-mismatch term
    c_max: int = 128             # contacts per environment per substep
    escape_radius: float = 0.3   # object farther than this from the palm = diverged
    warm_start: bool = False     # start each contact's impulse from its pair's last substep
    # the hand: "kinematic" (joints follow u_t exactly) or "pd" (joint-angle PD
    # controller toward u_t, joints pushed back by the contacts)
    hand: str = "kinematic"
    kp: float = 2.0              # PD stiffness (N m/rad)
    kd: float = 0.05             # PD damping (N m s/rad)
    armature: float = 1e-3       # joint inertia (kg m^2)
    v_slip: float = 0.005        # translational slip threshold (m/s)
    w_slip: float = 0.1          # rotational slip threshold (rad/s)
    # weights w1..w10 of the full cost (PD hand): q, pad position, pad rotation,
    # contact mismatch, force magnitude, force angle, slip mismatch, slip angle,
    # rotational-slip mismatch, rotational-slip direction
    w_full: tuple = (10.0, 100.0, 10.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)


@dataclasses.dataclass
class OptConfig:
    """Optimizer run every `window` frames.

    kind "elite": elite-weighted Gaussian resample (the configuration's PBO
    variant); "wrs" / "reps": a PMF over all simulations (softmax of the costs
    with temperature wrs_lambda, or the REPS temperature for the KL bound
    reps_epsilon), N draws with replacement, and isotropic exploration of every
    simulation: parameters by sigma_theta, and the pose by sigma_pose
    (explore "pose") or the velocity by sigma_vel (explore "velocity")."""

    window: int = 10
    elite_frac: float = 0.1
    floor_std: tuple = (0.001, 0.001, 0.001, 0.01, 0.01, 0.01, 0.005, 0.02)
    m_range: tuple = (0.01, 1.0)
    mu_range: tuple = (0.05, 2.0)
    kind: str = "elite"
    wrs_lambda: float = 1.0
    reps_epsilon: float = 0.5
    sigma_pose: tuple = (0.001, 0.001, 0.001, 0.01, 0.01, 0.01)
    sigma_theta: tuple = (0.005, 0.02)
    explore: str = "pose"
    sigma_vel: tuple = (0.01, 0.01, 0.01, 0.1, 0.1, 0.1)


@dataclasses.dataclass
class InitSampling:
    """Initial perturbation of pose and draw of (mass, friction)."""

    sigma_p: float = 0.005
    sigma_r: float = math.radians(5.0)
    m_range: tuple = (0.05, 0.3)
    mu_range: tuple = (0.3, 1.2)


# ----------------------------------------------------------------------------
# hand, pads, trajectory
# ----------------------------------------------------------------------------


def make_hand(n_fingers: int, root_radius: float, palm_top: float = 0.01,
              yaw0: float = 0.0) -> np.ndarray:
    yaws = yaw0 + 2 * math.pi * np.arange(n_fingers) / n_fingers
    return np.array([(root_radius * math.cos(a), root_radius * math.sin(a), palm_top, a)
                     for a in yaws], dtype=np.float64)


def pads_fingertips(n_fingers: int):
    """Two whole-link pads per finger: distal (link 3) and middle (link 2)."""
    link, s0, s1 = [], [], []
    for f in range(n_fingers):
        for j in (3, 2):
            link.append(1 + 4 * f + j)
            s0.append(0.0)
            s1.append(1.0)
    return (np.array(link, dtype=np.int32), np.array(s0), np.array(s1))


def pads_sixteen(n_fingers: int = 5):
    """Distal link split in two axial halves, middle link, and the palm."""
    link, s0, s1 = [], [], []
    for f in range(n_fingers):
        d = 1 + 4 * f + 3
        link += [d, d]
        s0 += [0.0, 0.5]
        s1 += [0.5, 1.0]
    for f in range(n_fingers):
        link.append(1 + 4 * f + 2)
        s0.append(0.0)
        s1.append(1.0)
    link.append(0)
    s0.append(0.0)
    s1.append(1.0)
    return (np.array(link, dtype=np.int32), np.array(s0), np.array(s1))


def joint_trajectory(n_fingers: int, frames: int, frame_dt: float, seed: int,
                     amp=(0.3, 0.8), freq=(0.5, 1.5)) -> np.ndarray:
    """Commanded joint angles u_t at the frame boundaries, (frames + 1, 4F) float32.

    Joint 4f+0 is the finger's abduction, 0.25 A sin(2 pi f t + phi); joints
    4f+1..4f+3 are flexions, A (1 - cos(2 pi f t)) / 2, so the hand starts open
    at rest and closes into a grasp. A ~ U[amp], f ~ U[freq], phi ~ U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    d = 4 * n_fingers
    a = rng.uniform(amp[0], amp[1], d)
    f = rng.uniform(freq[0], freq[1], d)
    ph = rng.uniform(0.0, 2 * math.pi, d)
    t = np.arange(frames + 1, dtype=np.float64)[:, None] * frame_dt
    q = a * (1 - np.cos(2 * math.pi * f * t)) / 2
    abd = 0.25 * a * np.sin(2 * math.pi * f * t + ph)
    for k in range(n_fingers):
        q[:, 4 * k] = abd[:, 4 * k]
    return q.astype(np.float32)


def theta_draw(seed: int, m_range, mu_range):
    """Hidden ground-truth (mass, friction) drawn from the prior's ranges."""
    rng = np.random.default_rng(seed)
    return (float(rng.uniform(*m_range)), float(rng.uniform(*mu_range)))


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    sim: SimConfig
    opt: OptConfig
    init: InitSampling
    n_envs: int
    frames: int
    q_traj: np.ndarray            # (frames + 1, D) float32
    shape_id: np.ndarray          # (N,) int32
    iters: np.ndarray             # (N,) int32
    nominal_pose: np.ndarray      # (8,) float32: x y z pad, qw qx qy qz -- the initial estimate
    theta_gt: tuple
    seed: int
    gt_pose: np.ndarray = None    # (8,) float32: the true initial pose (the estimate's error applied)

    def describe(self) -> dict:
        s = [len(x) for x in self.scene.shapes]
        return {"workload": self.name, "n_envs": self.n_envs, "frames": self.frames,
                "spheres_per_shape": s, "links": self.scene.n_links,
                "pads": self.scene.n_pads, "substeps": self.sim.substeps,
                "iters": sorted(set(int(i) for i in self.iters)), "seed": self.seed}


def _nominal(rows: np.ndarray, palm_top: float = 0.01) -> np.ndarray:
    return np.array([0.0, 0.0, palm_top + bottom_depth(rows), 0.0, 1.0, 0.0, 0.0, 0.0],
                    dtype=np.float32)


def _root_radius(rows_list, link_rad: float) -> float:
    return max(horizontal_halfwidth(r) for r in rows_list) + link_rad + 0.0025


def make_workload(name: str, n_envs: int | None = None, frames: int | None = None,
                  seed: int = 2002_12160) -> Workload:
    """Synthetic workloads standing in for the paper's objects and trajectories.

    tracking_box27   N=16,  box of 27 spheres, 4 fingers, 8 pads, I=20, 2 substeps,
                     150 frames (the FP32-vs-FP64 parity workload)
    tracking_cyl64   N=1024, cylinder of 64 spheres, same hand, 300 frames,
                     optimizer every 10 frames
    uneven_mixed     N=8192, shapes from {16, 27, 64, 256 spheres}, 5 fingers,
                     16 pads, I drawn from {10, 20, 40}
    adjoint_mixed    N=1024, box and cylinder, 30-frame horizon
    sweep_mug128     N=1024..32768, mug of 128 spheres, 5 fingers, 16 pads,
                     I=40, 4 substeps
    """
    link_len, link_rad = 0.03, 0.008
    palm_half = np.array([0.04, 0.04, 0.01])
    rng = np.random.default_rng(seed + 17)
    sim = SimConfig()
    opt = OptConfig()
    init = InitSampling()
    if name == "tracking_box27":
        shapes = [box27()]
        n, fr, nf = 16, 150, 4
        pads = pads_fingertips(nf)
        sid = np.zeros(n if n_envs is None else n_envs, np.int32)
    elif name == "tracking_cyl64":
        shapes = [cylinder64()]
        n, fr, nf = 1024, 300, 4
        pads = pads_fingertips(nf)
        sid = np.zeros(n if n_envs is None else n_envs, np.int32)
    elif name == "uneven_mixed":
        shapes = [sphere16(), box27(), cylinder64(), l_composite256()]
        n, fr, nf = 8192, 60, 5
        pads = pads_sixteen(nf)
        sim.c_max = 256
        sid = rng.integers(0, 4, n if n_envs is None else n_envs).astype(np.int32)
    elif name == "adjoint_mixed":
        shapes = [box27(), cylinder64()]
        n, fr, nf = 1024, 30, 4
        pads = pads_fingertips(nf)
        sid = rng.integers(0, 2, n if n_envs is None else n_envs).astype(np.int32)
    elif name == "sweep_mug128":
        shapes = [mug128()]
        n, fr, nf = 1024, 60, 5
        pads = pads_sixteen(nf)
        sim.substeps, sim.iters, sim.c_max = 4, 40, 256
        sid = np.zeros(n if n_envs is None else n_envs, np.int32)
    else:
        raise ValueError(f"unknown workload {name!r}")
    n = n if n_envs is None else n_envs
    fr = fr if frames is None else frames
    if name == "uneven_mixed":
        iters = rng.choice(np.array([10, 20, 40], np.int32), n).astype(np.int32)
    else:
        iters = np.full(n, sim.iters, np.int32)
    # fingers at 72 deg spacing put the mug handle (at 36 deg) between two fingers
    root = make_hand(nf, _root_radius(shapes, link_rad), palm_top=palm_half[2])
    scene = Scene(shapes=shapes, palm_half=palm_half, finger_root=root,
                  link_len=link_len, link_rad=link_rad,
                  pad_link=pads[0], pad_s0=pads[1], pad_s1=pads[2])
    q = joint_trajectory(nf, fr, sim.frame_dt, seed)
    nominal = _nominal(shapes[0], palm_half[2])
    theta_gt = theta_draw(seed + 1, init.m_range, init.mu_range)
    return Workload(name=name, scene=scene, sim=sim, opt=opt, init=init, n_envs=n,
                    frames=fr, q_traj=q, shape_id=sid, iters=iters,
                    nominal_pose=nominal, theta_gt=theta_gt, seed=seed,
                    gt_pose=estimate_error(nominal, init, seed + 2))


def estimate_error(nominal: np.ndarray, init: InitSampling, seed: int) -> np.ndarray:
    """The true initial pose: the initial estimate (`nominal`) off by one draw
    of the same noise the simulations are sampled with (translation
    N(0, sigma_p^2) per axis; rotation by a world-frame rotation vector
    N(0, sigma_r^2) per axis, applied on the left), so that the truth is
    not the centre of the samples (the paper's initial pose noise, Sec. IV)."""
    rng = np.random.default_rng(seed)
    dp = rng.normal(0.0, init.sigma_p, 3)
    w = rng.normal(0.0, init.sigma_r, 3)
    th = float(np.linalg.norm(w))
    axis = w / th if th > 0 else np.array([1.0, 0.0, 0.0])
    qd = np.array([math.cos(th / 2), *(math.sin(th / 2) * axis)])
    q0 = nominal[4:8].astype(np.float64)
    qw = np.array([qd[0] * q0[0] - qd[1:] @ q0[1:],
                   *(qd[0] * q0[1:] + q0[0] * qd[1:] + np.cross(qd[1:], q0[1:]))])
    qw /= np.linalg.norm(qw)
    out = nominal.astype(np.float64).copy()
    out[:3] += dp
    out[4:8] = qw
    return out.astype(np.float32)


def nominal_pose_for(scene: Scene, shape: int, palm_top: float = 0.01) -> np.ndarray:
    """Resting pose (centre above the palm top, identity rotation) for a shape."""
    return _nominal(scene.shapes[shape], palm_top)


# ----------------------------------------------------------------------------
# small scenes for closed-form checks
# ----------------------------------------------------------------------------


def ground_scene(shape_rows: np.ndarray, ground_half=(0.5, 0.5, 0.01)) -> Scene:
    """A wide static ground box (the palm, link 0) and no fingers."""
    return Scene(shapes=[np.asarray(shape_rows, np.float64)],
                 palm_half=np.asarray(ground_half, np.float64),
                 finger_root=np.zeros((0, 4)), link_len=0.03, link_rad=0.008,
                 pad_link=np.array([0], np.int32), pad_s0=np.array([0.0]),
                 pad_s1=np.array([1.0]))


def slab9(spacing: float = 0.0167, radius: float = 0.0083) -> np.ndarray:
    """A flat 3x3 layer of spheres (low centre of mass, for sliding tests)."""
    g = np.array([-spacing, 0.0, spacing])
    pts = np.array([(x, y, 0.0) for y in g for x in g])
    return _centred(np.column_stack([pts, np.full(9, radius)]))


def pose8(pos, quat_wxyz) -> np.ndarray:
    p = np.zeros(8, np.float32)
    p[:3] = pos
    p[4:] = quat_wxyz
    return p
