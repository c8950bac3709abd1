"""FP64 CPU oracle of the in-hand tracking hot path (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path never does: it shares
no code with the oracle, and the oracle shares none with it. The arithmetic
lives in ``inhand_oracle.c`` (plain C, FP64); this module compiles it with gcc
when needed and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inhand_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DIAG = 6  # per-env diagnostics of orc_step
NONFINITE, ESCAPED, OVERFLOW = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so with gcc (FP64, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Scene(C.Structure):
    _fields_ = [("n_shapes", C.c_int32), ("shape_first", C.c_void_p), ("shape_count", C.c_void_p),
                ("spheres", C.c_void_p), ("palm_half", C.c_double * 3), ("n_fingers", C.c_int32),
                ("finger_root", C.c_void_p), ("link_len", C.c_double), ("link_rad", C.c_double),
                ("n_pads", C.c_int32), ("pad_link", C.c_void_p), ("pad_s0", C.c_void_p),
                ("pad_s1", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("frame_dt", C.c_double), ("substeps", C.c_int32), ("iters", C.c_int32),
                ("margin", C.c_double), ("beta", C.c_double), ("slop", C.c_double),
                ("vmax", C.c_double), ("gravity", C.c_double * 3), ("tau", C.c_double),
                ("w_force", C.c_double), ("w_contact", C.c_double), ("c_max", C.c_int32),
                ("escape_radius", C.c_double)]


class PD(C.Structure):
    _fields_ = [("kp", C.c_double), ("kd", C.c_double), ("armature", C.c_double), ("v_slip", C.c_double),
                ("w_slip", C.c_double)]


class Opt(C.Structure):
    _fields_ = [("elite_frac", C.c_double), ("floor_std", C.c_double * 8), ("m_lo", C.c_double),
                ("m_hi", C.c_double), ("mu_lo", C.c_double), ("mu_hi", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_fk.argtypes = [P, P, P]
            L.orc_contacts.argtypes = [P, P, C.c_int, P, P, C.c_int, P]
            L.orc_unit_inertia.argtypes = [P, C.c_int, P]
            L.orc_step.argtypes = [P, P, C.c_int, P, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P, P, C.c_int]
            L.orc_cost.argtypes = [P, C.c_int, C.c_int, P, P, P, P, C.c_int, P, P]
            L.orc_step_pd.argtypes = [P, P, P, C.c_int, P, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P, P, P,
                                      P, P, P, P, C.c_int]
            L.orc_cost_full.argtypes = [P, C.c_double, C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P, P,
                                        P, C.c_int, P, P]
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_philox4x32_10.restype = None
            L.orc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, P]
            L.orc_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P]
            L.orc_sample_initial.argtypes = [C.c_int, P, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_double, C.c_double, C.c_uint64, P, P]
            L.orc_cholesky8.argtypes = [P, P]
            L.orc_optimizer.argtypes = [P, C.c_int, P, P, P, P, P, C.c_uint64, C.c_uint32, P, P]
            L.orc_softmax_update.argtypes = [P, C.c_int, P, P, P, P, P, C.c_uint64, C.c_uint32, P, P]
            L.orc_reps_eta.argtypes = [C.c_int, P, C.c_double, C.POINTER(C.c_int)]
            L.orc_reps_eta.restype = C.c_double
            L.orc_add.argtypes = [P, C.c_int, P, P]
            L.orc_add.restype = C.c_double
            L.orc_quat_exp.argtypes = [P, P]
            L.orc_link_point_velocity.argtypes = [P, P, P, C.c_double, P]
            L.orc_link_point_velocity.restype = None
            L.orc_quat_log.argtypes = [P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleScene:
    """Holds the ctypes scene record and keeps its numpy buffers alive."""

    def __init__(self, scene):
        first, count, rows = scene.flat_spheres()
        self._keep = [np.ascontiguousarray(first, np.int32), np.ascontiguousarray(count, np.int32),
                      np.ascontiguousarray(rows, np.float64),
                      np.ascontiguousarray(scene.finger_root, np.float64).reshape(-1, 4),
                      np.ascontiguousarray(scene.pad_link, np.int32),
                      np.ascontiguousarray(scene.pad_s0, np.float64),
                      np.ascontiguousarray(scene.pad_s1, np.float64)]
        k = self._keep
        self.rec = Scene(len(scene.shapes), k[0].ctypes.data, k[1].ctypes.data, k[2].ctypes.data,
                         (C.c_double * 3)(*scene.palm_half), scene.n_fingers,
                         k[3].ctypes.data if k[3].size else None, scene.link_len, scene.link_rad,
                         scene.n_pads, k[4].ctypes.data, k[5].ctypes.data, k[6].ctypes.data)
        self.n_links = 1 + 4 * scene.n_fingers
        self.n_pads = scene.n_pads
        self.n_joints = 4 * scene.n_fingers
        self.scene = scene


def make_config(sim) -> Config:
    return Config(sim.frame_dt, sim.substeps, sim.iters, sim.margin, sim.beta, sim.slop, sim.vmax,
                  (C.c_double * 3)(*sim.gravity), sim.tau, sim.w_force, sim.w_contact, sim.c_max,
                  sim.escape_radius)


def make_opt(opt) -> Opt:
    return Opt(opt.elite_frac, (C.c_double * 8)(*opt.floor_std), opt.m_range[0], opt.m_range[1],
               opt.mu_range[0], opt.mu_range[1])


def pose8_to7(p8: np.ndarray) -> np.ndarray:
    """(…, 8) float pose (xyz, pad, wxyz) -> (…, 7) float64 (xyz, wxyz), exact."""
    p8 = np.asarray(p8)
    return np.concatenate([p8[..., :3], p8[..., 4:8]], axis=-1).astype(np.float64)


def vel8_to6(v8: np.ndarray) -> np.ndarray:
    v8 = np.asarray(v8)
    return np.concatenate([v8[..., :3], v8[..., 4:7]], axis=-1).astype(np.float64)


def fk(osc: OracleScene, q) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    out = np.zeros((osc.n_links, 7))
    lib().orc_fk(C.byref(osc.rec), _p(q), _p(out))
    return out


def contacts(osc: OracleScene, sim, shape: int, pose7, link_pose, max_out: int = 4096) -> np.ndarray:
    cfg = make_config(sim)
    pose7 = np.ascontiguousarray(pose7, np.float64)
    lp = np.ascontiguousarray(link_pose, np.float64)
    out = np.zeros((max_out, 12))
    n = lib().orc_contacts(C.byref(osc.rec), C.byref(cfg), shape, _p(pose7), _p(lp), max_out, _p(out))
    return out[:min(n, max_out)]


def link_point_velocity(pose_a7, pose_b7, p, h: float) -> np.ndarray:
    """Velocity of the point p carried rigidly by a link from pose A to pose B
    over a substep h (the contact's link velocity of the kinematic hand)."""
    a = np.ascontiguousarray(pose_a7, np.float64)
    b = np.ascontiguousarray(pose_b7, np.float64)
    pp = np.ascontiguousarray(p, np.float64)
    out = np.zeros(3)
    lib().orc_link_point_velocity(_p(a), _p(b), _p(pp), h, _p(out))
    return out


def unit_inertia(osc: OracleScene, shape: int) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_unit_inertia(C.byref(osc.rec), shape, _p(out))
    return out.reshape(3, 3)


class State:
    """FP64 state of N environments: pose (N,7), vel (N,6), theta (N,2), status (N,)."""

    def __init__(self, pose7, vel6, theta, shape=None, iters=None, status=None):
        self.pose = np.ascontiguousarray(pose7, np.float64).copy()
        self.vel = np.ascontiguousarray(vel6, np.float64).copy()
        self.theta = np.ascontiguousarray(theta, np.float64).copy()
        n = self.pose.shape[0]
        self.shape = np.zeros(n, np.int32) if shape is None else np.ascontiguousarray(shape, np.int32).copy()
        self.iters = None if iters is None else np.ascontiguousarray(iters, np.int32).copy()
        self.status = np.zeros(n, np.int32) if status is None else np.ascontiguousarray(status, np.int32).copy()

    @property
    def n(self) -> int:
        return self.pose.shape[0]

    def subset(self, idx):
        s = State(self.pose[idx], self.vel[idx], self.theta[idx], self.shape[idx],
                  None if self.iters is None else self.iters[idx], self.status[idx])
        if self.cache_n is not None:
            s.cache_n, s.cache_id, s.cache_lam = (a[idx].copy() for a in (self.cache_n, self.cache_id, self.cache_lam))
        if self.qj is not None:
            s.qj, s.qdj = self.qj[idx].copy(), self.qdj[idx].copy()
        return s

    cache_n = cache_id = cache_lam = None
    qj = qdj = None   # PD-driven hand: joint positions and velocities (N, D)

    def hand(self, q0, D: int | None = None):
        """Start a PD-driven hand at joint positions q0 (D,) or (N, D), at rest."""
        q0 = np.asarray(q0, np.float64)
        self.qj = np.ascontiguousarray(np.broadcast_to(q0, (self.n, q0.shape[-1])), np.float64).copy()
        self.qdj = np.zeros_like(self.qj)
        return self

    def copy_hand(self, parent):
        """Replaced environments take their parent's hand state with the rest of it."""
        if self.qj is not None:
            self.qj = self.qj[parent].copy()
            self.qdj = self.qdj[parent].copy()

    def warm_cache(self, cap: int):
        """Start a (cold) warm-start cache of `cap` pairs per environment."""
        self.cache_n = np.zeros(self.n, np.int32)
        self.cache_id = np.zeros((self.n, cap), np.int32)
        self.cache_lam = np.zeros((self.n, cap, 3))
        return self

    def drop_cache(self, envs):
        """Environments whose state was replaced start cold again."""
        if self.cache_n is not None:
            self.cache_n[envs] = 0


def step(osc: OracleScene, sim, st: State, q_traj, frame0: int, n_frames: int = 1):
    """Advance `st` in place; returns (forces (N,P,3) of the last frame, diag (N,6))."""
    cfg = make_config(sim)
    q = np.ascontiguousarray(q_traj, np.float64)
    forces = np.zeros((st.n, osc.n_pads, 3))
    diag = np.zeros((st.n, DIAG))
    warm = getattr(sim, "warm_start", False)
    if warm and st.cache_n is None:
        st.warm_cache(int(sim.c_max))
    cache = (_p(st.cache_n), _p(st.cache_id), _p(st.cache_lam), st.cache_id.shape[1]) if warm else (None, None, None, 0)
    lib().orc_step(C.byref(osc.rec), C.byref(cfg), st.n, _p(q), frame0, n_frames, _p(st.pose),
                   _p(st.vel), _p(st.theta), _p(st.shape),
                   None if st.iters is None else _p(st.iters), _p(st.status), _p(forces), _p(diag), *cache)
    return forces, diag


def make_pd(sim) -> PD:
    return PD(sim.kp, sim.kd, sim.armature, sim.v_slip, sim.w_slip)


class Obs:
    """Observation o_t of N environments with the PD-driven hand (Sec. III-A):
    q (N, D), pad pose (N, P, 7: position, wxyz), force (N, P, 3), slip
    direction (N, P, 2) and flags (N, P: bit 0 translational slip, bit 1
    rotational slip, bit 2 spin > 0)."""

    def __init__(self, q, pad_pose, forces, slip_d, flags, slip_mag=None):
        self.q, self.pad_pose, self.forces, self.slip_d, self.flags = q, pad_pose, forces, slip_d, flags
        self.slip_mag = slip_mag   # (N, P, 2): mean relative tangential speed and spin (oracle only)

    def env(self, i) -> "Obs":
        return Obs(*(a[i:i + 1].copy() for a in (self.q, self.pad_pose, self.forces, self.slip_d, self.flags)))


def step_pd(osc: OracleScene, sim, st: State, q_traj, frame0: int, n_frames: int = 1, last_cap: int = 0):
    """Advance `st` (with st.qj, st.qdj) in place with the PD-driven hand.
    Returns (Obs of the last frame, diag (N, 6)) and, with last_cap > 0, the
    last substep's contacts (N, last_cap, 7: link, point, impulse) and counts."""
    assert st.qj is not None, "the state has no hand joints: State.hand(q0)"
    cfg = make_config(sim)
    pd = make_pd(sim)
    q = np.ascontiguousarray(q_traj, np.float64)
    n, P = st.n, osc.n_pads
    forces = np.zeros((n, P, 3))
    pad_pose = np.zeros((n, P, 7))
    slip_d = np.zeros((n, P, 2))
    flags = np.zeros((n, P), np.int32)
    slip_mag = np.zeros((n, P, 2))
    diag = np.zeros((n, DIAG))
    last = np.zeros((n, max(last_cap, 1), 7))
    last_n = np.zeros(n, np.int32)
    lib().orc_step_pd(C.byref(osc.rec), C.byref(cfg), C.byref(pd), n, _p(q), frame0, n_frames, _p(st.pose),
                      _p(st.vel), _p(st.theta), _p(st.shape), None if st.iters is None else _p(st.iters),
                      _p(st.status), _p(st.qj), _p(st.qdj), _p(forces), _p(pad_pose), _p(slip_d), _p(flags),
                      _p(slip_mag), _p(diag), _p(last) if last_cap > 0 else None, _p(last_n) if last_cap > 0 else None, last_cap)
    obs = Obs(st.qj.copy(), pad_pose, forces, slip_d, flags, slip_mag)
    if last_cap > 0:
        return obs, diag, last, last_n
    return obs, diag


def cost_full(sim, obs: Obs, gt: Obs, status, c_sum, n_window: int):
    """Full cost of Sec. III-C (all ten terms) of every environment against the
    ground-truth observation `gt` (one environment); accumulates into c_sum in
    place and returns (i*, c_mean, frame cost)."""
    w = np.ascontiguousarray(sim.w_full, np.float64)
    n, D = obs.q.shape
    P = obs.forces.shape[1]
    arr = lambda a, t=np.float64: np.ascontiguousarray(a, t)
    o = [arr(obs.q), arr(obs.pad_pose), arr(obs.forces), arr(obs.slip_d), arr(obs.flags, np.int32)]
    g = [arr(gt.q), arr(gt.pad_pose), arr(gt.forces), arr(gt.slip_d), arr(gt.flags, np.int32)]
    status = arr(status, np.int32)
    c_mean = np.zeros(n)
    c_frame = np.zeros(n)
    i = lib().orc_cost_full(_p(w), C.c_double(sim.tau), n, D, P, *[_p(a) for a in o], *[_p(a) for a in g],
                            _p(status), _p(c_sum), n_window, _p(c_mean), _p(c_frame))
    return i, c_mean, c_frame


def cost(sim, forces, obs, status, c_sum, n_window: int):
    """Accumulates one frame's cost into c_sum (in place); returns (i*, c_mean, frame cost)."""
    cfg = make_config(sim)
    forces = np.ascontiguousarray(forces, np.float64)
    obs = np.ascontiguousarray(obs, np.float64)
    status = np.ascontiguousarray(status, np.int32)
    n, p = forces.shape[0], forces.shape[1]
    c_mean = np.zeros(n)
    c_frame = np.zeros(n)
    i = lib().orc_cost(C.byref(cfg), n, p, _p(forces), _p(obs), _p(status), _p(c_sum), n_window,
                       _p(c_mean), _p(c_frame))
    return i, c_mean, c_frame


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def normals(seed: int, stream: int, index: int, env: int, n: int) -> np.ndarray:
    out = np.zeros(n)
    lib().orc_normals(seed, stream, index, env, n, _p(out))
    return out


def uniforms(seed: int, stream: int, index: int, env: int, blk: int) -> np.ndarray:
    out = np.zeros(2)
    lib().orc_uniforms(seed, stream, index, env, blk, _p(out))
    return out


def sample_initial(n: int, nominal7, init, seed: int):
    nominal7 = np.ascontiguousarray(nominal7, np.float64)
    pose = np.zeros((n, 7))
    theta = np.zeros((n, 2))
    lib().orc_sample_initial(n, _p(nominal7), init.sigma_p, init.sigma_r, init.m_range[0],
                             init.m_range[1], init.mu_range[0], init.mu_range[1], seed,
                             _p(pose), _p(theta))
    return pose, theta


def cholesky8(A) -> tuple[int, np.ndarray]:
    A = np.ascontiguousarray(A, np.float64)
    L = np.zeros((8, 8))
    rc = lib().orc_cholesky8(_p(A), _p(L))
    return rc, L


def optimizer(opt, st: State, C_mean, seed: int, update_index: int):
    """In-place update of st; returns (i*, parent (N,), stats dict)."""
    o = make_opt(opt)
    Cm = np.ascontiguousarray(C_mean, np.float64)
    parent = np.zeros(st.n, np.int32)
    stats = np.zeros(139)
    i = lib().orc_optimizer(C.byref(o), st.n, _p(Cm), _p(st.pose), _p(st.vel), _p(st.theta),
                            _p(st.status), seed, update_index, _p(parent), _p(stats))
    st.drop_cache(parent != np.arange(st.n))   # replaced environments start cold
    if i >= 0:
        st.copy_hand(parent)
    return i, parent, {"mean": stats[:8].copy(), "cov": stats[8:72].reshape(8, 8).copy(),
                       "L": stats[72:136].reshape(8, 8).copy(), "k": int(stats[136]),
                       "istar": int(stats[137]), "sd": float(stats[138])}


class SoftOpt(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lam", C.c_double), ("epsilon", C.c_double),
                ("sigma_pose", C.c_double * 6), ("sigma_theta", C.c_double * 2),
                ("explore_velocity", C.c_int32), ("sigma_vel", C.c_double * 6),
                ("m_lo", C.c_double), ("m_hi", C.c_double), ("mu_lo", C.c_double), ("mu_hi", C.c_double)]


def make_soft_opt(opt) -> SoftOpt:
    kind = {"wrs": 1, "reps": 2}[opt.kind]
    return SoftOpt(kind, opt.wrs_lambda, opt.reps_epsilon, (C.c_double * 6)(*opt.sigma_pose),
                   (C.c_double * 2)(*opt.sigma_theta), 1 if opt.explore == "velocity" else 0,
                   (C.c_double * 6)(*opt.sigma_vel), opt.m_range[0], opt.m_range[1], opt.mu_range[0],
                   opt.mu_range[1])


def softmax_update(opt, st: State, C_mean, seed: int, update_index: int):
    """WRS / REPS update of st in place (Sec. III-D); returns (i*, parent, stats)."""
    o = make_soft_opt(opt)
    Cm = np.ascontiguousarray(C_mean, np.float64)
    parent = np.zeros(st.n, np.int32)
    stats = np.zeros(7)
    i = lib().orc_softmax_update(C.byref(o), st.n, _p(Cm), _p(st.pose), _p(st.vel), _p(st.theta),
                                 _p(st.status), seed, update_index, _p(parent), _p(stats))
    st.drop_cache(np.arange(st.n))   # every environment is replaced
    st.copy_hand(parent)
    return i, parent, {"eta": stats[0], "wsum": stats[1], "kl": stats[2], "n_finite": int(stats[3]),
                       "cmin": stats[4], "cmax": stats[5], "iters": int(stats[6])}


def reps_eta(C_mean, epsilon: float):
    """REPS temperature eta* minimising the dual (+inf: uniform; 0: on the minima)."""
    Cm = np.ascontiguousarray(C_mean, np.float64)
    it = C.c_int(0)
    eta = lib().orc_reps_eta(len(Cm), _p(Cm), C.c_double(epsilon), C.byref(it))
    return eta, it.value


def add(osc: OracleScene, shape: int, pose_a7, pose_b7) -> float:
    a = np.ascontiguousarray(pose_a7, np.float64)
    b = np.ascontiguousarray(pose_b7, np.float64)
    return float(lib().orc_add(C.byref(osc.rec), shape, _p(a), _p(b)))


def quat_exp(w3) -> np.ndarray:
    w = np.ascontiguousarray(w3, np.float64)
    out = np.zeros(4)
    lib().orc_quat_exp(_p(w), _p(out))
    return out


def quat_log(q4) -> np.ndarray:
    q = np.ascontiguousarray(q4, np.float64)
    out = np.zeros(3)
    lib().orc_quat_log(_p(q), _p(out))
    return out
