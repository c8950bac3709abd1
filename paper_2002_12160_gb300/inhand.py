"""Thin ctypes binding of libinhand.so (include/inhand.h).

Argument marshalling only: every function forwards torch CUDA tensors' data
pointers and the current CUDA stream to the C ABI of the same name. All
computation runs in the library's kernels; there is no CPU fallback, and
loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libinhand.so")

IH_OK, IH_ERR_ARG, IH_ERR_CUDA, IH_ERR_OOM, IH_ERR_TIMEOUT, IH_ERR_STATE, IH_ERR_OVERFLOW = range(7)
ENV_NONFINITE, ENV_ESCAPED, ENV_OVERFLOW, ENV_INVALID = 1, 2, 4, 8
MAX_CONTACTS = 256


class InhandError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


class IHScene(C.Structure):
    _fields_ = [("n_shapes", C.c_int32), ("shape_first", C.c_void_p), ("shape_count", C.c_void_p),
                ("spheres", C.c_void_p), ("palm_half", C.c_float * 3), ("n_fingers", C.c_int32),
                ("finger_root", C.c_void_p), ("link_len", C.c_float), ("link_rad", C.c_float),
                ("n_pads", C.c_int32), ("pad_link", C.c_void_p), ("pad_s0", C.c_void_p),
                ("pad_s1", C.c_void_p)]


class IHConfig(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("max_frames", C.c_int32), ("frame_dt", C.c_float),
                ("substeps", C.c_int32), ("iters", C.c_int32), ("margin", C.c_float),
                ("beta", C.c_float), ("slop", C.c_float), ("vmax", C.c_float),
                ("gravity", C.c_float * 3), ("tau", C.c_float), ("w_force", C.c_float),
                ("w_contact", C.c_float), ("c_max", C.c_int32), ("escape_radius", C.c_float),
                ("warm_start", C.c_int32), ("hand", C.c_int32), ("kp", C.c_float), ("kd", C.c_float),
                ("armature", C.c_float), ("v_slip", C.c_float), ("w_slip", C.c_float),
                ("w_full", C.c_float * 10)]

HANDS = {"kinematic": 0, "pd": 1}


class IHOptConfig(C.Structure):
    _fields_ = [("elite_frac", C.c_float), ("floor_std", C.c_float * 8), ("m_lo", C.c_float),
                ("m_hi", C.c_float), ("mu_lo", C.c_float), ("mu_hi", C.c_float), ("kind", C.c_int32),
                ("wrs_lambda", C.c_float), ("reps_epsilon", C.c_float), ("sigma_pose", C.c_float * 6),
                ("sigma_theta", C.c_float * 2), ("explore_velocity", C.c_int32), ("sigma_vel", C.c_float * 6)]


OPT_KINDS = {"elite": 0, "wrs": 1, "reps": 2}


_lib = None
EXPORTS = ["sim_create", "sim_destroy", "sim_set_stream", "sim_set_commands", "sim_sample_initial",
           "sim_set_state", "sim_get_state", "sim_step", "sim_read_sensors", "cost_eval",
           "optimizer_update", "sim_work_counters", "sim_sync", "sim_last_error", "sim_autotune",
           "sim_set_variant", "sim_step_variants", "sim_step_track", "sim_track_window",
           "cost_eval_static", "sim_adjoint", "sim_mark_window", "sim_refine_elites",
           "sim_step_frames", "sim_frames_argmin", "sim_set_adjoint_memory", "sim_set_adjoint_variant",
           "sim_get_warm_cache", "sim_read_observation", "sim_set_hand", "sim_get_hand", "cost_eval_full", "sim_step_frames_full",
           "ih_fp32_peak"]


def lib() -> C.CDLL:
    """Load libinhand.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, I, U32 = C.c_void_p, C.c_int32, C.c_uint32
        sig = {
            "sim_create": [P, P, C.c_uint64, P, C.POINTER(P)],
            "sim_destroy": [P],
            "sim_set_stream": [P, P],
            "sim_set_commands": [P, I, I, P],
            "sim_sample_initial": [P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float],
            "sim_set_state": [P, P, P, P, P, P],
            "sim_get_state": [P, P, P, P, P],
            "sim_get_warm_cache": [P, P, P],
            "sim_read_observation": [P, P, P, P],
            "sim_set_hand": [P, P, P],
            "sim_get_hand": [P, P, P],
            "cost_eval_full": [P, P, P, P, P, P, P, P],
            "sim_step_frames_full": [P, I, I, P, P, P, P],
            "sim_step": [P, I, I],
            "sim_read_sensors": [P, P, P],
            "cost_eval": [P, P, P, P, P],
            "optimizer_update": [P, P, U32, P, P],
            "sim_work_counters": [P, P, I],
            "sim_sync": [P],
            "sim_autotune": [P, I, I, P, P],
            "sim_set_variant": [P, I, I],
            "sim_step_variants": [P, I],
            "sim_step_track": [P, I, P, P, P, P],
            "sim_track_window": [P, I, I, P, P, U32, P, P],
            "sim_adjoint": [P, I, I, I, P, P, I, C.c_float, C.c_float, P, P, P],
            "sim_mark_window": [P],
            "sim_set_adjoint_memory": [P, C.c_uint64],
            "sim_set_adjoint_variant": [P, I, I],
            "sim_step_frames": [P, I, I, P],
            "sim_frames_argmin": [P, P, P],
            "sim_refine_elites": [P, I, I, P, P, I, C.c_float, C.c_float, C.c_float, P, P, P, P, P, P],
            "ih_fp32_peak": [I, I, P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.sim_last_error.argtypes = [P]
        L.sim_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _check(t, dtype, shape, name):
    if t is None:
        return
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")


def _opt(opt) -> IHOptConfig:
    return IHOptConfig(opt.elite_frac, (C.c_float * 8)(*opt.floor_std), opt.m_range[0],
                       opt.m_range[1], opt.mu_range[0], opt.mu_range[1], OPT_KINDS[opt.kind], opt.wrs_lambda,
                       opt.reps_epsilon, (C.c_float * 6)(*opt.sigma_pose), (C.c_float * 2)(*opt.sigma_theta),
                       1 if opt.explore == "velocity" else 0, (C.c_float * 6)(*opt.sigma_vel))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Sim:
    """One handle of the C ABI: N environments of one scene on the current device."""

    def __init__(self, scene, sim_cfg, n_envs: int, max_frames: int, seed: int):
        L = lib()
        first, count, rows = scene.flat_spheres()
        self._keep = [np.ascontiguousarray(first, np.int32), np.ascontiguousarray(count, np.int32),
                      np.ascontiguousarray(rows, np.float32),
                      np.ascontiguousarray(scene.finger_root, np.float32).reshape(-1, 4),
                      np.ascontiguousarray(scene.pad_link, np.int32),
                      np.ascontiguousarray(scene.pad_s0, np.float32),
                      np.ascontiguousarray(scene.pad_s1, np.float32)]
        k = self._keep
        self._scene = IHScene(len(scene.shapes), k[0].ctypes.data, k[1].ctypes.data, k[2].ctypes.data,
                              (C.c_float * 3)(*scene.palm_half), scene.n_fingers,
                              k[3].ctypes.data if k[3].size else None, scene.link_len, scene.link_rad,
                              scene.n_pads, k[4].ctypes.data, k[5].ctypes.data, k[6].ctypes.data)
        self._cfg = IHConfig(n_envs, max_frames, sim_cfg.frame_dt, sim_cfg.substeps, sim_cfg.iters,
                             sim_cfg.margin, sim_cfg.beta, sim_cfg.slop, sim_cfg.vmax,
                             (C.c_float * 3)(*sim_cfg.gravity), sim_cfg.tau, sim_cfg.w_force,
                             sim_cfg.w_contact, sim_cfg.c_max, sim_cfg.escape_radius,
                             int(bool(sim_cfg.warm_start)), HANDS[sim_cfg.hand], sim_cfg.kp, sim_cfg.kd,
                             sim_cfg.armature, sim_cfg.v_slip, sim_cfg.w_slip, (C.c_float * 10)(*sim_cfg.w_full))
        self.n = n_envs
        self.n_pads = scene.n_pads
        self.n_joints = scene.n_joints
        self.max_frames = max_frames
        self.c_max = sim_cfg.c_max
        self.warm_start = bool(sim_cfg.warm_start)
        self.pd = sim_cfg.hand == "pd"
        h = C.c_void_p()
        rc = L.sim_create(C.byref(self._scene), C.byref(self._cfg), seed, _stream(), C.byref(h))
        if rc != IH_OK:
            raise InhandError("sim_create", rc, L.sim_last_error(None).decode())
        self._h = h

    # -- helpers
    def _call(self, name, *args):
        L = lib()
        L.sim_set_stream(self._h, _stream())
        rc = getattr(L, name)(self._h, *args)
        if rc != IH_OK:
            raise InhandError(name, rc, L.sim_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the C ABI, one method per entry point
    def sim_set_commands(self, frame0: int, q: torch.Tensor):
        _check(q, torch.float32, (q.shape[0], self.n_joints), "q")
        self._call("sim_set_commands", frame0, q.shape[0] - 1, _ptr(q) if q.numel() else None)

    def sim_sample_initial(self, nominal_pose, sigma_p, sigma_r, m_range, mu_range):
        nom = (C.c_float * 8)(*[float(v) for v in nominal_pose])
        self._call("sim_sample_initial", nom, sigma_p, sigma_r, m_range[0], m_range[1],
                   mu_range[0], mu_range[1])

    def sim_set_state(self, pose, vel, params, shape_id=None, iters=None):
        _check(pose, torch.float32, (self.n, 8), "pose")
        _check(vel, torch.float32, (self.n, 8), "vel")
        _check(params, torch.float32, (self.n, 2), "params")
        _check(shape_id, torch.int32, (self.n,), "shape_id")
        _check(iters, torch.int32, (self.n,), "iters")
        self._call("sim_set_state", _ptr(pose), _ptr(vel), _ptr(params), _ptr(shape_id), _ptr(iters))

    def sim_get_state(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        pose = torch.empty((self.n, 8), dtype=torch.float32, device=dev)
        vel = torch.empty((self.n, 8), dtype=torch.float32, device=dev)
        params = torch.empty((self.n, 2), dtype=torch.float32, device=dev)
        status = torch.empty((self.n,), dtype=torch.int32, device=dev)
        self._call("sim_get_state", _ptr(pose), _ptr(vel), _ptr(params), _ptr(status))
        return pose, vel, params, status

    def sim_step(self, frame0: int, n_frames: int = 1):
        self._call("sim_step", frame0, n_frames)

    def sim_get_warm_cache(self):
        """(count int32[N], impulse float32[N, c_max, 3], pair id int32[N, c_max]) of a
        warm-started handle: each environment's last substep's contacts."""
        dev = torch.device("cuda", torch.cuda.current_device())
        count = torch.empty((self.n,), dtype=torch.int32, device=dev)
        ent = torch.empty((self.n, self.c_max, 4), dtype=torch.float32, device=dev)
        self._call("sim_get_warm_cache", _ptr(count), _ptr(ent))
        return count, ent[..., :3], ent[..., 3].contiguous().view(torch.int32)

    def sim_read_sensors(self, forces=None, status=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        if forces is None:
            forces = torch.empty((self.n, self.n_pads, 3), dtype=torch.float32, device=dev)
        if status is None:
            status = torch.empty((self.n,), dtype=torch.int32, device=dev)
        self._call("sim_read_sensors", _ptr(forces), _ptr(status))
        return forces, status

    def cost_eval(self, obs, cost_mean=None, argmin=None, est_pose=None):
        _check(obs, torch.float32, (self.n_pads, 3), "obs")
        _check(cost_mean, torch.float64, (self.n,), "cost_mean")
        _check(argmin, torch.int32, (1,), "argmin")
        _check(est_pose, torch.float32, (8,), "est_pose")
        self._call("cost_eval", _ptr(obs), _ptr(cost_mean), _ptr(argmin), _ptr(est_pose))

    def sim_read_observation(self, q=None, pad_pose=None, slip=None):
        """PD hand: (q float32[N, D], pad_pose float32[N, P, 8], slip float32[N, P, 4]) of the last frame."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if q is None:
            q = torch.empty((self.n, self.n_joints), dtype=torch.float32, device=dev)
        if pad_pose is None:
            pad_pose = torch.empty((self.n, self.n_pads, 8), dtype=torch.float32, device=dev)
        if slip is None:
            slip = torch.empty((self.n, self.n_pads, 4), dtype=torch.float32, device=dev)
        self._call("sim_read_observation", _ptr(q), _ptr(pad_pose), _ptr(slip))
        return q, pad_pose, slip

    def sim_set_hand(self, q, qd=None):
        _check(q, torch.float32, (self.n, self.n_joints), "q")
        _check(qd, torch.float32, (self.n, self.n_joints), "qd")
        self._call("sim_set_hand", _ptr(q), _ptr(qd))

    def sim_get_hand(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        q = torch.empty((self.n, self.n_joints), dtype=torch.float32, device=dev)
        qd = torch.empty_like(q)
        self._call("sim_get_hand", _ptr(q), _ptr(qd))
        return q, qd

    def cost_eval_full(self, q, pad_pose, forces, slip, cost_mean=None, argmin=None, est_pose=None):
        """PD hand: the full ten-term cost against the ground truth's observation
        (q [D], pad_pose [P, 8], forces [P, 3], slip [P, 4])."""
        _check(q, torch.float32, (self.n_joints,), "q")
        _check(pad_pose, torch.float32, (self.n_pads, 8), "pad_pose")
        _check(forces, torch.float32, (self.n_pads, 3), "forces")
        _check(slip, torch.float32, (self.n_pads, 4), "slip")
        _check(cost_mean, torch.float64, (self.n,), "cost_mean")
        _check(argmin, torch.int32, (1,), "argmin")
        _check(est_pose, torch.float32, (8,), "est_pose")
        self._call("cost_eval_full", _ptr(q), _ptr(pad_pose), _ptr(forces), _ptr(slip), _ptr(cost_mean),
                   _ptr(argmin), _ptr(est_pose))

    def sim_step_frames_full(self, frame0: int, q, pad_pose, forces, slip):
        """PD hand: T frames in one step launch, each then scored with the full
        cost against the truth's observation (q [T, D], pad_pose [T, P, 8], forces [T, P, 3],
        slip [T, P, 4]); follow with sim_frames_argmin."""
        T = forces.shape[0]
        _check(q, torch.float32, (T, self.n_joints), "q")
        _check(pad_pose, torch.float32, (T, self.n_pads, 8), "pad_pose")
        _check(forces, torch.float32, (T, self.n_pads, 3), "forces")
        _check(slip, torch.float32, (T, self.n_pads, 4), "slip")
        self._call("sim_step_frames_full", frame0, T, _ptr(q), _ptr(pad_pose), _ptr(forces), _ptr(slip))

    def sim_step_track(self, frame: int, obs, cost_mean=None, argmin=None, est_pose=None):
        _check(obs, torch.float32, (self.n_pads, 3), "obs")
        _check(cost_mean, torch.float64, (self.n,), "cost_mean")
        _check(argmin, torch.int32, (1,), "argmin")
        _check(est_pose, torch.float32, (8,), "est_pose")
        self._call("sim_step_track", frame, _ptr(obs), _ptr(cost_mean), _ptr(argmin), _ptr(est_pose))

    def sim_step_frames(self, frame0: int, obs):
        T = obs.shape[0]
        _check(obs, torch.float32, (T, self.n_pads, 3), "obs")
        self._call("sim_step_frames", frame0, T, _ptr(obs))

    def sim_frames_argmin(self, est_pose=None, argmin=None):
        self._call("sim_frames_argmin", _ptr(est_pose), _ptr(argmin))

    def sim_track_window(self, frame0: int, obs, opt, update_index: int, est_pose=None, argmin=None):
        T = obs.shape[0]
        _check(obs, torch.float32, (T, self.n_pads, 3), "obs")
        _check(est_pose, torch.float32, (T, 8), "est_pose")
        _check(argmin, torch.int32, (T,), "argmin")
        self._call("sim_track_window", frame0, T, _ptr(obs), C.byref(_opt(opt)), C.c_uint32(update_index),
                   _ptr(est_pose), _ptr(argmin))

    def optimizer_update(self, opt, update_index: int, argmin=None, parent=None):
        oc = _opt(opt)
        _check(argmin, torch.int32, (1,), "argmin")
        _check(parent, torch.int32, (self.n,), "parent")
        self._call("optimizer_update", C.byref(oc), C.c_uint32(update_index), _ptr(argmin), _ptr(parent))

    def sim_work_counters(self, reset: bool = False):
        out = (C.c_uint64 * 6)()
        self._call("sim_work_counters", out, 1 if reset else 0)
        return {"pairs": out[0], "contacts": out[1], "contact_iters": out[2], "env_substeps": out[3],
                "env_iters": out[4], "cluster_tests": out[5]}

    def sim_sync(self):
        self._call("sim_sync")

    def sim_autotune(self, frame0: int, n_frames: int):
        chosen = (C.c_int32 * 2)()
        ms = (C.c_float * 16)(*([float("nan")] * 16))
        self._call("sim_autotune", frame0, n_frames, chosen, ms)
        variants = step_variants()
        return (chosen[0], chosen[1]), {v: ms[k] for k, v in enumerate(variants) if k < 16}

    def sim_set_variant(self, threads_per_env: int, contacts_per_thread: int):
        self._call("sim_set_variant", threads_per_env, contacts_per_thread)

    def sim_adjoint(self, frame0: int, obs, envs=None, checkpoint_every: int = 10, beta: float = 1e3,
                    width: float = 1e-3, cost=None, grad=None, grad_quat=None, want_quat: bool = False):
        """Horizon cost and its gradient for each selected environment
        (horizon = obs.shape[0] frames from frame0). Returns (cost float64[n],
        grad float32[n][8] = d/d(x, y, z, rx, ry, rz, m, mu), grad_quat
        float32[n][4] or None)."""
        H = obs.shape[0]
        _check(obs, torch.float32, (H, self.n_pads, 3), "obs")
        n = self.n if envs is None else envs.shape[0]
        _check(envs, torch.int32, (n,), "envs")
        dev = torch.device("cuda", torch.cuda.current_device())
        if cost is None:
            cost = torch.empty((n,), dtype=torch.float64, device=dev)
        if grad is None:
            grad = torch.empty((n, 8), dtype=torch.float32, device=dev)
        if grad_quat is None and want_quat:
            grad_quat = torch.empty((n, 4), dtype=torch.float32, device=dev)
        _check(cost, torch.float64, (n,), "cost")
        _check(grad, torch.float32, (n, 8), "grad")
        _check(grad_quat, torch.float32, (n, 4), "grad_quat")
        self._call("sim_adjoint", frame0, H, checkpoint_every, _ptr(obs), _ptr(envs), n, C.c_float(beta),
                   C.c_float(width), _ptr(cost), _ptr(grad), _ptr(grad_quat))
        return cost, grad, grad_quat

    def sim_set_adjoint_memory(self, nbytes: int):
        self._call("sim_set_adjoint_memory", C.c_uint64(nbytes))

    def sim_set_adjoint_variant(self, warps_per_env: int = 0, contacts_per_thread: int = 0):
        """The adjoint kernel's shape; (0, 0) = automatic."""
        self._call("sim_set_adjoint_variant", warps_per_env, contacts_per_thread)

    def sim_mark_window(self):
        self._call("sim_mark_window")

    def sim_refine_elites(self, frame0: int, obs, opt, steps: int = 3, step_scale: float = 0.5,
                          beta: float = 1e3, width: float = 1e-3, report: bool = False, detail: bool = False):
        """Refine the window's elites (see include/inhand.h). With report=True
        returns (elites int32[k], cost_before float64[k], cost_after float64[k]);
        with detail=True also (accepted int64[k] decision bits, start_pose
        float32[k][8], start_params float32[k][2])."""
        T = obs.shape[0]
        _check(obs, torch.float32, (T, self.n_pads, 3), "obs")
        out = (None, None, None)
        more = (None, None, None)
        if report or detail:
            k = max(1, min(self.n, int(np.floor(np.float64(np.float32(opt.elite_frac)) * self.n))))
            dev = torch.device("cuda", torch.cuda.current_device())
            out = (torch.empty(k, dtype=torch.int32, device=dev), torch.empty(k, dtype=torch.float64, device=dev),
                   torch.empty(k, dtype=torch.float64, device=dev))
            if detail:
                more = (torch.empty(k, dtype=torch.int64, device=dev),
                        torch.empty((k, 8), dtype=torch.float32, device=dev),
                        torch.empty((k, 2), dtype=torch.float32, device=dev))
        self._call("sim_refine_elites", frame0, T, _ptr(obs), C.byref(_opt(opt)), steps, C.c_float(step_scale),
                   C.c_float(beta), C.c_float(width), *(_ptr(t) for t in out), *(_ptr(t) for t in more))
        if detail:
            return out + more
        return out if report else None


def fp32_peak(iters: int = 2048, reps: int = 40):
    """Measured FP32 FMA throughput of the current device (ih_fp32_peak):
    (TFLOP/s, ms per launch, SM count)."""
    tf, ms, sms = C.c_double(), C.c_double(), C.c_int32()
    code = lib().ih_fp32_peak(iters, reps, _stream(), C.byref(tf), C.byref(ms), C.byref(sms))
    if code != IH_OK:
        raise InhandError("ih_fp32_peak", code, "FP32 peak probe failed")
    return tf.value, ms.value, sms.value


def step_variants():
    """Supported step-kernel shapes (threads per env, contacts per thread)."""
    out = (C.c_int32 * 64)()
    n = lib().sim_step_variants(out, 32)
    return [(out[2 * k], out[2 * k + 1]) for k in range(n)]


def make_sim(workload, n_envs: int | None = None, max_frames: int | None = None, seed: int | None = None) -> Sim:
    """A handle for a workload from paper_2002_12160_gb300.workloads."""
    n = workload.n_envs if n_envs is None else n_envs
    mf = (workload.frames if max_frames is None else max_frames)
    return Sim(workload.scene, workload.sim, n, mf, workload.seed if seed is None else seed)
