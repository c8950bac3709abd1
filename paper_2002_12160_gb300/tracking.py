"""Algorithm 1 (sample-based optimization for in-hand pose tracking) on the GPU.

The tracker holds two handles of the C ABI: the N tracking environments and
one ground-truth environment (its true initial pose, hidden mass and friction) whose
pad forces stand in for the real robot's observations o_t^(gt) (Sec. IV-A
uses a simulated ground truth the same way). A window is T frames of
"step all environments, score them, take i* = argmin C_i", followed by the
optimizer update. All of it runs in libinhand.so's kernels; this module only
orders the calls and moves buffers.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import inhand, workloads as W


class Tracker:
    def __init__(self, wl: W.Workload, seed: int | None = None, n_envs: int | None = None,
                 gt_sim: W.SimConfig | None = None):
        """`gt_sim`: the ground truth's solver settings when they differ from the
        tracking environments' (e.g. a converged solve behind a cheaper one)."""
        self.wl = wl
        self.T = wl.opt.window
        self.seed = wl.seed if seed is None else seed
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.sim = inhand.make_sim(wl, n_envs=n_envs, max_frames=wl.frames, seed=self.seed)
        gt_wl = wl if gt_sim is None else dataclasses.replace(wl, sim=gt_sim)
        self.gt = inhand.make_sim(gt_wl, n_envs=1, max_frames=wl.frames, seed=self.seed + 1)
        self.n = self.sim.n
        P = wl.scene.n_pads
        self.obs = torch.zeros((wl.frames, P, 3), dtype=torch.float32, device=self.dev)
        self.gt_pose = torch.zeros((wl.frames, 8), dtype=torch.float32, device=self.dev)
        self.argmin = torch.zeros((wl.frames,), dtype=torch.int32, device=self.dev)
        self.est = torch.zeros((wl.frames, 8), dtype=torch.float32, device=self.dev)
        self.pd = self.sim.pd
        if self.pd:   # the ground truth's full observation of every frame
            D = wl.scene.n_joints
            self.obs_q = torch.zeros((wl.frames, D), dtype=torch.float32, device=self.dev)
            self.obs_pp = torch.zeros((wl.frames, P, 8), dtype=torch.float32, device=self.dev)
            self.obs_slip = torch.zeros((wl.frames, P, 4), dtype=torch.float32, device=self.dev)

    def prepare(self):
        """Commands for every frame, the ground-truth run, and the initial samples."""
        wl = self.wl
        q = torch.from_numpy(wl.q_traj).contiguous().to(self.dev)
        self.sim.sim_set_commands(0, q)
        self.gt.sim_set_commands(0, q)
        gt0 = wl.gt_pose if wl.gt_pose is not None else wl.nominal_pose
        pose = torch.from_numpy(gt0[None].copy()).to(self.dev)
        vel = torch.zeros((1, 8), dtype=torch.float32, device=self.dev)
        par = torch.tensor([wl.theta_gt], dtype=torch.float32, device=self.dev)
        self.gt.sim_set_state(pose, vel, par)
        f_buf = torch.empty((1, wl.scene.n_pads, 3), dtype=torch.float32, device=self.dev)
        st_buf = torch.empty((1,), dtype=torch.int32, device=self.dev)
        for f in range(wl.frames):
            self.gt.sim_step(f, 1)
            self.gt.sim_read_sensors(f_buf, st_buf)
            self.obs[f].copy_(f_buf[0])
            self.gt_pose[f].copy_(self.gt.sim_get_state()[0][0])
            if self.pd:
                q, pp, slip = self.gt.sim_read_observation()
                self.obs_q[f].copy_(q[0])
                self.obs_pp[f].copy_(pp[0])
                self.obs_slip[f].copy_(slip[0])
        self.sim.sim_sample_initial(wl.nominal_pose, wl.init.sigma_p, wl.init.sigma_r,
                                    wl.init.m_range, wl.init.mu_range)
        n = self.n
        if len(wl.scene.shapes) > 1 or not np.all(wl.iters[:n] == wl.sim.iters):
            # uneven batch: each environment's own shape (resting at its own height) and
            # solver iteration count
            dz = np.array([W.nominal_pose_for(wl.scene, k)[2] - wl.nominal_pose[2]
                           for k in range(len(wl.scene.shapes))], np.float32)
            sid = torch.from_numpy(wl.shape_id[:n].astype(np.int32)).to(self.dev)
            its = torch.from_numpy(wl.iters[:n].astype(np.int32)).to(self.dev)
            pose, vel, par, _ = self.sim.sim_get_state()
            pose[:, 2] += torch.from_numpy(dz).to(self.dev)[sid.long()]
            self.sim.sim_set_state(pose, vel, par, sid, its)
        torch.cuda.synchronize()

    def window(self, w: int):
        """Frames [wT, (w+1)T) -- step, score, argmin each frame -- then the
        optimizer update, replayed from one captured CUDA graph."""
        T = self.T
        f0 = w * T
        self.sim.sim_track_window(f0, self.obs[f0:f0 + T], self.wl.opt, w, self.est[f0:f0 + T],
                                  self.argmin[f0:f0 + T])

    # The PD window's T frames in one step launch (then scored by two launches)
    # is faster while the environments fit in about one wave (cylinder,
    # N = 1024: 0.97 against 1.77 ms per window); with several waves per-frame
    # step and cost launches win (N = 8192: 6.27 against 6.48 ms).
    PD_FUSED_MAX_N = 4096

    def window_pd(self, w: int):
        """A window with the PD-driven hand: its T frames in one step launch,
        each then scored with the full ten-term cost against the ground truth's
        observation, every frame's argmin and estimate, then the optimizer
        update (per-frame launches above PD_FUSED_MAX_N environments)."""
        if self.n > self.PD_FUSED_MAX_N:
            return self.window_pd_unfused(w)
        T = self.T
        f0 = w * T
        self.sim.sim_step_frames_full(f0, self.obs_q[f0:f0 + T], self.obs_pp[f0:f0 + T], self.obs[f0:f0 + T],
                                      self.obs_slip[f0:f0 + T])
        self.sim.sim_frames_argmin(self.est[f0:f0 + T], self.argmin[f0:f0 + T])
        self.sim.optimizer_update(self.wl.opt, w)

    def window_pd_unfused(self, w: int):
        """The same window as per-frame calls: one step launch and one full-cost
        launch per frame, then the optimizer update."""
        T = self.T
        for k in range(T):
            f = w * T + k
            self.sim.sim_step(f, 1)
            self.sim.cost_eval_full(self.obs_q[f], self.obs_pp[f], self.obs[f], self.obs_slip[f], None,
                                    self.argmin[f:f + 1], self.est[f])
        self.sim.optimizer_update(self.wl.opt, w)

    def window_eye(self, w: int):
        """The identity baseline (EYE, Sec. IV): the window's frames stepped,
        scored and argmin'd, with no optimizer update -- the simulations keep
        their initial samples and the window mean runs from the start."""
        T = self.T
        f0 = w * T
        self.sim.sim_step_frames(f0, self.obs[f0:f0 + T])
        self.sim.sim_frames_argmin(self.est[f0:f0 + T], self.argmin[f0:f0 + T])

    def prepare_open_loop(self):
        """The open-loop baseline (OLP, Sec. IV): one simulation from the
        nominal pose with the parameter ranges' midpoints; run it with
        window_eye (its estimate is its own pose)."""
        assert self.n == 1, "open loop tracks with one simulation"
        wl = self.wl
        pose = torch.from_numpy(wl.nominal_pose[None].copy()).to(self.dev)
        vel = torch.zeros((1, 8), dtype=torch.float32, device=self.dev)
        par = torch.tensor([[0.5 * (wl.init.m_range[0] + wl.init.m_range[1]),
                             0.5 * (wl.init.mu_range[0] + wl.init.mu_range[1])]], dtype=torch.float32,
                           device=self.dev)
        self.sim.sim_set_state(pose, vel, par)
        torch.cuda.synchronize()

    def window_unfused(self, w: int, step_events=None):
        """The same window as separate calls -- the T-frame step launch (bracketed
        by `step_events` when given), the per-frame argmin, the optimizer -- for
        timing the step kernel alone."""
        T = self.T
        f0 = w * T
        if step_events is not None:
            step_events[0].record()
        self.sim.sim_step_frames(f0, self.obs[f0:f0 + T])
        if step_events is not None:
            step_events[1].record()
        self.sim.sim_frames_argmin(self.est[f0:f0 + T], self.argmin[f0:f0 + T])
        self.sim.optimizer_update(self.wl.opt, w)

    def window_refined(self, w: int, steps: int = 3, step_scale: float = 0.5, report: bool = False):
        """The window with a gradient refinement of its elites before the
        optimizer update: mark the window start, step and score its T frames,
        refine the elites' window-start states along the adjoint gradient of
        the window's cost, then resample."""
        T = self.T
        f0 = w * T
        self.sim.sim_mark_window()
        # the window's T frames in one step launch, then each frame's argmin
        # (the same results as T per-frame launches, bit for bit)
        self.sim.sim_step_frames(f0, self.obs[f0:f0 + T])
        self.sim.sim_frames_argmin(self.est[f0:f0 + T], self.argmin[f0:f0 + T])
        rep = self.sim.sim_refine_elites(f0, self.obs[f0:f0 + T], self.wl.opt, steps, step_scale,
                                         report=report)
        self.sim.optimizer_update(self.wl.opt, w)
        return rep

    def e2e_windows(self, w0: int, count: int):
        """Windows driven through the public API from pinned host buffers: per
        window the commands and observations go host -> device and the
        estimates and argmins come back device -> host, all on the handle's
        stream. Pipelined: the host enqueues every window's copies and calls
        without waiting, and synchronises once after the last window's
        read-back (the timed region spans all of them). Also reported: the same
        windows with the host waiting for each window's read-back."""
        T, D, P = self.T, self.wl.scene.n_joints, self.wl.scene.n_pads
        n_in, n_out = (T + 1) * D + T * P * 3, T * 8 + T
        frames = self.wl.frames
        # each window's inputs (commands of its T + 1 frame boundaries, then the
        # observations of its T frames) packed in one pinned host block, and its
        # outputs (estimates, then argmins) in one device block: one copy each way
        in_host = torch.empty((frames // T, n_in), dtype=torch.float32).pin_memory()
        q_all = torch.from_numpy(self.wl.q_traj)
        obs_all = self.obs.cpu()
        for w in range(w0, w0 + count):
            f0 = w * T
            in_host[w, :(T + 1) * D] = q_all[f0:f0 + T + 1].reshape(-1)
            in_host[w, (T + 1) * D:] = obs_all[f0:f0 + T].reshape(-1)
        out_host = torch.empty((count, n_out), dtype=torch.float32).pin_memory()
        in_dev = torch.empty((n_in,), dtype=torch.float32, device=self.dev)
        out_dev = torch.empty((n_out,), dtype=torch.float32, device=self.dev)
        q_dev = in_dev[:(T + 1) * D].view(T + 1, D)
        obs_dev = in_dev[(T + 1) * D:].view(T, P, 3)
        est_dev = out_dev[:T * 8].view(T, 8)
        am_dev = out_dev[T * 8:].view(torch.int32)

        def window(i, w):
            f0 = w * T
            in_dev.copy_(in_host[w], non_blocking=True)
            self.sim.sim_set_commands(f0, q_dev)
            self.sim.sim_track_window(f0, obs_dev, self.wl.opt, w, est_dev, am_dev)
            out_host[i].copy_(out_dev, non_blocking=True)

        half = count // 2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, w in enumerate(range(w0, w0 + half)):
            window(i, w)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / half
        sync_times = []
        for i, w in enumerate(range(w0 + half, w0 + count)):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            window(half + i, w)
            torch.cuda.synchronize()
            sync_times.append(time.perf_counter() - t1)
        ms_sync = 1e3 * sum(sync_times) / len(sync_times)
        for i, w in enumerate(range(w0, w0 + count)):   # the estimates as the tracker keeps them
            f0 = w * T
            self.est[f0:f0 + T].copy_(out_host[i, :T * 8].view(T, 8))
            self.argmin[f0:f0 + T].copy_(out_host[i, T * 8:].view(torch.int32))
        return {"value": self.n * T / (ms / 1e3), "unit": "env-steps/s", "ms_per_step": ms,
                "h2d_bytes_per_step": n_in * 4, "d2h_bytes_per_step": n_out * 4, "windows": half, "pipelined": True,
                "host_waits_each_window": {"value": self.n * T / (ms_sync / 1e3), "ms_per_step": ms_sync,
                                           "windows": count - half}}

    def add_mm(self, frames: int | None = None) -> float:
        """Mean ADD (mm) of the argmin estimate against the ground truth over the
        scored frames, on the object's sphere centres (evaluation, Sec. IV)."""
        est = self.est.cpu().numpy().astype(np.float64)
        gt = self.gt_pose.cpu().numpy().astype(np.float64)
        used = frames if frames is not None else int((np.abs(est).sum(1) > 0).sum())
        pts = self.wl.scene.shapes[0][:, :3]
        pts = pts - pts.mean(0)   # the pose is the centroid's

        def world(p):
            w, x, y, z = p[4:]
            R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                          [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                          [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
            return p[:3] + pts @ R.T

        errs = [np.linalg.norm(world(est[f]) - world(gt[f]), axis=1).mean() for f in range(used)
                if np.abs(est[f]).sum() > 0]
        return 1e3 * float(np.mean(errs)) if errs else float("nan")

    def close(self):
        self.sim.close()
        self.gt.close()
