"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and hand its FP32 state, converted exactly to FP64, to the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2002_12160_gb300 import workloads as W

torch = pytest.importorskip("torch")

# tolerances of the FP32 path against the FP64 oracle, one frame from the same state
POS_TOL = 1e-5      # m
ROT_TOL = 1e-5      # rad
FORCE_REL = 1e-3    # relative pad force ...
FORCE_ABS = 1e-4    # ... with an absolute floor (N)
FRAGILE = 1e-6      # m: contact-set or pad membership within this of a threshold
# velocities after the frame: the pose tolerances over the longest substep
# (1/60 s), the velocity error that would move the pose by that much in one
# substep of the symplectic update x += h v, R <- exp(h w) R
VEL_TOL = 6e-4      # m/s
ANGVEL_TOL = 6e-4   # rad/s
MIN_OK_FRAC = 0.85  # share of environments clear of every branch threshold


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch.device("cuda", 0)


def scene32(scene: W.Scene) -> W.Scene:
    """The scene as the GPU sees it (FP32), widened exactly to FP64 for the oracle."""
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return W.Scene(shapes=[f(s) for s in scene.shapes], palm_half=f(scene.palm_half),
                   finger_root=f(scene.finger_root), link_len=float(np.float32(scene.link_len)),
                   link_rad=float(np.float32(scene.link_rad)), pad_link=scene.pad_link,
                   pad_s0=f(scene.pad_s0), pad_s1=f(scene.pad_s1))


def sim32(sim: W.SimConfig) -> W.SimConfig:
    import dataclasses
    c = dataclasses.replace(sim)
    for name in ["frame_dt", "margin", "beta", "slop", "vmax", "tau", "w_force", "w_contact", "escape_radius"]:
        setattr(c, name, float(np.float32(getattr(c, name))))
    c.gravity = tuple(float(np.float32(g)) for g in c.gravity)
    for name in ["kp", "kd", "armature", "v_slip", "w_slip"]:
        setattr(c, name, float(np.float32(getattr(c, name))))
    c.w_full = tuple(float(np.float32(w)) for w in c.w_full)
    return c


def oracle_state(gpu_state, shape=None, iters=None):
    pose, vel, params, status = (t.detach().cpu().numpy() for t in gpu_state)
    return O.State(O.pose8_to7(pose), O.vel8_to6(vel), params.astype(np.float64), shape, iters, status)


def rot_angle(q7a, q7b):
    qa, qb = q7a[..., 3:7], q7b[..., 3:7]
    d = np.abs(np.sum(qa * qb, axis=-1)) / (np.linalg.norm(qa, axis=-1) * np.linalg.norm(qb, axis=-1))
    return 2 * np.arccos(np.clip(d, -1, 1))


def place_shapes(wl, pose_t, shape_ids):
    """Move each env's sampled offset onto the resting height of its own shape."""
    base = wl.nominal_pose
    for i, sid in enumerate(shape_ids):
        nom = W.nominal_pose_for(wl.scene, int(sid))
        pose_t[i, 2] += float(nom[2] - base[2])
    return pose_t


def start(wl, n=None, frames=None):
    """Create the handle, upload the commands and sample the initial state on the GPU."""
    d = dev()
    from paper_2002_12160_gb300 import inhand
    sim = inhand.make_sim(wl, n_envs=n, max_frames=frames)
    sim.sim_set_commands(0, torch.from_numpy(wl.q_traj[: (frames or wl.frames) + 1]).contiguous().to(d))
    sim.sim_sample_initial(wl.nominal_pose, wl.init.sigma_p, wl.init.sigma_r, wl.init.m_range, wl.init.mu_range)
    nn = sim.n
    if len(wl.scene.shapes) > 1 or not np.all(wl.iters[:nn] == wl.sim.iters):
        pose, vel, params, _ = sim.sim_get_state()
        sid = torch.from_numpy(wl.shape_id[:nn].astype(np.int32)).to(d)
        its = torch.from_numpy(wl.iters[:nn].astype(np.int32)).to(d)
        pose = place_shapes(wl, pose.cpu(), wl.shape_id[:nn]).to(d)
        sim.sim_set_state(pose.contiguous(), vel, params, sid, its)
    return sim


def oracle_cache(sim, st):
    """Put the GPU's warm-start cache, widened exactly to FP64, onto an oracle State."""
    n, lam, ids = (t.cpu().numpy() for t in sim.sim_get_warm_cache())
    st.cache_n = n.astype(np.int32).copy()
    st.cache_id = ids.astype(np.int32).copy()
    st.cache_lam = lam.astype(np.float64).copy()
    return st


def compare_frame(wl, sim, frame, envs=None):
    """Step the GPU one frame and the oracle one frame from the GPU's state; return a report.
    A warm-started handle hands its impulse cache to the oracle too, and the
    report carries both caches after the frame."""
    nn = sim.n
    shape = wl.shape_id[:nn].astype(np.int32)
    iters = wl.iters[:nn].astype(np.int32)
    pre = [t.clone() for t in sim.sim_get_state()]
    st = oracle_state(pre, shape, iters)
    warm = getattr(sim, "warm_start", False)
    if warm:
        oracle_cache(sim, st)
    if envs is not None:
        st = st.subset(envs)
    osc = O.OracleScene(scene32(wl.scene))
    f_or, diag = O.step(osc, sim32(wl.sim), st, wl.q_traj, frame, 1)
    sim.sim_work_counters(reset=True)
    sim.sim_step(frame, 1)
    work = sim.sim_work_counters()
    forces, status = sim.sim_read_sensors()
    g = oracle_state(sim.sim_get_state())
    forces = forces.cpu().numpy().astype(np.float64)
    status = status.cpu().numpy()
    if envs is not None:
        g = g.subset(envs)
        forces = forces[envs]
        status = status[envs]
    fragile = (diag[:, 2] < FRAGILE) | (diag[:, 3] < FRAGILE) | (diag[:, 4] < FRAGILE)
    ok = ~fragile
    pos_err = np.linalg.norm(g.pose[:, :3] - st.pose[:, :3], axis=1)
    rot_err = rot_angle(g.pose, st.pose)
    fe = np.linalg.norm(forces - f_or, axis=2)
    fmag = np.linalg.norm(f_or, axis=2)
    f_bad = fe > FORCE_REL * fmag + FORCE_ABS
    rep = {"ok": ok, "pos_err": pos_err, "rot_err": rot_err, "force_bad": f_bad, "force_err": fe,
           "status_gpu": status, "status_or": st.status, "contacts_or": diag[:, 0].sum(),
           "work": work, "diag": diag,
           "vel_err": np.linalg.norm(g.vel[:, :3] - st.vel[:, :3], axis=1),
           "angvel_err": np.linalg.norm(g.vel[:, 3:] - st.vel[:, 3:], axis=1)}
    if not warm:
        # the contacts the GPU generates for the environments clear of every
        # threshold (and not diverged before the frame), counted by the step
        # kernel on a handle holding just those environments' start states
        pre_status = oracle_state(pre).status[envs if envs is not None else slice(None)]
        sel = np.nonzero(ok & (pre_status == 0) & ((st.status & O.OVERFLOW) == 0))[0]
        full = sel if envs is None else np.asarray(envs)[sel]
        if len(full):
            rep["contacts_sub"] = (gpu_contacts(wl, pre, frame, full), int(diag[sel, 0].sum()), len(full))
    if warm:
        n, lam, ids = (t.cpu().numpy() for t in sim.sim_get_warm_cache())
        if envs is not None:
            n, lam, ids = n[envs], lam[envs], ids[envs]
        rep["cache_gpu"] = (n, ids, lam.astype(np.float64))
        rep["cache_or"] = (st.cache_n, st.cache_id, st.cache_lam)
        rep["h"] = wl.sim.frame_dt / wl.sim.substeps
    return rep


def gpu_contacts(wl, pre, frame, idx):
    """Contacts the GPU step generates in frame `frame` for environments idx
    from their start states `pre` (pose, vel, params, status tensors): the step
    kernel's contact counter on a handle holding just those environments."""
    from paper_2002_12160_gb300 import inhand
    d = dev()
    ix = torch.from_numpy(np.asarray(idx, np.int64)).to(d)
    sub = inhand.make_sim(wl, n_envs=len(idx), max_frames=frame + 2)
    sub.sim_set_commands(0, torch.from_numpy(wl.q_traj[: frame + 2]).contiguous().to(d))
    shape = torch.from_numpy(wl.shape_id[np.asarray(idx)].astype(np.int32)).to(d)
    iters = torch.from_numpy(wl.iters[np.asarray(idx)].astype(np.int32)).to(d)
    sub.sim_set_state(pre[0][ix].contiguous(), pre[1][ix].contiguous(), pre[2][ix].contiguous(), shape, iters)
    sub.sim_work_counters(reset=True)
    sub.sim_step(frame, 1)
    n = sub.sim_work_counters()["contacts"]
    sub.close()
    return n


def assert_report(rep, min_ok_frac=MIN_OK_FRAC):
    ok = rep["ok"]
    assert ok.mean() >= min_ok_frac, f"too many envs near a branch threshold: {(~ok).sum()} of {len(ok)}"
    np.testing.assert_array_equal(rep["status_gpu"][ok], rep["status_or"][ok])
    assert rep["pos_err"][ok].max(initial=0) < POS_TOL, rep["pos_err"][ok].max()
    assert rep["rot_err"][ok].max(initial=0) < ROT_TOL, rep["rot_err"][ok].max()
    assert not rep["force_bad"][ok].any(), rep["force_err"][ok].max()
    assert rep["vel_err"][ok].max(initial=0) < VEL_TOL, rep["vel_err"][ok].max()
    assert rep["angvel_err"][ok].max(initial=0) < ANGVEL_TOL, rep["angvel_err"][ok].max()
    if "contacts_sub" in rep:
        # the culled GPU enumeration finds exactly the oracle's brute-force
        # contact set on every environment clear of a threshold
        g, o, k = rep["contacts_sub"]
        assert g == o, f"contacts over {k} envs: GPU {g}, oracle {o}"
    if "cache_gpu" in rep:
        # the caches hold the same contact pairs (the GPU's in (link, sphere)
        # order, the oracle's in its enumeration order) with the same final
        # impulses (compared as forces lambda / h, pad-force tolerance)
        (ng, ig, lg), (no, io, lo) = rep["cache_gpu"], rep["cache_or"]
        np.testing.assert_array_equal(ng[ok], no[ok])
        for i in np.nonzero(ok)[0]:
            k = int(no[i])
            sg, so = np.argsort(ig[i, :k]), np.argsort(io[i, :k])
            np.testing.assert_array_equal(ig[i, :k][sg], io[i, :k][so])
            assert np.all(np.diff(ig[i, :k]) > 0)
            fg, fo = lg[i, :k][sg] / rep["h"], lo[i, :k][so] / rep["h"]
            err = np.linalg.norm(fg - fo, axis=1)
            assert np.all(err <= FORCE_REL * np.linalg.norm(fo, axis=1) + FORCE_ABS), (i, err.max())
