"""The PD-driven hand on the GPU against the oracle (through the C ABI).

- one frame from the GPU's own state (object and joints, widened exactly to
  FP64) on the box and cylinder trajectories and the uneven batch: object
  pose, pad forces, joint angles and velocities, pad poses, status bits,
  slip flags and directions (pads whose slip speed or spin sits within 2 %
  of its threshold, and envs at a contact or pad boundary, are excluded and
  counted, as FP32 and FP64 may decide them differently);
- the full cost of the GPU's observation against one environment's, in FP64,
  equals the oracle's on the same (widened) arrays to 1e-12 relative, with
  the same argmin;
- the free joints settle on a held command exactly (no contact);
- an optimizer update (elite and REPS) hands every replaced environment its
  parent's joints;
- calls that the PD hand does not support are refused.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2002_12160_gb300 import workloads as W

from gpu_common import (FORCE_ABS, FORCE_REL, FRAGILE, POS_TOL, ROT_TOL, dev, oracle_state, rot_angle, scene32,
                        sim32, start, torch)

pytestmark = pytest.mark.gpu


def _pd(name, n, frames, **kw):
    wl = W.make_workload(name, n_envs=n, frames=frames)
    wl.sim = dataclasses.replace(wl.sim, hand="pd", **kw)
    return wl


def _hand_state(sim, shape, iters):
    st = oracle_state(sim.sim_get_state(), shape, iters)
    q, qd = (t.cpu().numpy().astype(np.float64) for t in sim.sim_get_hand())
    st.qj, st.qdj = q.copy(), qd.copy()
    return st


def _gpu_obs(sim):
    forces, status = sim.sim_read_sensors()
    q, pp, slip = sim.sim_read_observation()
    pp = pp.cpu().numpy()
    slip = slip.cpu().numpy()
    obs = O.Obs(q.cpu().numpy().astype(np.float64),
                np.concatenate([pp[..., :3], pp[..., 4:8]], axis=-1).astype(np.float64),
                forces.cpu().numpy().astype(np.float64), slip[..., :2].astype(np.float64),
                slip[..., 2].copy().view(np.int32))
    return obs, status.cpu().numpy()


def compare_pd_frame(wl, sim, frame):
    n = sim.n
    shape = wl.shape_id[:n].astype(np.int32)
    iters = wl.iters[:n].astype(np.int32)
    st = _hand_state(sim, shape, iters)
    osc = O.OracleScene(scene32(wl.scene))
    ob, diag = O.step_pd(osc, sim32(wl.sim), st, wl.q_traj, frame, 1)
    sim.sim_step(frame, 1)
    g = _hand_state(sim, shape, iters)
    go, status = _gpu_obs(sim)
    ok = ~((diag[:, 2] < FRAGILE) | (diag[:, 3] < FRAGILE) | (diag[:, 4] < FRAGILE))
    assert ok.mean() >= 0.75, f"too many envs near a branch threshold: {(~ok).sum()}"
    np.testing.assert_array_equal(status[ok], st.status[ok])
    assert np.linalg.norm(g.pose[ok, :3] - st.pose[ok, :3], axis=1).max(initial=0) < POS_TOL
    assert rot_angle(g.pose[ok], st.pose[ok]).max(initial=0) < ROT_TOL
    fe = np.linalg.norm(go.forces - ob.forces, axis=2)
    assert not (fe > FORCE_REL * np.linalg.norm(ob.forces, axis=2) + FORCE_ABS)[ok].any(), fe[ok].max()
    np.testing.assert_allclose(g.qj[ok], st.qj[ok], atol=1e-5)
    np.testing.assert_allclose(g.qdj[ok], st.qdj[ok], atol=2e-4, rtol=1e-3)
    np.testing.assert_allclose(go.pad_pose[ok][..., :3], ob.pad_pose[ok][..., :3], atol=1e-5)
    assert rot_angle(go.pad_pose[ok].reshape(-1, 7), ob.pad_pose[ok].reshape(-1, 7)).max(initial=0) < ROT_TOL
    # slip: flags where the speed and spin are clear of their thresholds
    sim_c = wl.sim
    vt, spin = ob.slip_mag[..., 0], ob.slip_mag[..., 1]
    clear = (np.abs(vt - sim_c.v_slip) > 0.02 * sim_c.v_slip) & (np.abs(np.abs(spin) - sim_c.w_slip) > 0.02 * sim_c.w_slip)
    clear &= ok[:, None]
    np.testing.assert_array_equal(go.flags[clear], ob.flags[clear])
    fast = clear & (vt > 2 * sim_c.v_slip)
    np.testing.assert_allclose(go.slip_d[fast], ob.slip_d[fast], atol=5e-3)
    return {"ok": ok, "contacts": diag[:, 0].sum(), "slipping": int((ob.flags[clear] & 1).sum()),
            "spinning": int((ob.flags[clear] & 2).sum()), "clear": int(clear.sum())}


@pytest.mark.parametrize("name,n,frames,check", [
    ("tracking_box27", 16, 30, [2, 15, 29]),
    ("tracking_cyl64", 61, 24, [3, 12, 23]),
    ("uneven_mixed", 67, 12, [4, 11]),
])
def test_pd_one_frame_parity(name, n, frames, check):
    wl = _pd(name, n, frames)
    sim = start(wl, n=n, frames=frames)
    assert sim.pd
    contacts, slipping = 0, 0
    for f in range(frames):
        if f in check:
            rep = compare_pd_frame(wl, sim, f)
            contacts += rep["contacts"]
            slipping += rep["slipping"] + rep["spinning"]
        else:
            sim.sim_step(f, 1)
    assert contacts > 0 and slipping > 0


def test_pd_full_cost_matches_oracle():
    n = 200
    wl = _pd("tracking_cyl64", n, 8)
    sim = start(wl, n=n, frames=8)
    d = dev()
    sim.sim_step(0, 6)
    q, pp, slip = sim.sim_read_observation()
    forces, status = sim.sim_read_sensors()
    gt = (q[7].clone(), pp[7].clone(), forces[7].clone(), slip[7].clone())
    cm = torch.empty(n, dtype=torch.float64, device=d)
    am = torch.empty(1, dtype=torch.int32, device=d)
    c_sum = np.zeros(n)
    for k in range(2):
        sim.sim_step(6 + k, 1)
        obs, st = _gpu_obs(sim)
        sim.cost_eval_full(*gt, cm, am)
        # the ground truth as it was stored
        gq, gpp, gf, gs = (t.cpu().numpy() for t in gt)
        g = O.Obs(gq[None].astype(np.float64), np.concatenate([gpp[:, :3], gpp[:, 4:8]], -1)[None].astype(np.float64),
                  gf[None].astype(np.float64), gs[None, :, :2].astype(np.float64), gs[None, :, 2].copy().view(np.int32))
        i, c_mean, _ = O.cost_full(sim32(wl.sim), obs, g, st, c_sum, k + 1)
        got = cm.cpu().numpy()
        fin = np.isfinite(c_mean)
        np.testing.assert_array_equal(np.isfinite(got), fin)
        np.testing.assert_allclose(got[fin], c_mean[fin], rtol=1e-12, atol=1e-12)
        assert int(am.item()) == i
    assert np.unique(got[fin]).size > n // 2


def test_pd_free_joints_settle_on_the_command():
    from paper_2002_12160_gb300 import inhand
    d = dev()
    wl = _pd("tracking_box27", 4, 300, gravity=(0.0, 0.0, 0.0))
    sim = inhand.make_sim(wl, n_envs=4, max_frames=300)
    u = np.linspace(-0.3, 0.6, wl.scene.n_joints).astype(np.float32)
    sim.sim_set_commands(0, torch.from_numpy(np.tile(u, (301, 1))).to(d))
    pose = torch.from_numpy(np.tile(wl.nominal_pose, (4, 1))).to(d)
    pose[:, 2] = 0.25
    sim.sim_set_state(pose, torch.zeros((4, 8), dtype=torch.float32, device=d),
                      torch.tensor([[0.1, 0.5]] * 4, dtype=torch.float32, device=d))
    sim.sim_set_hand(torch.zeros((4, wl.scene.n_joints), dtype=torch.float32, device=d))
    sim.sim_step(0, 300)
    q, qd = sim.sim_get_hand()
    np.testing.assert_allclose(q.cpu().numpy(), np.tile(u, (4, 1)), atol=2e-6)
    assert np.abs(qd.cpu().numpy()).max() < 1e-4


@pytest.mark.parametrize("kind", ["elite", "reps"])
def test_pd_optimizer_copies_the_parents_joints(kind):
    n = 120
    wl = _pd("tracking_cyl64", n, 6)
    wl.opt = dataclasses.replace(wl.opt, kind=kind)
    sim = start(wl, n=n, frames=6)
    d = dev()
    cm = torch.empty(n, dtype=torch.float64, device=d)
    for f in range(3):
        sim.sim_step(f, 1)
        q, pp, slip = sim.sim_read_observation()
        forces, _ = sim.sim_read_sensors()
        sim.cost_eval_full(q[5].clone(), pp[5].clone(), forces[5].clone(), slip[5].clone(), cm)
    qb, qdb = (t.clone() for t in sim.sim_get_hand())
    par = torch.empty(n, dtype=torch.int32, device=d)
    sim.optimizer_update(wl.opt, 0, None, par)
    qa, qda = sim.sim_get_hand()
    p = par.cpu().numpy().astype(np.int64)
    assert (p != np.arange(n)).any()
    assert torch.equal(qa, qb[p]) and torch.equal(qda, qdb[p])


def test_pd_refuses_unsupported_calls():
    from paper_2002_12160_gb300 import inhand
    d = dev()
    wl = _pd("tracking_box27", 4, 4)
    sim = start(wl, n=4, frames=4)
    obs = torch.zeros((1, wl.scene.n_pads, 3), dtype=torch.float32, device=d)
    with pytest.raises(inhand.InhandError):
        sim.sim_step_track(0, obs[0])
    with pytest.raises(inhand.InhandError):
        sim.sim_step_frames(0, obs)
    with pytest.raises(inhand.InhandError):
        sim.sim_adjoint(0, obs)
    with pytest.raises(inhand.InhandError):
        sim.sim_autotune(0, 1)
    wl2 = _pd("tracking_box27", 4, 4, warm_start=True)
    with pytest.raises(inhand.InhandError):
        inhand.make_sim(wl2, n_envs=4, max_frames=4)
    cold = start(W.make_workload("tracking_box27", n_envs=4, frames=4), n=4, frames=4)
    with pytest.raises(inhand.InhandError):
        cold.sim_read_observation()


@pytest.mark.parametrize("v0,w0", [((0.3, 0.0, 0.0), (0.0, 0.0, 2.0)), ((0.0, -0.3, 0.0), (0.0, 0.0, -2.0))])
def test_pd_palm_pad_slip_without_fingers(v0, w0):
    """A hand with no fingers (no joints): a slab sliding and spinning on the
    palm pad, one frame, against the oracle."""
    from paper_2002_12160_gb300 import inhand
    d = dev()
    rows = W.slab9()
    scene = W.ground_scene(rows)
    cfg = dataclasses.replace(W.SimConfig(), hand="pd")
    sim = inhand.Sim(scene, cfg, 3, 2, seed=1)
    sim.sim_set_commands(0, torch.zeros((3, 0), dtype=torch.float32, device=d))
    z0 = 0.01 + W.bottom_depth(rows)
    pose = torch.tensor([[0, 0, z0 - 0.0005, 0, 1, 0, 0, 0]] * 3, dtype=torch.float32, device=d)
    vel = torch.tensor([[*v0, 0, *w0, 0], [0.5 * v0[0], 0.5 * v0[1], 0, 0, 0, 0, 0, 0], [0] * 8],
                       dtype=torch.float32, device=d)
    sim.sim_set_state(pose, vel, torch.tensor([[0.1, 0.3]] * 3, dtype=torch.float32, device=d))
    st = oracle_state(sim.sim_get_state()).hand(np.zeros(0))
    ob, _ = O.step_pd(O.OracleScene(scene32(scene)), sim32(cfg), st, np.zeros((3, 0)), 0, 1)
    sim.sim_step(0, 1)
    go, status = _gpu_obs(sim)
    np.testing.assert_array_equal(go.flags, ob.flags)
    assert go.flags[0, 0] & 1 and go.flags[0, 0] & 2 and go.flags[2, 0] == 0
    np.testing.assert_allclose(go.slip_d, ob.slip_d, atol=5e-3)
    fe = np.linalg.norm(go.forces - ob.forces, axis=2)
    assert (fe <= FORCE_REL * np.linalg.norm(ob.forces, axis=2) + FORCE_ABS).all()
    np.testing.assert_allclose(go.pad_pose[:, 0], [[0, 0, 0.01, 1, 0, 0, 0]] * 3, atol=1e-7)


def test_pd_overflow_and_escape_flags_match_oracle():
    wl = _pd("tracking_cyl64", 4, 3, c_max=8)
    sim = start(wl, n=4, frames=3)
    pose, vel, params, _ = sim.sim_get_state()
    pose[3, 2] = 0.29
    vel[3, 2] = 3.0
    q, qd = sim.sim_get_hand()
    sim.sim_set_state(pose, vel, params)
    sim.sim_set_hand(q, qd)
    st = _hand_state(sim, wl.shape_id[:4].astype(np.int32), wl.iters[:4].astype(np.int32))
    O.step_pd(O.OracleScene(scene32(wl.scene)), sim32(wl.sim), st, wl.q_traj, 0, 1)
    sim.sim_step(0, 1)
    status = sim.sim_get_state()[3].cpu().numpy()
    np.testing.assert_array_equal(status, st.status)
    assert status[3] & 2 and (status[:3] & 4).all()
    # the flagged environments are no longer stepped
    before = sim.sim_get_state()[0].clone()
    sim.sim_step(1, 1)
    assert torch.equal(sim.sim_get_state()[0], before)


@pytest.mark.parametrize("name,n,lens", [("tracking_cyl64", 150, (3, 5, 2)), ("tracking_box27", 40, (35, 4)),
                                         ("uneven_mixed", 67, (4, 3))])
def test_pd_window_launch_equals_the_separate_calls(name, n, lens):
    """sim_step_frames_full + sim_frames_argmin (the window's frames in one step
    launch, then scored by the frames' cost launches) equal per-frame calls of
    sim_step and cost_eval_full bit for bit: estimates, argmins, the optimizer's
    parents, the state and the joints, over windows of 3, 5 and 2 frames (the
    per-frame buffers grow, then are reused), of 35 and 4 frames (the window
    means run over more frames than a warp has lanes), and on the uneven batch
    (five fingers, 16 pads, mixed shapes and iteration counts)."""
    from paper_2002_12160_gb300 import inhand
    F = sum(lens)
    wl = _pd(name, n, F)
    d = dev()
    g = start(wl, n=n, frames=F)   # the truth's observations: environment 3 of another run
    D, P = wl.scene.n_joints, wl.scene.n_pads
    oq = torch.empty((F, D), dtype=torch.float32, device=d)
    opp = torch.empty((F, P, 8), dtype=torch.float32, device=d)
    of = torch.empty((F, P, 3), dtype=torch.float32, device=d)
    osl = torch.empty((F, P, 4), dtype=torch.float32, device=d)
    for f in range(F):
        g.sim_step(f, 1)
        q, pp, slip = g.sim_read_observation()
        forces, _ = g.sim_read_sensors()
        oq[f], opp[f], of[f], osl[f] = q[3], pp[3], forces[3], slip[3]
    a = start(wl, n=n, frames=F)
    b = start(wl, n=n, frames=F)
    est_a = torch.zeros((F, 8), dtype=torch.float32, device=d)
    est_b = torch.zeros_like(est_a)
    am_a = torch.zeros((F,), dtype=torch.int32, device=d)
    am_b = torch.zeros_like(am_a)
    par_a = torch.empty(n, dtype=torch.int32, device=d)
    par_b = torch.empty_like(par_a)
    f0 = 0
    for w, T in enumerate(lens):
        for f in range(f0, f0 + T):
            a.sim_step(f, 1)
            a.cost_eval_full(oq[f], opp[f], of[f], osl[f], None, am_a[f:f + 1], est_a[f])
        a.optimizer_update(wl.opt, w, None, par_a)
        s = slice(f0, f0 + T)
        b.sim_step_frames_full(f0, oq[s], opp[s], of[s], osl[s])
        if w == 0:   # scoring again before the argmin is refused
            with pytest.raises(inhand.InhandError):
                b.cost_eval_full(oq[0], opp[0], of[0], osl[0])
        b.sim_frames_argmin(est_b[s], am_b[s])
        b.optimizer_update(wl.opt, w, None, par_b)
        assert torch.equal(par_a, par_b)
        f0 += T
    assert torch.equal(est_a, est_b) and torch.equal(am_a, am_b)
    for x, y in zip(a.sim_get_state(), b.sim_get_state()):
        assert torch.equal(x, y)
    for x, y in zip(a.sim_get_hand(), b.sim_get_hand()):
        assert torch.equal(x, y)
    for x, y in zip(a.sim_read_observation(), b.sim_read_observation()):
        assert torch.equal(x, y)


def test_pd_full_size_window_launch_sampled_parity():
    """At the benchmark's size (N = 1024 cylinders) and in the launch the
    benchmark times (a window's step launch and its frames' cost launches), a sample of
    environments checked one by one against the oracle's step, and the
    launch's argmin and estimate against the oracle's full cost of the GPU's
    observation."""
    n = 1024
    wl = _pd("tracking_cyl64", n, 8)
    sim = start(wl, n=n, frames=8)
    d = dev()
    sim.sim_step(0, 5)
    q, pp, slip = sim.sim_read_observation()
    forces, _ = sim.sim_read_sensors()
    gt = [t[17:18].clone() for t in (q, pp, forces, slip)]   # one environment's observation as the truth
    shape = wl.shape_id[:n].astype(np.int32)
    iters = wl.iters[:n].astype(np.int32)
    rng = np.random.default_rng(0)
    envs = np.sort(rng.choice(n, 24, replace=False))
    envs[-1] = n - 1
    st = _hand_state(sim, shape, iters).subset(envs)
    ob, diag = O.step_pd(O.OracleScene(scene32(wl.scene)), sim32(wl.sim), st, wl.q_traj, 5, 1)
    sim.sim_step_frames_full(5, *gt)
    est = torch.empty((1, 8), dtype=torch.float32, device=d)
    am = torch.empty(1, dtype=torch.int32, device=d)
    sim.sim_frames_argmin(est, am)
    g = _hand_state(sim, shape, iters).subset(envs)
    ok = ~((diag[:, 2] < FRAGILE) | (diag[:, 3] < FRAGILE) | (diag[:, 4] < FRAGILE))
    assert ok.mean() >= 0.75
    np.testing.assert_array_equal(g.status[ok], st.status[ok])
    assert np.linalg.norm(g.pose[ok, :3] - st.pose[ok, :3], axis=1).max() < POS_TOL
    assert rot_angle(g.pose[ok], st.pose[ok]).max() < ROT_TOL
    np.testing.assert_allclose(g.qj[ok], st.qj[ok], atol=1e-5)
    # the cost means the launch left for the optimizer, against the oracle's
    # cost of the GPU's own observation (FP64 on both sides, same inputs)
    go, status = _gpu_obs(sim)
    gq, gpp, gf, gs = (t.cpu().numpy()[0] for t in gt)
    truth = O.Obs(gq[None].astype(np.float64), np.concatenate([gpp[:, :3], gpp[:, 4:8]], -1)[None].astype(np.float64),
                  gf[None].astype(np.float64), gs[None, :, :2].astype(np.float64), gs[None, :, 2].copy().view(np.int32))
    c_sum = np.zeros(n)
    i_or, c_mean, _ = O.cost_full(sim32(wl.sim), go, truth, status, c_sum, 1)
    assert int(am.item()) == i_or
    # the estimate is the argmin environment's pose after the frame
    pose = sim.sim_get_state()[0]
    assert torch.equal(est[0], pose[i_or])
