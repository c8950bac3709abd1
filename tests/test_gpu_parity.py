"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every comparison starts both sides from the same state -- the GPU's FP32
state widened exactly to FP64 -- and advances one frame. Tolerances: pose
1e-5 m and 1e-5 rad, pad force 1e-3 relative with a 1e-4 N floor; status bits,
contact counts, elite sets and parents are compared exactly. Environments
whose contact set or pad membership sits within 1e-6 m of a threshold are
excluded and counted (a branch that FP32 and FP64 may take differently).
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_12160_gb300 import workloads as W

from gpu_common import (assert_report, compare_frame, dev, oracle_state, scene32, sim32, start,
                        torch)

pytestmark = pytest.mark.gpu


def test_initial_sampling_matches_oracle():
    wl = W.make_workload("tracking_cyl64", n_envs=257, frames=4)
    sim = start(wl, n=257, frames=4)
    pose, vel, params, status = (t.cpu().numpy() for t in sim.sim_get_state())
    p_or, th_or = O.sample_initial(257, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    np.testing.assert_allclose(pose[:, :3], p_or[:, :3], atol=1e-7)
    q = pose[:, 4:]
    assert np.max(np.abs(np.abs(np.sum(q * p_or[:, 3:], 1)) - 1)) < 1e-6
    np.testing.assert_allclose(params, th_or, rtol=1e-6)
    assert np.all(vel == 0) and np.all(status == 0)


@pytest.mark.parametrize("name,n,frames,check", [
    ("tracking_box27", 16, 40, [0, 5, 17, 30, 39]),
    ("tracking_cyl64", 61, 30, [3, 12, 29]),
    ("uneven_mixed", 67, 20, [2, 9, 19]),
    ("sweep_mug128", 29, 12, [4, 11]),
])
def test_one_frame_parity(name, n, frames, check):
    wl = W.make_workload(name, n_envs=n, frames=frames)
    sim = start(wl, n=n, frames=frames)
    total_ok = 0
    contacts = 0
    for f in range(frames):
        if f in check:
            rep = compare_frame(wl, sim, f)
            assert_report(rep)
            total_ok += rep["ok"].sum()
            contacts += rep["contacts_or"]
            if rep["ok"].all():
                # culled GPU enumeration finds exactly the oracle's brute-force contact set
                assert rep["work"]["contacts"] == rep["contacts_or"]
        else:
            sim.sim_step(f, 1)
    assert contacts > 0 and total_ok > 0


@pytest.mark.parametrize("name,n,frames,warm", [
    ("tracking_cyl64", 1024, 8, 6),
    ("uneven_mixed", 8192, 6, 4),
    ("sweep_mug128", 32768, 4, 2),
])
def test_full_size_sampled_parity(name, n, frames, warm):
    """At the benchmark sizes and launch shape, a sample of envs is checked one by one."""
    wl = W.make_workload(name, n_envs=n, frames=frames)
    sim = start(wl, n=n, frames=frames)
    sim.sim_step(0, warm)
    rng = np.random.default_rng(0)
    envs = np.sort(rng.choice(n, 24, replace=False))
    envs[-1] = n - 1          # the ragged tail of the last block
    rep = compare_frame(wl, sim, warm, envs)
    assert_report(rep)


def test_cost_and_argmin_match_oracle_bit_for_bit():
    wl = W.make_workload("tracking_box27", n_envs=16, frames=8)
    sim = start(wl, n=16, frames=8)
    d = dev()
    c_sum = np.zeros(16)
    cm = torch.empty(16, dtype=torch.float64, device=d)
    am = torch.empty(1, dtype=torch.int32, device=d)
    est = torch.empty(8, dtype=torch.float32, device=d)
    for f in range(8):
        sim.sim_step(f, 1)
        forces, status = sim.sim_read_sensors()
        obs = forces[3].clone()           # score everybody against env 3
        sim.cost_eval(obs, cm, am, est)
        i_or, c_or, _ = O.cost(sim32(wl.sim), forces.cpu().numpy().astype(np.float64),
                               obs.cpu().numpy().astype(np.float64), status.cpu().numpy(), c_sum, f + 1)
        np.testing.assert_array_equal(cm.cpu().numpy(), c_or)
        # env 3 scores zero against itself; a lower index with zero cost wins the tie
        assert int(am.item()) == i_or <= 3 and c_or[i_or] == 0.0 == c_or.min()
        pose = sim.sim_get_state()[0]
        np.testing.assert_array_equal(est.cpu().numpy(), pose[i_or].cpu().numpy())


@pytest.mark.parametrize("n", [300, 3000])   # one CTA for select + statistics + Cholesky; separate launches
def test_optimizer_update_matches_oracle(n):
    wl = W.make_workload("tracking_cyl64", n_envs=n, frames=6)
    sim = start(wl, n=n, frames=6)
    d = dev()
    cm = torch.empty(n, dtype=torch.float64, device=d)
    for f in range(6):
        sim.sim_step(f, 1)
        forces, _ = sim.sim_read_sensors()
        sim.cost_eval(forces[7].clone(), cm)
    before = oracle_state(sim.sim_get_state())
    C = cm.cpu().numpy()
    am = torch.empty(1, dtype=torch.int32, device=d)
    par = torch.empty(n, dtype=torch.int32, device=d)
    sim.optimizer_update(wl.opt, 5, am, par)
    after = oracle_state(sim.sim_get_state())
    istar, parent, stats = O.optimizer(wl.opt, before, C, wl.seed, 5)
    assert int(am.item()) == istar
    np.testing.assert_array_equal(par.cpu().numpy(), parent)
    np.testing.assert_allclose(after.pose[:, :3], before.pose[:, :3], atol=2e-7)
    assert rot_close(after.pose, before.pose, 2e-6)
    np.testing.assert_allclose(after.theta, before.theta, rtol=2e-6)
    np.testing.assert_array_equal(after.vel, before.vel)
    np.testing.assert_array_equal(after.status, before.status)
    # the window restarts: the next frame's mean is that frame's cost alone
    sim.sim_step(0, 1)
    forces, status = sim.sim_read_sensors()
    sim.cost_eval(forces[7].clone(), cm)
    _, c_one, _ = O.cost(sim32(wl.sim), forces.cpu().numpy().astype(np.float64),
                         forces[7].cpu().numpy().astype(np.float64), status.cpu().numpy(), np.zeros(n), 1)
    np.testing.assert_array_equal(cm.cpu().numpy(), c_one)


def rot_close(a, b, tol):
    from gpu_common import rot_angle
    return rot_angle(a, b).max() < tol


def test_invalid_state_is_flagged_and_skipped():
    wl = W.make_workload("tracking_box27", n_envs=8, frames=3)
    sim = start(wl, n=8, frames=3)
    pose, vel, params, _ = sim.sim_get_state()
    params[2, 0] = float("nan")
    params[3, 0] = -1.0
    shape = torch.zeros(8, dtype=torch.int32, device=pose.device)
    shape[4] = 5
    sim.sim_set_state(pose, vel, params, shape, None)
    _, _, _, status = sim.sim_get_state()
    st = status.cpu().numpy()
    assert list(np.nonzero(st)[0]) == [2, 3, 4] and np.all(st[[2, 3, 4]] == 8)
    p_before = sim.sim_get_state()[0].cpu().numpy()
    sim.sim_step(0, 2)
    forces, _ = sim.sim_read_sensors()
    p_after = sim.sim_get_state()[0].cpu().numpy()
    np.testing.assert_array_equal(p_after[[2, 3, 4]], p_before[[2, 3, 4]])
    cm = torch.empty(8, dtype=torch.float64, device=pose.device)
    sim.cost_eval(forces[0].clone(), cm)
    assert np.all(np.isinf(cm.cpu().numpy()[[2, 3, 4]]))


def test_free_fall_and_resting_closed_forms_on_gpu():
    """The GPU step reproduces the discrete free fall and carries exactly the weight at rest."""
    from paper_2002_12160_gb300 import inhand
    d = dev()
    rows = W.box27()
    sc = W.ground_scene(rows)
    cfg = W.SimConfig()
    sim = inhand.Sim(sc, cfg, 2, 400, seed=1)
    sim.sim_set_commands(0, torch.zeros((401, 0), dtype=torch.float32, device=d))
    z0 = 0.01 + W.bottom_depth(rows)
    pose = torch.tensor([[0, 0, 0.2, 0, 1, 0, 0, 0], [0, 0, z0 - 0.001, 0, 1, 0, 0, 0]], dtype=torch.float32, device=d)
    vel = torch.tensor([[0.1, 0, 0.3, 0, 0, 0, 0, 0], [0] * 8], dtype=torch.float32, device=d)
    params = torch.tensor([[0.1, 0.5], [0.17, 0.6]], dtype=torch.float32, device=d)
    sim.sim_set_state(pose, vel, params)
    sim.sim_step(0, 3)
    p = sim.sim_get_state()[0].cpu().numpy()
    h = cfg.frame_dt / cfg.substeps
    n = 3 * cfg.substeps
    z_ref = 0.2 + n * h * 0.3 - 9.81 * h * h * n * (n + 1) / 2
    assert abs(p[0, 2] - z_ref) < 2e-6 and abs(p[0, 0] - 0.1 * n * h) < 1e-6
    sim.sim_step(3, 297)
    forces, status = sim.sim_read_sensors()
    f = forces.cpu().numpy()
    np.testing.assert_allclose(f[1, 0], [0, 0, -0.17 * 9.81], rtol=2e-4, atol=1e-5)
    v = sim.sim_get_state()[1].cpu().numpy()
    assert np.abs(v[1]).max() < 1e-5


def test_contact_overflow_and_escape_flags_match_oracle():
    wl = W.make_workload("tracking_cyl64", n_envs=4, frames=3)
    wl.sim.c_max = 8
    sim = start(wl, n=4, frames=3)
    d = dev()
    pose, vel, params, _ = sim.sim_get_state()
    pose[3, 2] = 0.29
    vel[3, 2] = 3.0
    sim.sim_set_state(pose, vel, params)
    rep = compare_frame(wl, sim, 0)
    np.testing.assert_array_equal(rep["status_gpu"], rep["status_or"])
    assert rep["status_gpu"][3] & 2
    assert (rep["status_gpu"][:3] & 4).all()


def test_single_environment_and_ragged_batches():
    for n in (1, 5, 33):
        wl = W.make_workload("tracking_box27", n_envs=n, frames=6)
        sim = start(wl, n=n, frames=6)
        sim.sim_step(0, 3)
        rep = compare_frame(wl, sim, 3)
        assert_report(rep, min_ok_frac=0.0)


@pytest.mark.parametrize("variant", [(16, 2), (16, 4), (32, 1), (32, 2), (32, 3), (32, 4), (64, 1), (64, 2), (128, 1)])
def test_every_step_shape_matches_oracle(variant):
    """Each threads-per-environment shape of the step kernel gives the oracle's frame."""
    from paper_2002_12160_gb300 import inhand
    assert variant in inhand.step_variants()
    wl = W.make_workload("tracking_cyl64", n_envs=37, frames=8)
    sim = start(wl, n=37, frames=8)
    sim.sim_set_variant(*variant)
    sim.sim_step(0, 5)
    rep = compare_frame(wl, sim, 5)
    assert_report(rep)
    if rep["ok"].all():
        assert rep["work"]["contacts"] == rep["contacts_or"]


def test_autotune_restores_the_state_and_picks_a_shape():
    from paper_2002_12160_gb300 import inhand
    wl = W.make_workload("tracking_cyl64", n_envs=300, frames=8)
    sim = start(wl, n=300, frames=8)
    sim.sim_step(0, 2)
    before = [t.clone() for t in sim.sim_get_state()]
    f_before, _ = sim.sim_read_sensors()
    w_before = sim.sim_work_counters()
    chosen, ms = sim.sim_autotune(2, 2)
    after = sim.sim_get_state()
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    assert torch.equal(f_before, sim.sim_read_sensors()[0])
    assert sim.sim_work_counters() == w_before
    assert chosen in inhand.step_variants()
    assert all(np.isfinite(v) for v in ms.values())
    rep = compare_frame(wl, sim, 2)
    assert_report(rep)


def _twin(name, n, frames):
    wl = W.make_workload(name, n_envs=n, frames=frames)
    return wl, start(wl, n=n, frames=frames), start(wl, n=n, frames=frames)


def test_fused_step_and_score_equal_the_separate_calls():
    wl, a, b = _twin("tracking_cyl64", 131, 6)
    d = dev()
    ca = torch.empty(131, dtype=torch.float64, device=d)
    cb = torch.empty_like(ca)
    ia = torch.empty(1, dtype=torch.int32, device=d)
    ib = torch.empty_like(ia)
    ea = torch.empty(8, dtype=torch.float32, device=d)
    eb = torch.empty_like(ea)
    obs = None
    for f in range(6):
        a.sim_step(f, 1)
        fa, _ = a.sim_read_sensors()
        if obs is None:
            obs = fa[5].clone()
        a.cost_eval(obs, ca, ia, ea)
        b.sim_step_track(f, obs, cb, ib, eb)
        fb, _ = b.sim_read_sensors()
        assert torch.equal(fa, fb)
        assert torch.equal(ca, cb) and torch.equal(ia, ib) and torch.equal(ea, eb)
    for x, y in zip(a.sim_get_state(), b.sim_get_state()):
        assert torch.equal(x, y)


def test_replayed_window_equals_the_separate_calls():
    T = 4
    wl, a, b = _twin("tracking_cyl64", 200, 3 * T)
    d = dev()
    obs = torch.rand((3 * T, wl.scene.n_pads, 3), dtype=torch.float32, device=d) * 0.2
    est_a = torch.zeros((3 * T, 8), dtype=torch.float32, device=d)
    est_b = torch.zeros_like(est_a)
    am_a = torch.zeros((3 * T,), dtype=torch.int32, device=d)
    am_b = torch.zeros_like(am_a)
    for w in range(3):
        for k in range(T):
            f = w * T + k
            a.sim_step_track(f, obs[f], None, am_a[f:f + 1], est_a[f])
        a.optimizer_update(wl.opt, w)
        # the same window replayed from one captured graph (captured on w = 0)
        b.sim_track_window(w * T, obs[w * T:(w + 1) * T], wl.opt, w, est_b[w * T:(w + 1) * T],
                           am_b[w * T:(w + 1) * T])
    assert torch.equal(est_a, est_b) and torch.equal(am_a, am_b)
    for x, y in zip(a.sim_get_state(), b.sim_get_state()):
        assert torch.equal(x, y)


def test_multi_frame_launch_equals_the_separate_calls():
    """sim_step_frames + sim_frames_argmin (the window's frames in one launch,
    the per-frame argmin afterwards) equal T calls of sim_step_track bit for bit,
    including the cost means handed to the optimizer and a second window."""
    T = 5
    wl, a, b = _twin("uneven_mixed", 333, 2 * T)
    d = dev()
    obs = torch.rand((2 * T, wl.scene.n_pads, 3), dtype=torch.float32, device=d) * 0.3
    est_a = torch.zeros((2 * T, 8), dtype=torch.float32, device=d)
    est_b = torch.zeros_like(est_a)
    am_a = torch.zeros((2 * T,), dtype=torch.int32, device=d)
    am_b = torch.zeros_like(am_a)
    par_a = torch.zeros((a.n,), dtype=torch.int32, device=d)
    par_b = torch.zeros_like(par_a)
    cm_a = torch.zeros((a.n,), dtype=torch.float64, device=d)
    for w in range(2):
        for k in range(T):
            f = w * T + k
            a.sim_step_track(f, obs[f], cm_a, am_a[f:f + 1], est_a[f])
        b.sim_step_frames(w * T, obs[w * T:(w + 1) * T])
        if w == 0:   # the frames' argmin comes before any further scoring
            from paper_2002_12160_gb300 import inhand
            with pytest.raises(inhand.InhandError) as e:
                b.sim_step_track(T, obs[T])
            assert e.value.code == inhand.IH_ERR_STATE
        b.sim_frames_argmin(est_b[w * T:(w + 1) * T], am_b[w * T:(w + 1) * T])
        a.optimizer_update(wl.opt, w, None, par_a)
        b.optimizer_update(wl.opt, w, None, par_b)
        assert torch.equal(par_a, par_b), w
    assert torch.equal(est_a, est_b) and torch.equal(am_a, am_b)
    for x, y in zip(a.sim_get_state(), b.sim_get_state()):
        assert torch.equal(x, y)
    from paper_2002_12160_gb300 import inhand
    with pytest.raises(inhand.InhandError) as e:
        b.sim_frames_argmin()
    assert e.value.code == inhand.IH_ERR_STATE


def _opt32(opt):
    """The optimizer constants as the GPU receives them (FP32), widened exactly."""
    import dataclasses
    f = lambda v: tuple(float(np.float32(x)) for x in v)
    return dataclasses.replace(opt, wrs_lambda=float(np.float32(opt.wrs_lambda)),
                               reps_epsilon=float(np.float32(opt.reps_epsilon)), sigma_pose=f(opt.sigma_pose),
                               sigma_theta=f(opt.sigma_theta), sigma_vel=f(opt.sigma_vel), m_range=f(opt.m_range),
                               mu_range=f(opt.mu_range))


@pytest.mark.parametrize("kind,explore", [("wrs", "pose"), ("reps", "pose"), ("reps", "velocity"), ("wrs", "velocity")])
def test_wrs_and_reps_updates_match_oracle(kind, explore):
    """WRS / REPS on the GPU (one CTA for the weights and the REPS temperature,
    then draws with replacement and exploration) against the oracle: i* and
    every parent exactly, states to FP32 rounding; a diverged environment is
    never drawn."""
    import dataclasses
    n = 517
    wl = W.make_workload("tracking_cyl64", n_envs=n, frames=6)
    sim = start(wl, n=n, frames=6)
    d = dev()
    cm = torch.empty(n, dtype=torch.float64, device=d)
    for f in range(5):
        sim.sim_step(f, 1)
        forces, _ = sim.sim_read_sensors()
        sim.cost_eval(forces[7].clone(), cm)
    # environment 5 made invalid before the last frame: its window mean is +inf
    pose, vel, params, _ = sim.sim_get_state()
    params = params.clone()
    params[5, 0] = -1.0
    sim.sim_set_state(pose, vel, params)
    sim.sim_step(5, 1)
    forces, _ = sim.sim_read_sensors()
    sim.cost_eval(forces[7].clone(), cm)
    before = oracle_state(sim.sim_get_state())
    C = cm.cpu().numpy().copy()
    assert np.isinf(C[5]) and np.isfinite(np.delete(C, 5)).all()
    opt = dataclasses.replace(wl.opt, kind=kind, explore=explore, wrs_lambda=0.8, reps_epsilon=0.7)
    am = torch.empty(1, dtype=torch.int32, device=d)
    par = torch.empty(n, dtype=torch.int32, device=d)
    sim.optimizer_update(opt, 9, am, par)
    after = oracle_state(sim.sim_get_state())
    istar, parent, stats = O.softmax_update(_opt32(opt), before, C, wl.seed, 9)
    assert int(am.item()) == istar
    np.testing.assert_array_equal(par.cpu().numpy(), parent)
    assert len(np.unique(parent)) > 5 and not np.any(parent == 5)
    np.testing.assert_allclose(after.pose[:, :3], before.pose[:, :3], atol=2e-7)
    assert rot_close(after.pose, before.pose, 2e-6)
    np.testing.assert_allclose(after.theta, before.theta, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(after.vel, before.vel, atol=2e-6)
    np.testing.assert_array_equal(after.status, before.status)
    # the window restarts
    sim.sim_step(0, 1)
    forces, status = sim.sim_read_sensors()
    sim.cost_eval(forces[7].clone(), cm)
    _, c_one, _ = O.cost(sim32(wl.sim), forces.cpu().numpy().astype(np.float64),
                         forces[7].cpu().numpy().astype(np.float64), status.cpu().numpy(), np.zeros(n), 1)
    np.testing.assert_array_equal(cm.cpu().numpy(), c_one)


def test_reps_window_replay_equals_the_separate_calls():
    """A REPS window captured in a graph equals the separate calls bit for bit."""
    import dataclasses
    T = 3
    wl, a, b = _twin("tracking_box27", 96, 2 * T)
    d = dev()
    opt = dataclasses.replace(wl.opt, kind="reps", explore="velocity")
    obs = torch.rand((2 * T, wl.scene.n_pads, 3), dtype=torch.float32, device=d) * 0.2
    for w in range(2):
        for k in range(T):
            a.sim_step_track(w * T + k, obs[w * T + k])
        a.optimizer_update(opt, w)
        b.sim_track_window(w * T, obs[w * T:(w + 1) * T], opt, w)
    for x, y in zip(a.sim_get_state(), b.sim_get_state()):
        assert torch.equal(x, y)


def test_maximum_sizes_match_oracle():
    """The library's capacities at once: 7 fingers (29 links, every bit of a
    warp's link mask but three), 32 sensor pads (distal and middle links split
    in axial halves, three proximal links, the palm), the 256-sphere object
    beside the mug, c_max = 256 contacts, iteration counts 10/20/40 -- one
    frame against the oracle, on the default shape and on the narrowest and
    widest groups."""
    import dataclasses
    n, frames, F = 45, 16, 7
    base = W.make_workload("uneven_mixed", n_envs=n, frames=frames)
    shapes = [W.l_composite256(), W.mug128()]
    link, s0, s1 = [], [], []
    for f in range(F):
        for j in (3, 2):
            link += [1 + 4 * f + j] * 2
            s0 += [0.0, 0.5]
            s1 += [0.5, 1.0]
    for f in range(3):
        link.append(1 + 4 * f + 1)
        s0.append(0.0)
        s1.append(1.0)
    link.append(0)
    s0.append(0.0)
    s1.append(1.0)
    assert len(link) == 32
    root = W.make_hand(F, W._root_radius(shapes, base.scene.link_rad), palm_top=base.scene.palm_half[2])
    scene = dataclasses.replace(base.scene, shapes=shapes, finger_root=root, pad_link=np.array(link, np.int32),
                                pad_s0=np.array(s0), pad_s1=np.array(s1))
    rng = np.random.default_rng(5)
    wl = dataclasses.replace(base, scene=scene, q_traj=W.joint_trajectory(F, frames, base.sim.frame_dt, base.seed),
                             shape_id=rng.integers(0, 2, n).astype(np.int32),
                             iters=rng.choice(np.array([10, 20, 40], np.int32), n).astype(np.int32),
                             nominal_pose=W.nominal_pose_for(scene, 0))
    assert scene.n_links == 29 and scene.n_pads == 32 and wl.sim.c_max == 256
    total = 0
    for shape in (None, (16, 2), (128, 1)):
        sim = start(wl, n=n, frames=frames)
        if shape:
            sim.sim_set_variant(*shape)
        sim.sim_step(0, 12)
        rep = compare_frame(wl, sim, 12)
        assert_report(rep)
        total += rep["contacts_or"]
        sim.close()
    assert total > 0
