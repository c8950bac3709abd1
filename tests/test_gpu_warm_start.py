"""The warm-started solver on the GPU (each contact starts from the final
impulse of its (link, sphere) pair in the environment's previous substep).

- one frame from the same state and the same impulse cache matches the
  oracle: pose, pad forces, status and the cache left behind (pairs exactly,
  impulses within the pad-force tolerance);
- the closed form survives: a resting box carries exactly its weight, and
  with one Jacobi iteration per substep it still converges to it (the oracle
  pin, on the GPU) where the cold-started solver does not;
- a window launch (T frames in one launch) equals T single-frame launches
  bit for bit, caches included;
- the cache starts empty after sim_sample_initial / sim_set_state, an
  optimizer update empties it for every replaced environment and keeps the
  elites', the autotuner leaves it as it found it, and the adjoint refuses
  a warm-started handle.
"""
import dataclasses

import numpy as np
import pytest

from paper_2002_12160_gb300 import workloads as W

from gpu_common import assert_report, compare_frame, dev, start, torch

pytestmark = pytest.mark.gpu


def _warm(name, n, frames, iters=None):
    wl = W.make_workload(name, n_envs=n, frames=frames)
    wl.sim = dataclasses.replace(wl.sim, warm_start=True)
    if iters is not None:
        wl.sim.iters = iters
        wl.iters[:] = iters
    return wl


@pytest.mark.parametrize("name,n,frames,check,iters", [
    ("tracking_box27", 16, 30, [1, 9, 29], None),
    ("tracking_cyl64", 61, 20, [2, 11, 19], None),
    ("tracking_cyl64", 40, 12, [5, 11], 3),
    ("uneven_mixed", 67, 12, [4, 11], None),
])
def test_warm_one_frame_parity(name, n, frames, check, iters):
    wl = _warm(name, n, frames, iters)
    sim = start(wl, n=n, frames=frames)
    assert sim.warm_start
    total_ok, contacts = 0, 0
    for f in range(frames):
        if f in check:
            rep = compare_frame(wl, sim, f)
            assert_report(rep)
            total_ok += rep["ok"].sum()
            contacts += rep["contacts_or"]
        else:
            sim.sim_step(f, 1)
    assert contacts > 0 and total_ok > 0
    cnt, _, _ = sim.sim_get_warm_cache()
    assert int(cnt.sum().item()) > 0


def test_every_step_shape_warm_matches_oracle():
    from paper_2002_12160_gb300 import inhand
    wl = _warm("tracking_cyl64", 37, 8)
    for variant in inhand.step_variants():
        sim = start(wl, n=37, frames=8)
        sim.sim_set_variant(*variant)
        sim.sim_step(0, 5)
        rep = compare_frame(wl, sim, 5)
        assert_report(rep)


def _resting(iters, warm, frames):
    from paper_2002_12160_gb300 import inhand
    d = dev()
    rows = W.box27()
    cfg = dataclasses.replace(W.SimConfig(), iters=iters, warm_start=warm)
    sim = inhand.Sim(W.ground_scene(rows), cfg, 1, frames, seed=1)
    sim.sim_set_commands(0, torch.zeros((frames + 1, 0), dtype=torch.float32, device=d))
    z0 = 0.01 + W.bottom_depth(rows)
    sim.sim_set_state(torch.tensor([[0, 0, z0 - 0.001, 0, 1, 0, 0, 0]], dtype=torch.float32, device=d),
                      torch.zeros((1, 8), dtype=torch.float32, device=d),
                      torch.tensor([[0.17, 0.6]], dtype=torch.float32, device=d))
    sim.sim_step(0, frames)
    forces, _ = sim.sim_read_sensors()
    pose, vel, _, _ = (t.cpu().numpy()[0] for t in sim.sim_get_state())
    return forces.cpu().numpy()[0, 0], pose[2] - z0, vel


def test_resting_box_closed_form_warm():
    slop = W.SimConfig().slop
    f, dz, v = _resting(20, True, 300)
    np.testing.assert_allclose(f, [0, 0, -0.17 * 9.81], rtol=2e-4, atol=1e-5)
    assert np.abs(v).max() < 1e-5 and abs(dz + slop) < 1e-5
    # one iteration per substep: the warm solve comes to rest within the slop,
    # the cold one sinks until the penetration bias makes up for the 1/n_c step
    f1, dz1, v1 = _resting(1, True, 150)
    _, dz1c, _ = _resting(1, False, 150)
    assert abs(f1[2] + 0.17 * 9.81) < 2e-4 * 0.17 * 9.81, f1
    assert -slop - 1e-5 <= dz1 <= 1e-5, dz1
    assert dz1c < -10 * slop, dz1c
    assert np.abs(v1).max() < 1e-4


def test_window_launch_warm_equals_the_separate_calls():
    T = 5
    wl = _warm("uneven_mixed", 211, 2 * T)
    a = start(wl, n=211, frames=2 * T)
    b = start(wl, n=211, frames=2 * T)
    d = dev()
    obs = torch.rand((2 * T, wl.scene.n_pads, 3), dtype=torch.float32, device=d) * 0.2
    est_a = torch.zeros((2 * T, 8), dtype=torch.float32, device=d)
    est_b = torch.zeros_like(est_a)
    am_a = torch.zeros((2 * T,), dtype=torch.int32, device=d)
    am_b = torch.zeros_like(am_a)
    for w in range(2):
        for k in range(T):
            f = w * T + k
            a.sim_step_track(f, obs[f], None, am_a[f:f + 1], est_a[f])
        a.optimizer_update(wl.opt, w)
        b.sim_step_frames(w * T, obs[w * T:(w + 1) * T])
        b.sim_frames_argmin(est_b[w * T:(w + 1) * T], am_b[w * T:(w + 1) * T])
        b.optimizer_update(wl.opt, w)
    assert torch.equal(est_a, est_b) and torch.equal(am_a, am_b)
    for x, y in zip(a.sim_get_state(), b.sim_get_state()):
        assert torch.equal(x, y)
    ca, cb = a.sim_get_warm_cache(), b.sim_get_warm_cache()
    assert torch.equal(ca[0], cb[0])
    for i in range(211):
        k = int(ca[0][i])
        assert torch.equal(ca[1][i, :k], cb[1][i, :k]) and torch.equal(ca[2][i, :k], cb[2][i, :k])


def test_cache_resets_and_the_optimizer_keeps_only_elites():
    from paper_2002_12160_gb300 import inhand
    n = 300
    wl = _warm("tracking_cyl64", n, 8)
    sim = start(wl, n=n, frames=8)
    d = dev()
    assert int(sim.sim_get_warm_cache()[0].abs().sum()) == 0
    cm = torch.empty(n, dtype=torch.float64, device=d)
    for f in range(4):
        sim.sim_step(f, 1)
        forces, _ = sim.sim_read_sensors()
        sim.cost_eval(forces[3].clone(), cm)
    before = sim.sim_get_warm_cache()
    assert int((before[0] > 0).sum()) > n // 4
    par = torch.empty(n, dtype=torch.int32, device=d)
    sim.optimizer_update(wl.opt, 0, None, par)
    after = sim.sim_get_warm_cache()
    parent = par.cpu().numpy()
    elite = parent == np.arange(n)
    assert elite.any() and (~elite).any()
    np.testing.assert_array_equal(after[0].cpu().numpy()[~elite], 0)
    np.testing.assert_array_equal(after[0].cpu().numpy()[elite], before[0].cpu().numpy()[elite])
    # the autotuner puts the cache back
    sim.sim_step(4, 1)
    c0 = [t.clone() for t in sim.sim_get_warm_cache()]
    sim.sim_autotune(5, 1)
    c1 = sim.sim_get_warm_cache()
    assert torch.equal(c0[0], c1[0])
    for i in range(n):
        k = int(c0[0][i])
        assert torch.equal(c0[1][i, :k], c1[1][i, :k]) and torch.equal(c0[2][i, :k], c1[2][i, :k])
    # new samples and an overwritten state start cold
    sim.sim_sample_initial(wl.nominal_pose, wl.init.sigma_p, wl.init.sigma_r, wl.init.m_range, wl.init.mu_range)
    assert int(sim.sim_get_warm_cache()[0].abs().sum()) == 0
    sim.sim_step(5, 1)
    assert int(sim.sim_get_warm_cache()[0].sum()) > 0
    sim.sim_set_state(*sim.sim_get_state()[:3])
    assert int(sim.sim_get_warm_cache()[0].abs().sum()) == 0
    # WRS replaces every environment
    sim.sim_step(6, 1)
    forces, _ = sim.sim_read_sensors()
    sim.cost_eval(forces[3].clone(), cm)
    sim.optimizer_update(dataclasses.replace(wl.opt, kind="wrs"), 1)
    assert int(sim.sim_get_warm_cache()[0].abs().sum()) == 0
    # the adjoint differentiates the cold-started solver only
    obs = torch.zeros((1, wl.scene.n_pads, 3), dtype=torch.float32, device=d)
    with pytest.raises(inhand.InhandError):
        sim.sim_adjoint(7, obs)


def test_cold_handle_has_no_cache():
    from paper_2002_12160_gb300 import inhand
    wl = W.make_workload("tracking_box27", n_envs=4, frames=2)
    sim = start(wl, n=4, frames=2)
    with pytest.raises(inhand.InhandError):
        sim.sim_get_warm_cache()
