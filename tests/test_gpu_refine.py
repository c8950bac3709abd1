"""Gradient refinement of the elites (sim_refine_elites) on the GPU.

Properties that hold whatever the scene: zero steps change nothing; the
refined window cost never exceeds the unrefined one, and is lower for some
elites; environments that are not elites keep their state bit for bit; the
unrefined cost is the scored window cost (to FP32 rounding); the call is
deterministic; and it refuses a window it did not see start.
"""
import numpy as np
import pytest

from paper_2002_12160_gb300 import inhand, workloads as W

from gpu_common import dev, start, torch

pytestmark = pytest.mark.gpu

T = 10


def _window(n=64, warm=20, name="tracking_cyl64"):
    wl = W.make_workload(name, n_envs=n, frames=warm + T + 2)
    sim = start(wl, n=n, frames=warm + T + 2)
    sim.sim_step(0, warm)
    d = dev()
    # observations: a ground-truth handle from environment 0's state
    gt = inhand.make_sim(wl, n_envs=1, max_frames=warm + T + 2)
    gt.sim_set_commands(0, torch.from_numpy(wl.q_traj[: warm + T + 3]).contiguous().to(d))
    pose, vel, params, _ = sim.sim_get_state()
    gt.sim_set_state(pose[:1].contiguous(), vel[:1].contiguous(),
                     torch.tensor([wl.theta_gt], dtype=torch.float32, device=d))
    obs = torch.empty((T, wl.scene.n_pads, 3), dtype=torch.float32, device=d)
    for k in range(T):
        gt.sim_step(warm + k, 1)
        f, _ = gt.sim_read_sensors()
        obs[k].copy_(f[0])
    gt.close()
    opt = W.OptConfig()
    opt.elite_frac = 0.25
    # a fresh cost window, then the scored window
    sim.sim_step_track(warm, obs[0])
    sim.optimizer_update(opt, 99)
    sim.sim_set_state(pose, vel, params)
    sim.sim_mark_window()
    cm = torch.empty(sim.n, dtype=torch.float64, device=d)
    for k in range(T):
        sim.sim_step_track(warm + k, obs[k], cm)
    return wl, sim, obs, opt, warm, cm


def test_zero_steps_is_a_noop():
    wl, sim, obs, opt, warm, cm = _window()
    before = sim.sim_get_state()
    el, c0, c1 = sim.sim_refine_elites(warm, obs, opt, steps=0, report=True)
    after = sim.sim_get_state()
    assert all(torch.equal(a, b) for a, b in zip(before, after))
    assert torch.equal(c0, c1)
    np.testing.assert_allclose(c0.cpu().numpy(), cm[el.long()].cpu().numpy() * T, rtol=1e-5)


def test_refinement_lowers_elite_costs_only():
    wl, sim, obs, opt, warm, cm = _window()
    before = [t.clone() for t in sim.sim_get_state()]
    el, c0, c1 = sim.sim_refine_elites(warm, obs, opt, steps=3, report=True)
    after = sim.sim_get_state()
    c0, c1 = c0.cpu().numpy(), c1.cpu().numpy()
    el = el.cpu().numpy()
    assert len(el) == 16 and np.all(np.diff(el) > 0)
    assert np.all(c1 <= c0) and np.any(c1 < c0), (c0, c1)
    # elites are the 16 lowest window means
    assert set(el) == set(np.argsort(cm.cpu().numpy(), kind="stable")[:16])
    d = dev()
    others = torch.from_numpy(np.setdiff1d(np.arange(sim.n), el)).long().to(d)
    improved = torch.from_numpy(el[c1 < c0]).long().to(d)
    for a, b in zip(before[:3], after[:3]):
        assert torch.equal(a[others], b[others])
        assert not torch.equal(a[improved], b[improved])
    np.testing.assert_allclose(c0, cm.cpu().numpy()[el] * T, rtol=1e-5)
    sim.optimizer_update(opt, 100)   # the update runs on the refined window means
    sim.sim_sync()


def test_refinement_is_deterministic_and_checks_its_window():
    runs = []
    for _ in range(2):
        wl, sim, obs, opt, warm, cm = _window(n=32)
        _, _, c1 = sim.sim_refine_elites(warm, obs, opt, steps=3, report=True)
        runs.append((c1.clone(), [t.clone() for t in sim.sim_get_state()]))
        # after the update the snapshot is gone
        sim.optimizer_update(opt, 7)
        with pytest.raises(inhand.InhandError) as e:
            sim.sim_refine_elites(warm, obs, opt, steps=1)
        assert e.value.code == inhand.IH_ERR_STATE
        # a window of the wrong length is refused
        sim.sim_mark_window()
        sim.sim_step_track(warm, obs[0])
        with pytest.raises(inhand.InhandError) as e:
            sim.sim_refine_elites(warm, obs, opt, steps=1)
        assert e.value.code == inhand.IH_ERR_STATE
        sim.close()
    assert torch.equal(runs[0][0], runs[1][0])
    assert all(torch.equal(a, b) for a, b in zip(runs[0][1], runs[1][1]))
