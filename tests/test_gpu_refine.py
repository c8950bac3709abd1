"""Gradient refinement of the elites (sim_refine_elites) on the GPU.

Properties that hold whatever the scene: zero steps change nothing; the
refined window cost never exceeds the unrefined one, and is lower for some
elites; environments that are not elites keep their state bit for bit; the
unrefined cost is the scored window cost (to FP32 rounding); the call is
deterministic; and it refuses a window it did not see start.
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_12160_gb300 import inhand, workloads as W

from gpu_common import dev, start, torch

pytestmark = pytest.mark.gpu

T = 10


def _window(n=64, warm=20, name="tracking_cyl64", T=T):
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
    sim._window_start = (pose, vel, params)
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


# --------------------------------------------------------------- parity with the refinement oracle
# A window of several frames tests ~10^4 sphere-link gaps, so its closest gap to
# the contact margin is typically ~1e-6 m: the one-frame threshold (FRAGILE)
# would leave out most windows. What can flip a branch is the FP32 state's
# distance from the FP64 one, ~3e-9 m after a frame (one-frame parity): a
# window is left out when a gap comes within 1e-7 m of a threshold.
WINDOW_FRAGILE = 1e-7


def _fragile_window(osc, sm, q_traj, f0, T, pose7, vel6, theta):
    """True when the oracle's window from this start passes within
    WINDOW_FRAGILE of a contact-set, pad-membership or palm-face threshold in
    some frame, or puts a pad force within 1e-3 of the contact threshold tau
    (where FP32 and FP64 may take different branches or count a different
    contact mismatch)."""
    st = O.State(pose7[None], vel6[None], theta[None])
    for k in range(T):
        f, diag = O.step(osc, sm, st, q_traj, f0 + k, 1)
        if diag[0, 2] < WINDOW_FRAGILE or diag[0, 3] < WINDOW_FRAGILE or diag[0, 4] < WINDOW_FRAGILE:
            return True
        mag = np.linalg.norm(f[0], axis=1)
        if np.any(np.abs(mag - sm.tau) < 1e-3 * sm.tau):
            return True
    return False


def _check_against_oracle(wl, sim, obs, opt, warm, cm, T, steps, k, order=None, max_checked=None):
    """Refine the window's elites, then compare elites (in `order`, up to
    max_checked of them) with the FP64 refinement oracle; returns (checked,
    skipped)."""
    from oracle import adjoint as A
    from gpu_common import POS_TOL, ROT_TOL, rot_angle, scene32, sim32
    pose0, vel0, par0 = (t.clone() for t in sim._window_start)
    before = [t.clone() for t in sim.sim_get_state()]
    el, c0, c1, acc, sp, spar = sim.sim_refine_elites(warm, obs, opt, steps=steps, detail=True)
    after = sim.sim_get_state()
    el, c0, c1, acc = (t.cpu().numpy() for t in (el, c0, c1, acc))
    sp, spar = sp.cpu().numpy().astype(np.float64), spar.cpu().numpy().astype(np.float64)
    cm = cm.cpu().numpy()
    np.testing.assert_array_equal(el, np.sort(np.argsort(cm, kind="stable")[:k]))
    # the oracle sees what the GPU computes with: FP32 scene, constants, observations and eta
    sc, sm = scene32(wl.scene), sim32(wl.sim)
    osc = O.OracleScene(sc)
    o32 = W.OptConfig(floor_std=tuple(float(np.float32(np.float32(0.5) * np.float32(v))) / 0.5
                                      for v in opt.floor_std),
                      m_range=tuple(float(np.float32(v)) for v in opt.m_range),
                      mu_range=tuple(float(np.float32(v)) for v in opt.mu_range))
    obs64 = obs.cpu().numpy().astype(np.float64)
    p7 = O.pose8_to7(pose0.cpu().numpy())
    v6 = O.vel8_to6(vel0.cpu().numpy())
    th = par0.cpu().numpy().astype(np.float64)
    live_p = O.pose8_to7(after[0].cpu().numpy())
    live_v = O.vel8_to6(after[1].cpu().numpy())
    live_th = after[2].cpu().numpy().astype(np.float64)
    checked, skipped = 0, 0
    for i in (range(len(el)) if order is None else order):
        if max_checked is not None and checked >= max_checked:
            break
        e = el[i]
        r = A.refine_elite(sc, sm, o32, p7[e], v6[e], th[e], wl.q_traj, warm, T, obs64, steps=steps,
                           step_scale=0.5, beta=1e3, width=float(np.float32(1e-3)))
        best_before = np.minimum.accumulate(r["costs"])
        decisive = all(abs(r["costs"][j] - best_before[j - 1]) > 1e-3 * abs(best_before[j - 1])
                       for j in range(1, steps + 1))
        if not decisive or any(_fragile_window(osc, sm, wl.q_traj, warm, T, tp, v6[e], tt)
                               for tp, tt in r["trials"]):
            skipped += 1
            continue
        bits = sum(1 << j for j, a in enumerate(r["accepted"]) if a)
        assert int(acc[i]) == bits, (e, bin(int(acc[i])), r["accepted"], r["costs"])
        assert abs(c0[i] - r["c0"]) <= 1e-3 * abs(r["c0"]), (e, c0[i], r["c0"])
        assert abs(c1[i] - r["best_c"]) <= 1e-3 * abs(r["best_c"]), (e, c1[i], r["best_c"])
        gp = O.pose8_to7(sp[i])
        assert np.linalg.norm(gp[:3] - r["pose7"][:3]) < POS_TOL, (e, gp, r["pose7"])
        assert rot_angle(gp, r["pose7"]) < ROT_TOL, (e, gp, r["pose7"])
        np.testing.assert_allclose(spar[i], r["theta"], rtol=1e-3)
        assert bool(c1[i] < c0[i]) == bool(r["improved"]), e
        if r["improved"]:
            end = r["end"]
            assert np.linalg.norm(live_p[e, :3] - end[:3]) < 5e-5, (e, live_p[e], end[:7])
            assert rot_angle(live_p[e], end[:7]) < 5e-5
            np.testing.assert_allclose(live_th[e], r["theta"], rtol=1e-3)
            assert np.allclose(live_v[e, :3], end[7:10], atol=5e-3)
        else:
            for a_, b_ in zip(before[:3], after[:3]):
                assert torch.equal(a_[int(e)], b_[int(e)])
        checked += 1
    return checked, skipped


def test_refinement_matches_oracle():
    """sim_refine_elites against the FP64 refinement oracle, elite by elite,
    from the GPU's window-start state widened exactly to FP64: the elites, the
    accept/halve decision of every evaluation, the refined window-start state
    (1e-5 m, 1e-5 rad, 1e-3 relative in m and mu), the unrefined and best window
    costs (1e-3 relative), and what is committed: an improved elite's live state
    is its best trial's window-end state (5e-5 m / rad after the window's five
    frames), its parameters the best ones and its window sum the best cost; the
    others keep their scored state bit for bit. Elites whose decisions are not
    decisive (a trial's cost within 1e-3 of the best before it) or whose trial
    windows pass near a branch threshold are skipped and counted."""
    n, T5, steps = 64, 5, 3
    wl, sim, obs, opt, warm, cm = _window(n=n, T=T5)
    k = 16   # elite_frac 0.25 of 64
    checked, skipped = _check_against_oracle(wl, sim, obs, opt, warm, cm, T5, steps, k)
    assert checked >= k // 2, (checked, skipped)


def test_full_size_refinement_matches_oracle_on_samples():
    """The refinement as bench.py times it -- 1024 cylinders, a 10-frame
    window, the optimizer's 10 % elites (102, four warps each), 3 steps --
    against the FP64 refinement oracle on sampled elites, with the checks
    and exclusions of the test above."""
    n, steps = 1024, 3
    wl, sim, obs, opt, warm, cm = _window(n=n, T=T)
    opt.elite_frac = 0.1
    k = int(np.floor(0.1 * n))
    order = np.random.default_rng(7).permutation(k)
    checked, skipped = _check_against_oracle(wl, sim, obs, opt, warm, cm, T, steps, k, order=order, max_checked=6)
    assert checked >= 4, (checked, skipped)
