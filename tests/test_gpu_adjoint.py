"""GPU adjoint (sim_adjoint through the C ABI) against the FP64 adjoint oracle.

Both sides start from the same state -- the GPU's FP32 state after a warm-up,
widened exactly to FP64 -- and differentiate the force term of the tracking
cost over a 5-frame horizon with respect to the initial position, rotation
tangent, mass and friction, with the same backward-only smoothing. Tolerance:
1e-3 relative per block (position, rotation, m, mu), with an absolute floor of
1e-3 of the environment's largest block norm. Environments whose horizon
passes within 1e-6 m of a contact or pad threshold are excluded and counted.
Every kernel shape is checked: four warps and one register contact per
thread, and one warp with one or two -- the cylinder's 60-100 contacts per
substep then also run the path that keeps the contacts past the register
slots in scratch memory.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2002_12160_gb300 import workloads as W

from gpu_common import FRAGILE, dev, oracle_state, scene32, sim32, start, torch

pytestmark = pytest.mark.gpu

WARM, H = 18, 5
BLOCKS = [slice(0, 3), slice(3, 6), slice(6, 7), slice(7, 8)]


def _setup(n=4, name="tracking_cyl64"):
    wl = W.make_workload(name, n_envs=n, frames=WARM + H + 2)
    sim = start(wl, n=n, frames=WARM + H + 2)
    sim.sim_step(0, WARM)
    st = oracle_state(sim.sim_get_state())
    sc, sm = scene32(wl.scene), sim32(wl.sim)
    osc = O.OracleScene(sc)
    # observations: the ground-truth parameters from environment 0's state (oracle)
    gt = O.State(st.pose[:1], st.vel[:1], np.array([wl.theta_gt], np.float64))
    obs, fragile = [], np.zeros(n, bool)
    probe = O.State(st.pose, st.vel, st.theta)
    _setup.frame_contacts = np.zeros(n)   # most contacts of a frame (summed over its substeps) per env
    for k in range(H):
        f, _ = O.step(osc, sm, gt, wl.q_traj, WARM + k, 1)
        obs.append(f[0])
        _, diag = O.step(osc, sm, probe, wl.q_traj, WARM + k, 1)
        fragile |= (diag[:, 2] < FRAGILE) | (diag[:, 3] < FRAGILE) | (diag[:, 4] < FRAGILE)
        _setup.frame_contacts = np.maximum(_setup.frame_contacts, diag[:, 0])
    obs = np.asarray(obs, np.float32)
    return wl, sim, st, sc, sm, obs, fragile


SHAPES = [(4, 1), (1, 1), (1, 2)]   # (warps per environment, register contacts per thread)


def test_adjoint_matches_oracle():
    wl, sim, st, sc, sm, obs, fragile = _setup()
    # some substep holds more contacts than the one-warp shapes keep in registers
    substeps = wl.sim.substeps
    assert _setup.frame_contacts.max() > substeps * 32 * max(pl for gw, pl in SHAPES if gw == 1)
    d = dev()
    gpu = {}
    for gw, pl in SHAPES:
        sim.sim_set_adjoint_variant(gw, pl)
        cost, grad, _ = sim.sim_adjoint(WARM, torch.from_numpy(obs).to(d), checkpoint_every=2)
        gpu[gw, pl] = (cost.cpu().numpy(), grad.cpu().numpy().astype(np.float64))
    sim.sim_set_adjoint_variant(0, 0)
    checked = 0
    for i in range(st.n):
        if fragile[i]:
            continue
        c_or, g_or, _, _, _ = A.horizon(sc, sm, st.pose[i], st.vel[i], st.theta[i], wl.q_traj, WARM, H,
                                        obs.astype(np.float64))
        floor = 1e-3 * max(np.linalg.norm(g_or[b]) for b in BLOCKS)
        for shape, (cost, grad) in gpu.items():
            assert np.isfinite(cost[i]) and abs(cost[i] - c_or) <= 1e-3 * abs(c_or) + 1e-6, (shape, i, cost[i], c_or)
            for b in BLOCKS:
                err = np.linalg.norm(grad[i, b] - g_or[b])
                assert err <= 1e-3 * np.linalg.norm(g_or[b]) + floor, (shape, i, b, grad[i, b], g_or[b])
        checked += 1
    assert checked >= 3


def test_adjoint_shape_arguments():
    wl = W.make_workload("tracking_cyl64", n_envs=4, frames=4)
    sim = start(wl, n=4, frames=4)
    for gw, pl in [(2, 1), (4, 2), (1, 4), (1, 0), (0, 1), (-1, 1)]:
        with pytest.raises(RuntimeError):
            sim.sim_set_adjoint_variant(gw, pl)
    for gw, pl in SHAPES + [(0, 0)]:
        sim.sim_set_adjoint_variant(gw, pl)
    sim.close()


@pytest.mark.parametrize("shape", [(0, 0), (1, 1)])
def test_checkpoint_interval_tape_mode_and_subset_do_not_change_results(shape):
    wl, sim, st, sc, sm, obs, fragile = _setup()
    d = dev()
    o = torch.from_numpy(obs).to(d)
    sim.sim_set_adjoint_variant(*shape)
    ref_c, ref_g, ref_q = sim.sim_adjoint(WARM, o, checkpoint_every=10, want_quat=True)
    for K in (1, 2, 3):
        c, g, q = sim.sim_adjoint(WARM, o, checkpoint_every=K, want_quat=True)
        assert torch.equal(c, ref_c) and torch.equal(g, ref_g) and torch.equal(q, ref_q), K
    # taping substep by substep (no memory for whole segments) gives the same bits
    sim.sim_set_adjoint_memory(0)
    for K in (2, 10):
        c, g, q = sim.sim_adjoint(WARM, o, checkpoint_every=K, want_quat=True)
        assert torch.equal(c, ref_c) and torch.equal(g, ref_g) and torch.equal(q, ref_q), K
    sim.sim_set_adjoint_memory(16 << 30)
    envs = torch.tensor([3, 1], dtype=torch.int32, device=d)
    c, g, _ = sim.sim_adjoint(WARM, o, envs=envs, checkpoint_every=2)
    assert torch.equal(c, ref_c[[3, 1]]) and torch.equal(g, ref_g[[3, 1]])
    # the state is left unchanged
    before = sim.sim_get_state()
    sim.sim_adjoint(WARM, o)
    after = sim.sim_get_state()
    assert all(torch.equal(a, b) for a, b in zip(before, after))


def test_adjoint_cost_is_the_scored_cost():
    """The adjoint's forward is the step's arithmetic (contact.cuh), contacts
    in the same order and summed in the same lane order as the 32-thread step
    shape: the FP64 costs agree with the scored step's to FP32 rounding (the
    compiler may fuse a multiply-add differently in the two kernels)."""
    wl, sim, st, sc, sm, obs, fragile = _setup()
    d = dev()
    o = torch.from_numpy(obs).to(d)
    sim.sim_set_variant(32, 4)
    c_adj, _, _ = sim.sim_adjoint(WARM, o)
    pose, vel, params, _ = sim.sim_get_state()
    sim.sim_set_state(pose, vel, params)   # also resets nothing but status; start a fresh window
    cm = torch.empty(sim.n, dtype=torch.float64, device=d)
    opt = W.OptConfig()
    sim.sim_step_track(WARM, o[0], cm)
    sim.optimizer_update(opt, 0)   # resets the window (the state changes but only after scoring)
    sim.sim_set_state(pose, vel, params)
    for k in range(H):
        sim.sim_step_track(WARM + k, o[k], cm)
    np.testing.assert_allclose(cm.cpu().numpy() * H, c_adj.cpu().numpy(), rtol=2e-6)


def test_autograd_function_and_invalid_env():
    wl, sim, st, sc, sm, obs, fragile = _setup()
    d = dev()
    from paper_2002_12160_gb300.autograd import tracking_cost
    o = torch.from_numpy(obs).to(d)
    pose, vel, params, _ = sim.sim_get_state()
    _, g_ref, q_ref = sim.sim_adjoint(WARM, o, want_quat=True)
    pose = pose.clone().requires_grad_(True)
    params = params.clone().requires_grad_(True)
    c = tracking_cost(sim, pose, params, vel, WARM, o)
    (2.0 * c).sum().backward()
    assert torch.equal(pose.grad[:, :3], 2.0 * g_ref[:, :3])
    assert torch.equal(pose.grad[:, 4:], 2.0 * q_ref)
    assert torch.equal(params.grad, 2.0 * g_ref[:, 6:])
    # the rotation tangent is the quaternion derivative projected: vec(qbar (x) conj(q)) / 2
    q = pose.detach()[:, 4:].cpu().numpy().astype(np.float64)
    qb = q_ref.cpu().numpy().astype(np.float64)
    w1, v1, w2, v2 = qb[:, 0], qb[:, 1:], q[:, 0], -q[:, 1:]
    vec = w1[:, None] * v2 + w2[:, None] * v1 + np.cross(v1, v2)
    np.testing.assert_allclose(0.5 * vec, g_ref[:, 3:6].cpu().numpy(), rtol=1e-4, atol=1e-6 * np.abs(qb).max())
    # an invalid environment (mass <= 0) has cost +inf and zero gradient
    p2 = params.detach().clone()
    p2[1, 0] = -1.0
    sim.sim_set_state(pose.detach().contiguous(), vel, p2)
    c2, g2, _ = sim.sim_adjoint(WARM, o)
    assert torch.isinf(c2[1]) and torch.all(g2[1] == 0)
    assert torch.isfinite(c2[[0, 2, 3]]).all()


def test_adjoint_matches_oracle_on_uneven_batch():
    """Per-environment shapes (16, 27, 64, 256 spheres; c_max 256) and
    iteration counts (10, 20, 40): each environment's gradient against the
    oracle adjoint of its own shape and iteration count, for every kernel
    shape (the contacts past 32, 64 or 128 register slots run from scratch
    memory)."""
    warm, H = 12, 3
    n = 6
    wl = W.make_workload("uneven_mixed", n_envs=n, frames=warm + H + 2)
    sim = start(wl, n=n, frames=warm + H + 2)
    sim.sim_step(0, warm)
    st = oracle_state(sim.sim_get_state())
    sc, sm = scene32(wl.scene), sim32(wl.sim)
    osc = O.OracleScene(sc)
    obs = np.zeros((H, wl.scene.n_pads, 3), np.float32)
    probe = O.State(st.pose, st.vel, st.theta, wl.shape_id[:n].astype(np.int32), wl.iters[:n].astype(np.int32))
    fragile = np.zeros(n, bool)
    for k in range(H):
        _, diag = O.step(osc, sm, probe, wl.q_traj, warm + k, 1)
        fragile |= (diag[:, 2] < FRAGILE) | (diag[:, 3] < FRAGILE) | (diag[:, 4] < FRAGILE)
    d = dev()
    gpu = {}
    for gw, pl in SHAPES:
        sim.sim_set_adjoint_variant(gw, pl)
        cost, grad, _ = sim.sim_adjoint(warm, torch.from_numpy(obs).to(d), checkpoint_every=2)
        gpu[gw, pl] = (cost.cpu().numpy(), grad.cpu().numpy().astype(np.float64))
    sim.sim_set_adjoint_variant(0, 0)
    checked, shapes = 0, set()
    for i in range(n):
        if fragile[i] or not all(np.isfinite(c[i]) for c, _ in gpu.values()):
            continue
        c_or, g_or, _, _, _ = A.horizon(sc, sm, st.pose[i], st.vel[i], st.theta[i], wl.q_traj, warm, H,
                                        obs.astype(np.float64), shape=int(wl.shape_id[i]), iters=int(wl.iters[i]))
        for shape, (cost, grad) in gpu.items():
            assert abs(cost[i] - c_or) <= 1e-3 * abs(c_or) + 1e-6, (shape, i, cost[i], c_or)
            if c_or == 0.0:
                assert np.all(grad[i] == 0), shape
                continue
            floor = 1e-3 * max(np.linalg.norm(g_or[b]) for b in BLOCKS)
            for b in BLOCKS:
                err = np.linalg.norm(grad[i, b] - g_or[b])
                assert err <= 1e-3 * np.linalg.norm(g_or[b]) + floor, (shape, i, b, grad[i, b], g_or[b])
        if c_or != 0.0:
            checked += 1
            shapes.add(int(wl.shape_id[i]))
    assert checked >= 3 and len(shapes) >= 2


def test_adjoint_of_an_environment_out_of_reach_is_zero():
    """No contact over the horizon: the pad forces are zero whatever the
    initial state, so the cost is sum |o|^2 and every derivative is 0."""
    wl, sim, st, sc, sm, obs, fragile = _setup()
    d = dev()
    pose, vel, params, _ = sim.sim_get_state()
    pose = pose.clone()
    # 12 cm to the side (beyond the palm and the fingers' reach) and 15 cm up:
    # 5 frames of free fall drop it 14 cm, still clear of the hand and inside
    # the 0.3 m escape radius
    pose[0, 0] += 0.12
    pose[0, 2] += 0.15
    vel = torch.zeros_like(vel)
    sim.sim_set_state(pose, vel, params)
    o = torch.from_numpy(obs).to(d)
    cost, grad, gq = sim.sim_adjoint(WARM, o, want_quat=True)
    o64 = obs.astype(np.float64)
    n2 = np.sum(o64 ** 2, axis=2)
    tau = float(np.float32(sm.tau))
    expect = float(np.sum(n2)) * sm.w_force + float(np.sum(n2 > tau * tau)) * sm.w_contact
    assert abs(cost[0].item() - expect) <= 1e-12 * expect, (cost[0].item(), expect)
    assert torch.all(grad[0] == 0) and torch.all(gq[0] == 0)
