"""GPU adjoint at the benchmarked size against the FP64 adjoint oracle.

The differentiable-tracking workload as bench.py times it: N = 1024
cylinders, a 30-frame horizon checkpointed every 10 frames and recomputed
between checkpoints, the automatic kernel shape (one warp per environment, two
register contacts per thread and the rest from scratch memory) and the
whole-segment tape, from the GPU's state after 20 frames. The oracle
differentiates sampled environments one by one from the same state widened to
FP64. Sampled environments hold more than 64 contacts in some substep (so the
scratch-memory path runs) and their oracle trajectory stays farther than
1e-6 m from every contact and pad threshold (closer, FP32 and FP64 may keep
different contact sets). Tolerances as the N = 4 test: 1e-3 relative per
block (position, rotation, m, mu) with an absolute floor of 1e-3 of the
environment's largest block norm, 1e-3 relative in the cost.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2002_12160_gb300 import workloads as W

from gpu_common import FRAGILE, dev, oracle_state, scene32, sim32, start, torch

pytestmark = pytest.mark.gpu

N, WARM, H, K = 1024, 20, 30, 10
SAMPLES = 6
BLOCKS = [slice(0, 3), slice(3, 6), slice(6, 7), slice(7, 8)]


def test_full_size_adjoint_matches_oracle_on_samples():
    wl = W.make_workload("tracking_cyl64", n_envs=N, frames=WARM + H + 2)
    sim = start(wl, n=N, frames=WARM + H + 2)
    sim.sim_step(0, WARM)
    st = oracle_state(sim.sim_get_state())
    sc, sm = scene32(wl.scene), sim32(wl.sim)
    osc = O.OracleScene(sc)
    gt = O.State(st.pose[:1], st.vel[:1], np.array([wl.theta_gt], np.float64))
    probe = O.State(st.pose, st.vel, st.theta)
    obs, fragile, frame_contacts = [], np.zeros(N, bool), np.zeros(N)
    for k in range(H):
        f, _ = O.step(osc, sm, gt, wl.q_traj, WARM + k, 1)
        obs.append(f[0])
        _, diag = O.step(osc, sm, probe, wl.q_traj, WARM + k, 1)
        fragile |= (diag[:, 2] < FRAGILE) | (diag[:, 3] < FRAGILE) | (diag[:, 4] < FRAGILE)
        frame_contacts = np.maximum(frame_contacts, diag[:, 0])
    obs = np.asarray(obs, np.float32)

    d = dev()
    cost, grad, _ = sim.sim_adjoint(WARM, torch.from_numpy(obs).to(d), checkpoint_every=K)
    cost, grad = cost.cpu().numpy(), grad.cpu().numpy().astype(np.float64)
    assert np.isfinite(cost).all() and np.isfinite(grad).all()

    # a frame's contacts summed over its substeps above substeps x 64: some
    # substep held more than the 64 register contacts of a one-warp group
    heavy = frame_contacts > wl.sim.substeps * 64
    order = np.random.default_rng(5).permutation(N)
    picked = [int(i) for i in order if heavy[i] and not fragile[i]][:SAMPLES]
    assert len(picked) >= 4, (int(heavy.sum()), int((~fragile).sum()))
    errs = []
    for i in picked:
        c_or, g_or, _, _, _ = A.horizon(sc, sm, st.pose[i], st.vel[i], st.theta[i], wl.q_traj, WARM, H,
                                        obs.astype(np.float64))
        assert abs(cost[i] - c_or) <= 1e-3 * abs(c_or) + 1e-6, (i, cost[i], c_or)
        floor = 1e-3 * max(np.linalg.norm(g_or[b]) for b in BLOCKS)
        for b in BLOCKS:
            err = np.linalg.norm(grad[i, b] - g_or[b])
            errs.append(err / max(np.linalg.norm(g_or[b]), floor))
            assert err <= 1e-3 * np.linalg.norm(g_or[b]) + floor, (i, b, grad[i, b], g_or[b])
    print(f"full-size adjoint: {len(picked)} environments, largest relative block error {max(errs):.2e}")
    sim.close()
