"""Pins of the oracle's warm-started solver (each contact's impulse starts from
its (link, sphere) pair's final impulse of the previous substep, zero for new
pairs).

- the fixed point is unchanged: a resting box settles to a support force of
  exactly m g with no drift, as with cold starts;
- warm starting carries the solve across substeps: with one Jacobi iteration
  per substep the resting box comes to rest carrying m g within the slop
  (the impulses accumulate from substep to substep), while the cold-started
  one (one relaxed step from zero reaches only about 1/n_c of the impulse)
  sinks more than ten times the slop before the bias makes up the rest;
- the cache holds exactly the last substep's contact pairs (distinct ids that
  decode to valid (link, sphere) pairs), and an optimizer update drops the
  cache of every environment it replaces.
"""
import dataclasses

import numpy as np

import oracle as O
from paper_2002_12160_gb300 import workloads as W

G = 9.81
SIM = W.SimConfig()


def _one(pose7, vel6, m, mu):
    return O.State(np.array([pose7], float), np.array([vel6], float), np.array([[m, mu]]))


def _resting(iters, warm, frames):
    rows = W.box27()
    osc = O.OracleScene(W.ground_scene(rows))
    m = 0.17
    z0 = 0.01 + W.bottom_depth(rows)
    st = _one([0, 0, z0 - 0.001, 1, 0, 0, 0], [0, 0, 0, 0, 0, 0], m, 0.6)
    sim = dataclasses.replace(SIM, iters=iters, warm_start=warm)
    forces, _ = O.step(osc, sim, st, np.zeros((frames + 1, 0)), 0, frames)
    return forces[0, 0], st, m, z0


def test_warm_start_keeps_the_fixed_point():
    f, st, m, z0 = _resting(20, True, 300)
    np.testing.assert_allclose(f, [0, 0, -m * G], rtol=1e-9, atol=1e-12)
    assert np.all(np.abs(st.vel[0]) < 1e-9)
    assert abs((st.pose[0, 2] - z0) + SIM.slop) < 1e-6


def test_warm_start_converges_across_substeps_with_one_iteration():
    # At rest both carry m g, but where they come to rest differs: the warm
    # solve accumulates the support impulse over substeps and stops inside the
    # zero-bias band [-slop, 0]; one relaxed step from zero delivers only about
    # 1/n_c of it, so the cold-started box sinks until the penetration bias
    # makes up the rest, more than ten times the slop deep. (Left running much
    # longer, that deep equilibrium turns out to be unstable: it tips over.)
    f_warm, st_w, m, z0 = _resting(1, True, 150)
    _, st_c, _, _ = _resting(1, False, 150)
    assert abs(f_warm[2] + m * G) < 1e-6 * m * G, f_warm
    assert -SIM.slop - 1e-9 <= st_w.pose[0, 2] - z0 <= 0.0
    assert st_c.pose[0, 2] - z0 < -10 * SIM.slop
    assert np.all(np.abs(st_w.vel[0]) < 1e-9)


def test_cache_holds_the_last_contacts_and_the_optimizer_drops_replaced_ones():
    wl = W.make_workload("tracking_cyl64", n_envs=24, frames=12)
    wl.sim = dataclasses.replace(wl.sim, warm_start=True)
    osc = O.OracleScene(wl.scene)
    pose, theta = O.sample_initial(24, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    st = O.State(pose, np.zeros((24, 6)), theta)
    _, diag = O.step(osc, wl.sim, st, wl.q_traj, 0, 8)
    assert st.cache_n is not None and np.all(st.cache_n > 0)
    n_links, n_sph = wl.scene.n_links, len(wl.scene.shapes[0])
    for i in range(24):
        ids = st.cache_id[i, :st.cache_n[i]]
        assert len(set(ids.tolist())) == len(ids)
        assert np.all((ids >> 8) < n_links) and np.all((ids & 0xff) < n_sph)
        # the cache has one substep's contacts: diag counts the frame's (both substeps)
        assert st.cache_n[i] <= diag[i, 0]
    C = np.linspace(0.1, 2.4, 24)
    _, parent, _ = O.optimizer(wl.opt, st, C, wl.seed, 0)
    replaced = parent != np.arange(24)
    assert np.all(st.cache_n[replaced] == 0) and np.all(st.cache_n[~replaced] > 0)
