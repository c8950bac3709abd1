"""Pins of the oracle's PD-driven hand and of the full cost (Sec. III-A, III-C).

- PD joint, no contact: the implicit substep recurrence converges at first
  order to the exact solution of I q'' = kp (u - q) - kd q' (matrix
  exponential, scipy) as the substep shrinks, and settles on u exactly;
- statics of a held grasp: once hand and object are at rest, every joint's
  PD force h kp (u - q) equals the moment of the contact impulses on its
  finger's links about its own axis (z_a . sum (p - o_a) x lambda, axes from
  the link frames), and the impulses carry the object's weight with no net
  moment;
- a very stiff PD hand moves the object as the kinematic hand does;
- slip sensing: a box sliding and spinning on the palm pad reports
  translational slip along the sliding direction in the pad's plane and
  rotational slip with the sign of the spin;
- the full cost: zero against itself, each of the ten terms alone by a
  hand-computed value, +inf when diverged, running mean and argmin;
- an optimizer update hands every replaced environment its parent's joints.
"""
import dataclasses

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation as Rot

import oracle as O
from paper_2002_12160_gb300 import workloads as W


def _pd_sim(**kw):
    return dataclasses.replace(W.SimConfig(), hand="pd", **kw)


def _far_object(wl, n=1):
    """The workload's object far above the hand, so nothing touches."""
    pose = np.tile(O.pose8_to7(wl.nominal_pose), (n, 1))
    pose[:, 2] = 0.25
    return O.State(pose, np.zeros((n, 6)), np.tile([0.1, 0.5], (n, 1)))


def test_pd_joint_converges_to_the_continuous_step_response():
    wl = W.make_workload("tracking_box27", n_envs=1, frames=3)
    osc = O.OracleScene(wl.scene)
    D = wl.scene.n_joints
    u = np.linspace(-0.3, 0.6, D)
    q_traj = np.tile(u, (4, 1))
    T = 3 * W.SimConfig().frame_dt
    errs = []
    for ns in (64, 128, 256):
        sim = _pd_sim(substeps=ns, gravity=(0.0, 0.0, 0.0))
        st = _far_object(wl).hand(np.zeros(D))
        O.step_pd(osc, sim, st, q_traj, 0, 3)
        A = np.array([[0.0, 1.0], [-sim.kp / sim.armature, -sim.kd / sim.armature]])
        E = expm(A * T)
        exact = np.array([E @ np.array([-ua, 0.0]) + np.array([ua, 0.0]) for ua in u])
        errs.append(max(np.abs(st.qj[0] - exact[:, 0]).max() / np.abs(u).max(),
                        np.abs(st.qdj[0] - exact[:, 1]).max() / (np.abs(exact[:, 1]).max() + 1e-12)))
    assert errs[2] < 0.05, errs
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2, errs
    # and it settles exactly on u
    sim = _pd_sim(gravity=(0.0, 0.0, 0.0))
    st = _far_object(wl).hand(np.zeros(D))
    O.step_pd(osc, sim, st, np.tile(u, (301, 1)), 0, 300)
    np.testing.assert_allclose(st.qj[0], u, atol=1e-12)


def test_held_grasp_statics():
    wl = W.make_workload("tracking_cyl64", n_envs=2, frames=400)
    sim = _pd_sim()
    osc = O.OracleScene(wl.scene)
    F0 = 40
    q = wl.q_traj.copy()
    q[F0:] = q[F0]   # hold the command from frame F0 on
    pose, theta = O.sample_initial(2, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    st = O.State(pose, np.zeros((2, 6)), theta).hand(q[0])
    for f in range(F0 + 300):
        _, _, last, last_n = O.step_pd(osc, sim, st, q, f, 1, last_cap=256)
    i = int(np.argmin(np.abs(st.vel).max(1)))
    assert np.abs(st.vel[i]).max() < 1e-3 and np.abs(st.qdj[i]).max() < 1e-4 and st.status[i] == 0
    h = sim.frame_dt / sim.substeps
    L = last[i, :last_n[i]]
    assert len(L) > 10
    lam, p = L[:, 4:7], L[:, 1:4]
    m = theta[i, 0]
    np.testing.assert_allclose(lam.sum(0), [0, 0, m * 9.81 * h], atol=1e-5 * m * 9.81 * h)
    moment = np.cross(p - st.pose[i, :3], lam).sum(0)
    assert np.abs(moment).max() < 1e-5 * m * 9.81 * h * 0.05
    lp = O.fk(osc, st.qj[i])
    lhs, rhs = [], []
    for f in range(wl.scene.n_fingers):
        for j in range(4):
            a = 4 * f + j
            if j == 0:
                z, o = np.array([0.0, 0.0, 1.0]), wl.scene.finger_root[f, :3]
            else:
                R = Rot.from_quat(np.r_[lp[1 + a, 4:7], lp[1 + a, 3]]).as_matrix()
                z, o = -R[:, 1], lp[1 + a, :3]
            on = (L[:, 0] >= 1 + a) & (L[:, 0] <= 4 + 4 * f)   # this finger, at or beyond joint a
            rhs.append(sum(z @ np.cross(p[k] - o, lam[k]) for k in np.nonzero(on)[0]))
            lhs.append(h * sim.kp * (q[F0, a] - st.qj[i, a]))
    lhs, rhs = np.array(lhs), np.array(rhs)
    assert np.abs(lhs).max() > 1e-6   # the fingers are loaded
    np.testing.assert_allclose(lhs, rhs, atol=1e-3 * np.abs(lhs).max())


def test_stiff_pd_hand_moves_the_object_like_the_kinematic_hand():
    wl = W.make_workload("tracking_cyl64", n_envs=3, frames=12)
    osc = O.OracleScene(wl.scene)
    pose, theta = O.sample_initial(3, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    kin = O.State(pose, np.zeros((3, 6)), theta)
    stiff = O.State(pose, np.zeros((3, 6)), theta).hand(wl.q_traj[0])
    sim = _pd_sim(kp=1e6, kd=2e2, armature=1e-3)
    soft = O.State(pose, np.zeros((3, 6)), theta).hand(wl.q_traj[0])
    for f in range(12):
        O.step(osc, wl.sim, kin, wl.q_traj, f, 1)
        O.step_pd(osc, sim, stiff, wl.q_traj, f, 1)
        O.step_pd(osc, _pd_sim(), soft, wl.q_traj, f, 1)
    d_stiff = np.abs(stiff.pose[:, :3] - kin.pose[:, :3]).max()
    d_soft = np.abs(soft.pose[:, :3] - kin.pose[:, :3]).max()
    assert np.abs(stiff.qj - wl.q_traj[12]).max() < 1e-3
    assert d_stiff < 1e-3 and d_stiff < 0.5 * d_soft, (d_stiff, d_soft)


@pytest.mark.parametrize("v0,w0,d_exp,spin_pos", [
    ((0.3, 0.0, 0.0), (0.0, 0.0, 2.0), (1.0, 0.0), True),
    ((0.0, -0.3, 0.0), (0.0, 0.0, -2.0), (0.0, -1.0), False),
])
def test_slip_direction_and_spin_on_the_palm_pad(v0, w0, d_exp, spin_pos):
    rows = W.slab9()
    osc = O.OracleScene(W.ground_scene(rows))
    z0 = 0.01 + W.bottom_depth(rows)
    st = O.State(np.array([[0, 0, z0 - 0.0005, 1, 0, 0, 0]], float), np.array([[*v0, *w0]], float),
                 np.array([[0.1, 0.3]])).hand(np.zeros(0))
    obs, _ = O.step_pd(osc, _pd_sim(), st, np.zeros((2, 0)), 0, 1)
    fl = int(obs.flags[0, 0])
    assert fl & 1 and fl & 2
    assert bool(fl & 4) == spin_pos
    # the spin adds w x r at each contact; with the load shifted toward the
    # leading edge that turns the mean slip by about a degree
    np.testing.assert_allclose(obs.slip_d[0, 0], d_exp, atol=0.03)
    assert abs(np.linalg.norm(obs.slip_d[0, 0]) - 1) < 1e-12
    # pad pose of the palm pad: the top centre of the palm, palm rotation
    np.testing.assert_allclose(obs.pad_pose[0, 0], [0, 0, 0.01, 1, 0, 0, 0], atol=1e-15)
    # at rest: contact, no slip
    st2 = O.State(np.array([[0, 0, z0 - 0.0005, 1, 0, 0, 0]], float), np.zeros((1, 6)),
                  np.array([[0.1, 0.3]])).hand(np.zeros(0))
    for f in range(30):
        obs2, _ = O.step_pd(osc, _pd_sim(), st2, np.zeros((31, 0)), f, 1)
    assert obs2.flags[0, 0] == 0 and np.linalg.norm(obs2.forces[0, 0]) > 0.5


def _obs(rng, D=4, P=3):
    q = rng.normal(size=(1, D))
    pp = np.zeros((1, P, 7))
    pp[0, :, :3] = rng.normal(size=(P, 3)) * 0.05
    pp[0, :, 3:] = Rot.random(P, random_state=1).as_quat()[:, [3, 0, 1, 2]]
    c = rng.normal(size=(1, P, 3))
    d = np.zeros((1, P, 2))
    ang = rng.uniform(0, 2 * np.pi, P)
    d[0, :, 0], d[0, :, 1] = np.cos(ang), np.sin(ang)
    fl = np.zeros((1, P), np.int32)
    return O.Obs(q, pp, c, d, fl)


def _cost(sim, a, b, status=0):
    c_sum = np.zeros(1)
    _, _, c = O.cost_full(sim, a, b, np.array([status]), c_sum, 1)
    return c[0]


def test_full_cost_terms_by_hand():
    rng = np.random.default_rng(3)
    w = tuple(float(2 + k) for k in range(10))   # distinct weights expose a swapped term
    sim = dataclasses.replace(W.SimConfig(), w_full=w, tau=0.02)
    g = _obs(rng)
    g.forces[0] = [[0.5, 0, 0], [0, 0.001, 0], [0, 0, 1.0]]   # pads 0, 2 in contact, 1 not
    g.flags[0] = [1 | 2 | 4, 0, 1]
    same = O.Obs(*(np.copy(x) for x in (g.q, g.pad_pose, g.forces, g.slip_d, g.flags)))
    assert _cost(sim, same, g) < 1e-14   # the rotation term of q^-1 q rounds to ~1e-16

    def alt(**kw):
        o = O.Obs(*(np.copy(x) for x in (g.q, g.pad_pose, g.forces, g.slip_d, g.flags)))
        for k, v in kw.items():
            v(getattr(o, k))
        return o

    dq = np.array([0.03, -0.04, 0, 0])
    assert np.isclose(_cost(sim, alt(q=lambda a: a.__iadd__(dq)), g), w[0] * 0.05, rtol=1e-12)
    assert np.isclose(_cost(sim, alt(pad_pose=lambda a: a[0, 1, :3].__iadd__([0.003, 0, 0.004])), g),
                      w[1] * 0.005, rtol=1e-12)
    th = 0.3
    rot = lambda a: a[0, 2, 3:].__setitem__(slice(None), (Rot.from_quat(np.r_[a[0, 2, 4:7], a[0, 2, 3]]) *
                                                          Rot.from_rotvec([0, th, 0])).as_quat()[[3, 0, 1, 2]])
    assert np.isclose(_cost(sim, alt(pad_pose=rot), g), w[2] * th, rtol=1e-9)
    # pad 1 goes into contact: mismatch w4
    assert np.isclose(_cost(sim, alt(forces=lambda a: a[0, 1].__setitem__(slice(None), [0, 0.5, 0])), g), w[3])
    # pad 0 stronger and turned by 90 degrees: w5 |dM| + w6 angle
    assert np.isclose(_cost(sim, alt(forces=lambda a: a[0, 0].__setitem__(slice(None), [0, 0.8, 0])), g),
                      w[4] * 0.3 + w[5] * np.pi / 2, rtol=1e-12)
    # pad 1 stays out of contact but changes magnitude: only w5 |dM| (no angle)
    assert np.isclose(_cost(sim, alt(forces=lambda a: a[0, 1].__setitem__(slice(None), [0.004, 0, 0])), g),
                      w[4] * 0.003, rtol=1e-9)
    # pad 1 starts slipping: w7; pad 0's slip direction turned by 60 degrees: w8 pi/3
    assert np.isclose(_cost(sim, alt(flags=lambda a: a.__setitem__((0, 1), 1)), g), w[6])
    turn = lambda a: a[0, 0].__setitem__(slice(None), [np.cos(np.arctan2(a[0, 0, 1], a[0, 0, 0]) + np.pi / 3),
                                                       np.sin(np.arctan2(a[0, 0, 1], a[0, 0, 0]) + np.pi / 3)])
    assert np.isclose(_cost(sim, alt(slip_d=turn), g), w[7] * np.pi / 3, rtol=1e-9)
    # pad 2 slips in both: its reversed direction counts pi
    assert np.isclose(_cost(sim, alt(slip_d=lambda a: a[0, 2].__imul__(-1.0)), g), w[7] * np.pi, rtol=1e-9)
    # pad 1 (no slip in either) direction is ignored
    assert _cost(sim, alt(slip_d=lambda a: a[0, 1].__imul__(-1.0)), g) < 1e-14
    # rotational slip: pad 2 starts spinning -> w9; pad 0 spins the other way -> w10
    assert np.isclose(_cost(sim, alt(flags=lambda a: a.__setitem__((0, 2), 1 | 2)), g), w[8])
    assert np.isclose(_cost(sim, alt(flags=lambda a: a.__setitem__((0, 0), 1 | 2)), g), w[9])
    # diverged: +inf
    assert _cost(sim, same, g, status=O.ESCAPED) == np.inf


def test_full_cost_running_mean_and_argmin():
    rng = np.random.default_rng(4)
    sim = W.SimConfig()
    g = _obs(rng)
    n = 5
    many = O.Obs(np.repeat(g.q, n, 0), np.repeat(g.pad_pose, n, 0), np.repeat(g.forces, n, 0),
                 np.repeat(g.slip_d, n, 0), np.repeat(g.flags, n, 0))
    many.q[:, 0] += np.array([0.3, 0.1, 0.0, 0.2, 0.0])
    c_sum = np.zeros(n)
    i, cm, c = O.cost_full(sim, many, g, np.zeros(n, np.int32), c_sum, 1)
    assert i == 2 and cm[4] < 1e-14
    i, cm, c2 = O.cost_full(sim, many, g, np.array([0, 0, O.ESCAPED, 0, 0], np.int32), c_sum, 2)
    assert i == 4 and np.isinf(cm[2])
    np.testing.assert_allclose(cm[[0, 1, 3]], c[[0, 1, 3]], rtol=1e-15)


def test_optimizer_copies_the_parents_hand():
    wl = W.make_workload("tracking_cyl64", n_envs=40, frames=4)
    pose, theta = O.sample_initial(40, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    st = O.State(pose, np.zeros((40, 6)), theta).hand(wl.q_traj[0])
    st.qj += np.arange(40)[:, None] * 1e-3
    before = st.qj.copy()
    C = np.random.default_rng(0).uniform(0, 1, 40)
    _, parent, _ = O.optimizer(wl.opt, st, C, wl.seed, 0)
    np.testing.assert_array_equal(st.qj, before[parent])
    assert (parent != np.arange(40)).any()
    _, parent2, _ = O.softmax_update(dataclasses.replace(wl.opt, kind="reps"), st, C, wl.seed, 1)
    np.testing.assert_array_equal(st.qj, before[parent][parent2])
