"""Pins of the oracle's dynamics step against closed forms and invariants.

Each test fixes a quantity that the mathematics of the step determines without
reference to the oracle's code: the discrete free-fall and constant-spin
solutions of symplectic Euler with the exact rotation update, the resting
contact force m g at the solver's fixed point, the slide-to-stop distance of
Coulomb friction, momentum conservation without friction, and the mass
invariance of a kinematically driven scene.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2002_12160_gb300 import workloads as W

SIM = W.SimConfig()
H = SIM.frame_dt / SIM.substeps
G = 9.81


def _one(pose7, vel6, m, mu):
    return O.State(np.array([pose7], float), np.array([vel6], float), np.array([[m, mu]], float))


def test_free_fall_matches_discrete_closed_form():
    """No contact: v_k = v0 + k h g, x_n = x0 + n h v0 + h^2 g n (n + 1) / 2."""
    osc = O.OracleScene(W.ground_scene(W.box27()))
    x0 = np.array([0.01, -0.02, 0.20])
    v0 = np.array([0.1, -0.05, 0.3])
    st = _one([*x0, 1, 0, 0, 0], [*v0, 0, 0, 0], 0.1, 0.5)
    frames = 3
    O.step(osc, SIM, st, np.zeros((frames + 1, 0)), 0, frames)
    n = frames * SIM.substeps
    g = np.array([0, 0, -G])
    x_ref = x0 + n * H * v0 + H * H * g * n * (n + 1) / 2
    np.testing.assert_allclose(st.pose[0, :3], x_ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(st.vel[0, :3], v0 + n * H * g, rtol=0, atol=1e-13)


def test_constant_spin_matches_rotation_exponential():
    """No contact, no gyroscopic term: R_n = exp(n h [w]x) R_0 (left, world frame)."""
    osc = O.OracleScene(W.ground_scene(W.box27()))
    w = np.array([1.3, -0.4, 2.2])
    r0 = Rotation.from_rotvec([0.2, 0.1, -0.3])
    q0 = r0.as_quat(scalar_first=True)
    st = _one([0, 0, 0.2, *q0], [0, 0, 0, *w], 0.1, 0.5)
    frames = 2
    O.step(osc, SIM, st, np.zeros((frames + 1, 0)), 0, frames)
    n = frames * SIM.substeps
    ref = Rotation.from_rotvec(n * H * w) * r0
    got = Rotation.from_quat(st.pose[0, 3:], scalar_first=True)
    assert (got.inv() * ref).magnitude() < 1e-12
    np.testing.assert_allclose(st.vel[0, 3:], w, rtol=0, atol=0)


def test_resting_box_supports_exactly_mg_without_drift():
    """A box of 27 spheres settled on the ground: sum of normal forces = m g.

    Started 1 mm deep (below the allowed slop), the recovery bias lifts it to
    the fixed point at depth = slop, where the velocity is zero and the
    support force is exactly the weight.
    """
    rows = W.box27()
    osc = O.OracleScene(W.ground_scene(rows))
    m = 0.17
    z0 = 0.01 + W.bottom_depth(rows)
    st = _one([0, 0, z0 - 0.001, 1, 0, 0, 0], [0, 0, 0, 0, 0, 0], m, 0.6)
    frames = 300
    forces, diag = O.step(osc, SIM, st, np.zeros((frames + 1, 0)), 0, frames)
    # the palm pad (link 0) receives the object's weight
    np.testing.assert_allclose(forces[0, 0], [0, 0, -m * G], rtol=1e-9, atol=1e-12)
    assert np.all(np.abs(st.vel[0]) < 1e-9)
    assert abs((st.pose[0, 2] - z0) + SIM.slop) < 1e-6
    assert diag[0, 0] == 9 * SIM.substeps  # the 9 bottom spheres touch


@pytest.mark.parametrize("mu,v0", [(0.5, 1.0), (0.3, 0.6), (1.0, 2.0)])
def test_slide_to_stop_distance(mu, v0):
    """Sliding slab decelerates at mu g: distance h sum_k (v0 - k mu g h) ~ v0^2/(2 mu g)."""
    rows = W.slab9()
    osc = O.OracleScene(W.ground_scene(rows))
    z0 = 0.01 + W.bottom_depth(rows)
    st = _one([0, 0, z0, 1, 0, 0, 0], [0, 0, 0, 0, 0, 0], 0.2, mu)
    q = np.zeros((200, 0))
    O.step(osc, SIM, st, q, 0, 30)          # settle on the ground
    x_start = st.pose[0, 0]
    st.vel[0, 0] = v0
    O.step(osc, SIM, st, q, 0, 60)
    dist = st.pose[0, 0] - x_start
    n = int(math.floor(v0 / (mu * G * H)))
    discrete = H * sum(v0 - k * mu * G * H for k in range(1, n + 1))
    assert abs(dist - v0 ** 2 / (2 * mu * G)) < v0 * H + 1e-6
    assert abs(dist - discrete) < 2e-4 * discrete
    assert abs(st.vel[0, 0]) < 1e-9


def test_frictionless_contact_conserves_horizontal_momentum():
    rows = W.slab9()
    osc = O.OracleScene(W.ground_scene(rows))
    z0 = 0.01 + W.bottom_depth(rows)
    v0 = np.array([0.06, -0.04])
    st = _one([0, 0, z0, 1, 0, 0, 0], [*v0, 0, 0, 0, 0], 0.2, 0.0)
    forces, diag = O.step(osc, SIM, st, np.zeros((41, 0)), 0, 40)
    assert diag[0, 0] > 0
    np.testing.assert_allclose(st.vel[0, :2], v0, rtol=1e-12, atol=0)
    assert np.all(np.abs(st.vel[0, 3:]) < 1e-9)
    assert abs(forces[0, 0, 0]) < 1e-12 and abs(forces[0, 0, 1]) < 1e-12


def test_grasp_dynamics_are_mass_invariant():
    """Kinematic hand + gravity: doubling m leaves the motion unchanged and doubles forces."""
    wl = W.make_workload("tracking_box27", n_envs=4, frames=40)
    osc = O.OracleScene(wl.scene)
    pose, theta = O.sample_initial(4, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    a = O.State(pose, np.zeros((4, 6)), theta)
    theta2 = theta.copy()
    theta2[:, 0] *= 2
    b = O.State(pose, np.zeros((4, 6)), theta2)
    fa, da = O.step(osc, wl.sim, a, wl.q_traj, 0, 40)
    fb, db = O.step(osc, wl.sim, b, wl.q_traj, 0, 40)
    assert da[:, 0].sum() > 0
    np.testing.assert_allclose(a.pose, b.pose, rtol=0, atol=1e-9)
    np.testing.assert_allclose(2 * fa, fb, rtol=1e-6, atol=1e-9)


def test_identical_environments_give_identical_observations():
    """The ground-truth environment compared with itself has zero cost every frame."""
    wl = W.make_workload("tracking_box27", n_envs=2, frames=30)
    osc = O.OracleScene(wl.scene)
    nom = O.pose8_to7(wl.nominal_pose)
    st = O.State(np.array([nom, nom]), np.zeros((2, 6)), np.array([wl.theta_gt, wl.theta_gt]))
    c_sum = np.zeros(2)
    for f in range(30):
        forces, _ = O.step(osc, wl.sim, st, wl.q_traj, f, 1)
        i, c_mean, _ = O.cost(wl.sim, forces, forces[0], st.status, c_sum, f + 1)
    assert np.all(c_mean == 0.0) and i == 0


def test_escaped_object_is_flagged_and_frozen():
    osc = O.OracleScene(W.ground_scene(W.box27()))
    st = _one([0, 0, 0.29, 1, 0, 0, 0], [0, 0, 3.0, 0, 0, 0], 0.1, 0.5)
    O.step(osc, SIM, st, np.zeros((4, 0)), 0, 1)
    assert st.status[0] & O.ESCAPED
    frozen = st.pose.copy()
    O.step(osc, SIM, st, np.zeros((4, 0)), 1, 2)
    np.testing.assert_array_equal(st.pose, frozen)


def test_contact_overflow_is_flagged():
    wl = W.make_workload("tracking_cyl64", n_envs=1, frames=2)
    wl.sim.c_max = 4
    osc = O.OracleScene(wl.scene)
    st = O.State(O.pose8_to7(wl.nominal_pose)[None], np.zeros((1, 6)), np.array([[0.1, 0.5]]))
    O.step(osc, wl.sim, st, wl.q_traj, 0, 1)
    assert st.status[0] & O.OVERFLOW
