"""Pins of the refinement oracle (oracle/adjoint.py: refine_rule, refine_elite).

The refinement of an elite's window-start state z takes normalised steepest
descent steps in coordinates scaled by eta, keeps a step only when the cost
strictly drops and otherwise halves the step. On costs whose minimiser and
geometry are known, the sequence of decisions and the final state follow from
the mathematics alone:

1. a cost isotropic in the scaled coordinates, |(z - z*) / eta|^2, started
   2.3 scaled units from z* in any direction: steepest descent runs along the
   ray through z*, one scaled unit per step (2.3 -> 1.3 -> 0.3), the third
   step overshoots to -0.7 (a higher cost: halved), and the fourth, half as
   long, lands at -0.2 (kept): decisions (kept, kept, kept, halved, kept) and
   the best state 0.2 units past z* on the ray;
2. the same for a rotation: the squared angle to R*, started at
   exp(2.3 eta_r a) R* with R* not the identity; steps must be applied on the
   left (world frame) to walk the angle along the same axis;
3. the mass clamp: a minimiser below the lowest allowed mass stops the walk
   at the bound, after which no step lowers the cost;
4. a zero gradient (a free-falling object never touches the hand, so every
   pad force is zero whatever its start): no step moves the state, every
   trial is halved, the cost is sum_l w_f |o_l|^2 + w_c #{|o_l| > tau}.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import adjoint as A
from paper_2002_12160_gb300 import workloads as W

pytest.importorskip("torch")

ETA = 0.5 * np.array(W.OptConfig().floor_std)
M_RANGE, MU_RANGE = (0.01, 1.0), (0.05, 2.0)


def _state(x=(0.0, 0.0, 0.05), q=(1.0, 0.0, 0.0, 0.0), m=0.2, mu=0.6):
    return np.array([*x, *q], float), np.array([m, mu], float)


def _z(p7, th):
    """Position, and mass and friction, as one 5-vector (rotation handled apart)."""
    return np.concatenate([p7[:3], th])


def test_isotropic_quadratic_walks_the_ray_to_the_minimum():
    rng = np.random.default_rng(3)
    eta5 = np.concatenate([ETA[:3], ETA[6:]])
    p0, th0 = _state()
    z_star = _z(p0, th0).copy()
    d = rng.normal(size=5)
    d /= np.linalg.norm(d)                       # unit direction in scaled coordinates
    z_start = z_star + 2.3 * eta5 * d
    p_start, th_start = p0.copy(), th0.copy()
    p_start[:3], th_start[:] = z_start[:3], z_start[3:]

    def evaluate(p, th):
        u = (_z(p, th) - z_star) / eta5
        g = np.zeros(8)
        g[:3] = 2 * u[:3] / eta5[:3]
        g[6:] = 2 * u[3:] / eta5[3:]
        return float(u @ u), g, None

    r = A.refine_rule(evaluate, p_start, th_start, ETA, 4, M_RANGE, MU_RANGE)
    assert r["accepted"] == [True, True, True, False, True]
    assert r["scales"] == [1.0, 1.0, 1.0, 0.5, 0.5]
    np.testing.assert_allclose(r["costs"], [5.29, 1.69, 0.09, 0.49, 0.04], rtol=1e-9)
    np.testing.assert_allclose(_z(r["pose7"], r["theta"]), z_star - 0.2 * eta5 * d, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(r["pose7"][3:], p0[3:])   # no rotation gradient, no rotation
    assert r["improved"] and r["best_c"] == r["costs"][4]


def test_rotation_steps_act_on_the_left():
    eta_r = ETA[3]
    assert np.all(ETA[3:6] == eta_r)
    r_star = Rotation.from_rotvec([0.4, -0.9, 0.3])
    a = np.array([1.0, 2.0, -2.0]) / 3.0
    r0 = Rotation.from_rotvec(2.3 * eta_r * a) * r_star
    p0, th0 = _state(q=r0.as_quat(scalar_first=True))

    def angle(p):
        return (Rotation.from_quat(p[3:7], scalar_first=True) * r_star.inv()).magnitude()

    def evaluate(p, th):
        # gradient of angle^2 w.r.t. a left rotation vector, by central differences
        g = np.zeros(8)
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-7
            qp = (Rotation.from_rotvec(e) * Rotation.from_quat(p[3:7], scalar_first=True))
            qm = (Rotation.from_rotvec(-e) * Rotation.from_quat(p[3:7], scalar_first=True))
            g[3 + k] = ((qp * r_star.inv()).magnitude() ** 2 - (qm * r_star.inv()).magnitude() ** 2) / 2e-7
        return angle(p) ** 2, g, None

    r = A.refine_rule(evaluate, p0, th0, ETA, 4, M_RANGE, MU_RANGE)
    assert r["accepted"] == [True, True, True, False, True]
    # each step turned the object about the same axis through R*
    assert abs(angle(r["pose7"]) - 0.2 * eta_r) < 1e-9
    rel = Rotation.from_quat(r["pose7"][3:7], scalar_first=True) * r_star.inv()
    np.testing.assert_allclose(rel.as_rotvec(), -0.2 * eta_r * a, atol=1e-9)
    np.testing.assert_array_equal(r["pose7"][:3], p0[:3])


def test_mass_walk_stops_at_its_lower_bound():
    p0, th0 = _state(m=M_RANGE[0] + 0.5 * ETA[6])
    m_star = M_RANGE[0] - 1.0

    def evaluate(p, th):
        g = np.zeros(8)
        g[6] = 2 * (th[0] - m_star)
        return (th[0] - m_star) ** 2, g, None

    r = A.refine_rule(evaluate, p0, th0, ETA, 3, M_RANGE, MU_RANGE)
    assert r["accepted"] == [True, True, False, False]
    assert r["theta"][0] == M_RANGE[0] and r["theta"][1] == th0[1]
    assert r["scales"] == [1.0, 1.0, 0.5, 0.25]


def test_free_fall_window_has_no_gradient_and_never_moves():
    """An object 20 cm to the side of the hand (inside the escape radius)
    falls freely for the whole window: every simulated pad force is exactly
    zero whatever its start, so the window cost is the observations' own and
    the gradient vanishes."""
    wl = W.make_workload("tracking_box27", n_envs=1, frames=8)
    T = 5
    rng = np.random.default_rng(7)
    obs = rng.normal(scale=0.05, size=(T, wl.scene.n_pads, 3))
    obs[:, 0] = 0.0                               # one pad off in every frame
    p0, th0 = _state(x=(0.2, 0.0, 0.15))
    r = A.refine_elite(wl.scene, wl.sim, wl.opt, p0, np.zeros(6), th0, wl.q_traj, 0, T, obs, steps=3)
    norms2 = (obs ** 2).sum(-1)
    c_ref = wl.sim.w_force * norms2.sum() + wl.sim.w_contact * (norms2 > wl.sim.tau ** 2).sum()
    assert abs(r["c0"] - c_ref) <= 1e-12 * c_ref
    assert r["accepted"] == [True, False, False, False]
    assert r["scales"] == [1.0, 0.5, 0.25, 0.125]
    np.testing.assert_array_equal(r["pose7"], p0)
    np.testing.assert_array_equal(r["theta"], th0)
    assert not r["improved"] and np.all(r["grad"] == 0.0)
    # the end state is the discrete free fall of the window
    n = T * wl.sim.substeps
    h = wl.sim.frame_dt / wl.sim.substeps
    z_ref = 0.15 + h * h * wl.sim.gravity[2] * n * (n + 1) / 2
    assert abs(r["end"][2] - z_ref) < 1e-13
    assert math.isfinite(r["best_c"])
