"""The seeded synthetic inputs match the workloads they stand in for.

Each configuration's geometry, sizes, trajectory and sampling ranges are
checked against the stated workload (the box of 27 spheres of 8.3 mm on a
3x3x3 grid filling a 5 cm cube, the cylinder of radius 3 cm and height 8 cm
from 64 spheres, the palm of 8 x 8 x 2 cm with 4 or 5 fingers of 4 capsule
links 3 cm long and 8 mm in radius, 8 or 16 pads, the uneven batch's shape
and iteration mix, the mug's 4 substeps and 40 iterations), and the
generator is deterministic in its seed. These properties hold by
construction of the inputs; none of the method's arithmetic is involved.
"""
import math

import numpy as np
import pytest

from paper_2002_12160_gb300 import workloads as W


def _extent(rows):
    """Per-axis (min, max) of the sphere surfaces of a body-frame cluster."""
    lo = (rows[:, :3] - rows[:, 3:4]).min(axis=0)
    hi = (rows[:, :3] + rows[:, 3:4]).max(axis=0)
    return lo, hi


def test_box_fills_a_5cm_cube_with_a_3x3x3_grid():
    rows = W.box27()
    assert rows.shape == (27, 4)
    assert np.allclose(rows[:, 3], 0.0083)
    lo, hi = _extent(rows)
    assert np.allclose(lo, -0.025, atol=1e-12) and np.allclose(hi, 0.025, atol=1e-12)
    for ax in range(3):
        assert len(np.unique(np.round(rows[:, ax], 12))) == 3
    assert np.allclose(rows[:, :3].mean(axis=0), 0.0, atol=1e-15)


def test_cylinder_envelope_is_r3cm_h8cm():
    rows = W.cylinder64()
    assert rows.shape == (64, 4)
    assert np.allclose(rows[:, 3], 0.008)
    radial = np.hypot(rows[:, 0], rows[:, 1]) + rows[:, 3]
    assert np.allclose(radial, 0.03, atol=1e-12)
    lo, hi = _extent(rows)
    assert math.isclose(lo[2], -0.04, abs_tol=1e-12) and math.isclose(hi[2], 0.04, abs_tol=1e-12)
    assert len(np.unique(np.round(rows[:, 2], 12))) == 4   # four rings of 16


def test_other_objects_have_their_sphere_counts():
    assert W.sphere16().shape == (16, 4)
    assert W.l_composite256().shape == (256, 4)
    mug = W.mug128()
    assert mug.shape == (128, 4)
    # the shell of 7 x 16 and the handle of 16 smaller spheres
    assert (mug[:, 3] == 0.006).sum() == 112 and (mug[:, 3] == 0.005).sum() == 16
    for rows in (W.sphere16(), W.l_composite256(), mug):
        assert np.allclose(rows[:, :3].mean(axis=0), 0.0, atol=1e-15)


@pytest.mark.parametrize("name, n, frames, fingers, pads, substeps, iters, spheres", [
    ("tracking_box27", 16, 150, 4, 8, 2, {20}, [27]),
    ("tracking_cyl64", 1024, 300, 4, 8, 2, {20}, [64]),
    ("uneven_mixed", 8192, 60, 5, 16, 2, {10, 20, 40}, [16, 27, 64, 256]),
    ("adjoint_mixed", 1024, 30, 4, 8, 2, {20}, [27, 64]),
    ("sweep_mug128", 1024, 60, 5, 16, 4, {40}, [128]),
])
def test_workload_sizes(name, n, frames, fingers, pads, substeps, iters, spheres):
    wl = W.make_workload(name)
    sc = wl.scene
    assert wl.n_envs == n and wl.frames == frames
    assert sc.n_fingers == fingers and sc.n_links == 1 + 4 * fingers and sc.n_pads == pads
    assert [len(s) for s in sc.shapes] == spheres
    assert wl.sim.substeps == substeps and set(int(i) for i in wl.iters) == iters
    assert math.isclose(wl.sim.frame_dt, 1 / 30) and wl.sim.gravity == (0.0, 0.0, -9.81)
    assert np.allclose(sc.palm_half, [0.04, 0.04, 0.01])
    assert sc.link_len == 0.03 and sc.link_rad == 0.008
    assert wl.q_traj.shape == (frames + 1, 4 * fingers) and wl.q_traj.dtype == np.float32
    assert wl.shape_id.shape == (n,) and wl.iters.shape == (n,)
    assert set(int(s) for s in wl.shape_id) == set(range(len(spheres)))
    # every finger roots on the palm top, outside the object's horizontal extent
    assert np.allclose(sc.finger_root[:, 2], 0.01)
    half = max(W.horizontal_halfwidth(s) for s in sc.shapes)
    assert np.all(np.hypot(sc.finger_root[:, 0], sc.finger_root[:, 1]) > half + sc.link_rad)
    # pads on existing links, axial intervals inside [0, 1]
    assert np.all((sc.pad_link >= 0) & (sc.pad_link < sc.n_links))
    assert np.all((0 <= sc.pad_s0) & (sc.pad_s0 < sc.pad_s1) & (sc.pad_s1 <= 1))
    # the estimate rests on the palm top, the truth is off it by one pose draw
    assert wl.nominal_pose[2] > 0.01 and np.isclose(np.linalg.norm(wl.nominal_pose[4:]), 1.0)
    assert not np.allclose(wl.gt_pose, wl.nominal_pose)
    assert np.isclose(np.linalg.norm(wl.gt_pose[4:]), 1.0, atol=1e-6)


def test_uneven_batch_mixes_shapes_and_iterations_evenly():
    wl = W.make_workload("uneven_mixed")
    for v in range(4):
        assert abs((wl.shape_id == v).mean() - 0.25) < 0.03
    for it in (10, 20, 40):
        assert abs((wl.iters == it).mean() - 1 / 3) < 0.03


def test_pad_layouts():
    link, s0, s1 = W.pads_fingertips(4)
    assert list(link) == [4, 3, 8, 7, 12, 11, 16, 15]   # distal then middle link of each finger
    assert np.all(s0 == 0) and np.all(s1 == 1)
    link, s0, s1 = W.pads_sixteen(5)
    assert len(link) == 16 and link[-1] == 0             # the palm pad last
    assert list(link[:10:2]) == [4, 8, 12, 16, 20] and list(s1[:10]) == [0.5, 1.0] * 5


def test_joint_trajectory_is_an_opening_and_closing_grasp():
    F, frames, dt = 5, 900, 1 / 30
    q = W.joint_trajectory(F, frames, dt, seed=7).astype(np.float64)
    flex = np.delete(q, np.arange(0, 4 * F, 4), axis=1)
    abd = q[:, 0::4]
    assert np.allclose(flex[0], 0.0)                     # the hand starts open
    assert flex.min() >= -1e-7 and flex.max() <= 0.8 + 1e-6
    # over 30 s every flexion closes to its amplitude A in [0.3, 0.8] and reopens
    assert np.all(flex.max(axis=0) >= 0.3 * 0.99) and np.all(flex.min(axis=0) <= 1e-3)
    assert np.abs(abd).max() <= 0.25 * 0.8 + 1e-6
    # frequencies within [0.5, 1.5] Hz: the flexion returns to ~0 at least
    # once per 2 s and at most every 0.66 s
    zeros = [np.sum((c[1:-1] < c[:-2]) & (c[1:-1] <= c[2:])) for c in flex.T]
    assert min(zeros) >= int(30 * 0.5) - 1 and max(zeros) <= int(30 * 1.5) + 1


def test_ground_truth_parameters_in_the_prior_ranges():
    for seed in range(20):
        m, mu = W.theta_draw(seed, (0.05, 0.3), (0.3, 1.2))
        assert 0.05 <= m <= 0.3 and 0.3 <= mu <= 1.2
    init = W.InitSampling()
    assert init.sigma_p == 0.005 and math.isclose(init.sigma_r, math.radians(5.0))
    assert init.m_range == (0.05, 0.3) and init.mu_range == (0.3, 1.2)


def test_generation_is_deterministic_in_the_seed():
    a = W.make_workload("uneven_mixed", n_envs=512, frames=20)
    b = W.make_workload("uneven_mixed", n_envs=512, frames=20)
    c = W.make_workload("uneven_mixed", n_envs=512, frames=20, seed=1)
    assert np.array_equal(a.q_traj, b.q_traj) and np.array_equal(a.shape_id, b.shape_id)
    assert np.array_equal(a.iters, b.iters) and np.array_equal(a.gt_pose, b.gt_pose)
    assert a.theta_gt == b.theta_gt
    assert not np.array_equal(a.q_traj, c.q_traj) and not np.array_equal(a.shape_id, c.shape_id)
