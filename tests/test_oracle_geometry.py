"""Pins of the oracle's kinematics, narrowphase, inertia and ADD.

The narrowphase is checked against brute force: the distance from a sphere
centre to a capsule axis or to a box surface, found by dense sampling of that
segment or surface. The finger kinematics is checked against planar
trigonometry of an upright finger curling toward the palm centre. ADD is
checked against its closed forms for a translation and for a rotation about
an axis through the centroid.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2002_12160_gb300 import workloads as W

SIM = W.SimConfig()


def _hand_scene(n_fingers=4):
    wl = W.make_workload("tracking_box27", n_envs=1, frames=2)
    return wl.scene


def test_fk_rest_pose_is_upright_fingers():
    sc = _hand_scene()
    osc = O.OracleScene(sc)
    lp = O.fk(osc, np.zeros(sc.n_joints))
    np.testing.assert_array_equal(lp[0], [0, 0, 0, 1, 0, 0, 0])
    for f in range(sc.n_fingers):
        root = sc.finger_root[f, :3]
        for j in range(4):
            p = lp[1 + 4 * f + j]
            np.testing.assert_allclose(p[:3], root + [0, 0, j * sc.link_len], atol=1e-15)
            # link +x points up
            ax = Rotation.from_quat(p[3:], scalar_first=True).apply([1, 0, 0])
            np.testing.assert_allclose(ax, [0, 0, 1], atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_fk_matches_planar_curl(seed):
    """Link j starts at root + L sum_{i<j} (cos(phi_i) z - sin(phi_i) r), phi_i the
    cumulative flexion, r the radial direction of the finger's bending plane."""
    sc = _hand_scene()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(seed)
    q = rng.uniform(-1.0, 1.0, sc.n_joints)
    lp = O.fk(osc, q)
    L = sc.link_len
    for f in range(sc.n_fingers):
        root = sc.finger_root[f, :3]
        yaw = sc.finger_root[f, 3] + q[4 * f]
        r = np.array([math.cos(yaw), math.sin(yaw), 0.0])
        z = np.array([0.0, 0.0, 1.0])
        phi = [0.0, q[4 * f + 1], q[4 * f + 1] + q[4 * f + 2], q[4 * f + 1] + q[4 * f + 2] + q[4 * f + 3]]
        p = root.copy()
        for j in range(4):
            got = lp[1 + 4 * f + j]
            np.testing.assert_allclose(got[:3], p, atol=1e-14)
            d = math.cos(phi[j]) * z - math.sin(phi[j]) * r
            ax = Rotation.from_quat(got[3:], scalar_first=True).apply([1, 0, 0])
            np.testing.assert_allclose(ax, d, atol=1e-14)
            p = p + L * d


def _segment_distance_sampled(c, a, b, n=200001):
    t = np.linspace(0, 1, n)
    pts = a[None] + t[:, None] * (b - a)[None]
    dd = np.linalg.norm(pts - c[None], axis=1)
    k = np.argmin(dd)
    return dd[k], t[k], pts[k]


@pytest.mark.parametrize("seed", range(8))
def test_sphere_capsule_against_sampled_segment(seed):
    sc = _hand_scene()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(100 + seed)
    q = rng.uniform(-0.8, 0.8, sc.n_joints)
    lp = O.fk(osc, q)
    link = 1 + int(rng.integers(0, 4 * sc.n_fingers))
    pl = lp[link]
    R = Rotation.from_quat(pl[3:], scalar_first=True)
    a = pl[:3]
    b = a + R.apply([sc.link_len, 0, 0])
    # an object made of one sphere placed near the link
    rs = 0.006
    c = a + rng.uniform(-0.3, 1.3) * (b - a) + rng.normal(size=3) * 0.007
    shape = np.array([[0.0, 0.0, 0.0, rs]])
    one = W.Scene(shapes=[shape], palm_half=sc.palm_half, finger_root=sc.finger_root,
                  link_len=sc.link_len, link_rad=sc.link_rad, pad_link=sc.pad_link,
                  pad_s0=sc.pad_s0, pad_s1=sc.pad_s1)
    osc1 = O.OracleScene(one)
    big = W.SimConfig(margin=1.0)   # report every pair
    rows = O.contacts(osc1, big, 0, [*c, 1, 0, 0, 0], lp)
    row = rows[rows[:, 1] == link][0]
    dist, t, closest = _segment_distance_sampled(c, a, b)
    assert abs(row[3] - (dist - rs - sc.link_rad)) < 2e-7
    assert abs(row[10] - t) < 2e-5
    n = (c - closest) / np.linalg.norm(c - closest)
    np.testing.assert_allclose(row[4:7], n, atol=1e-4)
    np.testing.assert_allclose(row[7:10], c - rs * row[4:7], atol=1e-15)


def _box_surface_distance_sampled(cl, half, n=401):
    """Distance from a point to the box surface by sampling its six faces."""
    best = np.inf
    best_pt = None
    g = [np.linspace(-h, h, n) for h in half]
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        U, V = np.meshgrid(g[o1], g[o2], indexing="ij")
        for s in (1, -1):
            pts = np.zeros((U.size, 3))
            pts[:, ax] = s * half[ax]
            pts[:, o1] = U.ravel()
            pts[:, o2] = V.ravel()
            d = np.linalg.norm(pts - cl[None], axis=1)
            k = np.argmin(d)
            if d[k] < best:
                best, best_pt = d[k], pts[k]
    return best, best_pt


@pytest.mark.parametrize("seed", range(8))
def test_sphere_box_against_sampled_surface(seed):
    rng = np.random.default_rng(200 + seed)
    half = np.array([0.04, 0.03, 0.01])
    rs = 0.005
    inside = seed % 2 == 1
    if inside:
        cl = rng.uniform(-0.8, 0.8, 3) * half
    else:
        cl = rng.uniform(-1.6, 1.6, 3) * half
        while np.all(np.abs(cl) <= half):
            cl = rng.uniform(-1.6, 1.6, 3) * half
    sc = W.Scene(shapes=[np.array([[0.0, 0.0, 0.0, rs]])], palm_half=half,
                 finger_root=np.zeros((0, 4)), link_len=0.03, link_rad=0.008,
                 pad_link=np.array([0], np.int32), pad_s0=np.array([0.0]), pad_s1=np.array([1.0]))
    osc = O.OracleScene(sc)
    rows = O.contacts(osc, W.SimConfig(margin=1.0), 0, [*cl, 1, 0, 0, 0], O.fk(osc, np.zeros(0)))
    assert len(rows) == 1
    dist, pt = _box_surface_distance_sampled(cl, half)
    h = 2 * max(half) / 400
    if inside:
        assert abs(rows[0, 3] - (-dist - rs)) < 1e-12 + h
        # normal: outward normal of the face that holds the nearest sampled point
        on_face = np.isclose(np.abs(pt), half, rtol=0, atol=1e-15)
        if on_face.sum() == 1:
            ax = int(np.argmax(on_face))
            n = np.zeros(3)
            n[ax] = np.sign(pt[ax])
            np.testing.assert_allclose(rows[0, 4:7], n, atol=0)
    else:
        assert abs(rows[0, 3] - (dist - rs)) < h
        if dist > 20 * h:   # the sampled direction is meaningful only well off the grid
            n = (cl - pt) / np.linalg.norm(cl - pt)
            np.testing.assert_allclose(rows[0, 4:7], n, atol=5e-2)


def test_contact_list_is_every_pair_under_the_margin():
    """The brute-force list equals an independent scan of pair distances."""
    wl = W.make_workload("tracking_cyl64", n_envs=1, frames=30)
    osc = O.OracleScene(wl.scene)
    lp = O.fk(osc, wl.q_traj[25])
    pose = O.pose8_to7(wl.nominal_pose)
    rows = O.contacts(osc, wl.sim, 0, pose, lp)
    assert len(rows) > 5
    shp = wl.scene.shapes[0]
    found = set((int(r[0]), int(r[1])) for r in rows)
    for j, s in enumerate(shp):
        c = pose[:3] + s[:3]   # identity rotation, centred cluster
        for l in range(1, wl.scene.n_links):
            pl = lp[l]
            a = pl[:3]
            b = a + Rotation.from_quat(pl[3:], scalar_first=True).apply([wl.scene.link_len, 0, 0])
            t = np.clip(np.dot(c - a, b - a) / np.dot(b - a, b - a), 0, 1)
            d = np.linalg.norm(c - (a + t * (b - a))) - s[3] - wl.scene.link_rad
            assert ((j, l) in found) == (d < wl.sim.margin)
        dpalm = c[2] - wl.scene.palm_half[2] - s[3]   # above the palm top, within its footprint
        if abs(c[0]) < wl.scene.palm_half[0] and abs(c[1]) < wl.scene.palm_half[1] and c[2] > wl.scene.palm_half[2]:
            assert ((j, 0) in found) == (dpalm < wl.sim.margin)


def test_pad_assignment_by_axial_interval():
    wl = W.make_workload("uneven_mixed", n_envs=1, frames=2)
    sc = wl.scene
    osc = O.OracleScene(sc)
    lp = O.fk(osc, np.zeros(sc.n_joints))
    one = W.Scene(shapes=[np.array([[0.0, 0.0, 0.0, 0.004]])], palm_half=sc.palm_half,
                  finger_root=sc.finger_root, link_len=sc.link_len, link_rad=sc.link_rad,
                  pad_link=sc.pad_link, pad_s0=sc.pad_s0, pad_s1=sc.pad_s1)
    osc1 = O.OracleScene(one)
    f = 2
    distal = 1 + 4 * f + 3
    middle = 1 + 4 * f + 2
    a = lp[distal, :3]
    inward = -np.array([math.cos(sc.finger_root[f, 3]), math.sin(sc.finger_root[f, 3]), 0])
    for t, want in [(0.2, 2 * f), (0.8, 2 * f + 1)]:
        c = a + [0, 0, t * sc.link_len] + inward * (sc.link_rad + 0.004 + 0.001)
        rows = O.contacts(osc1, SIM, 0, [*c, 1, 0, 0, 0], lp)
        r = rows[rows[:, 1] == distal][0]
        assert int(r[2]) == want
    c = lp[middle, :3] + [0, 0, 0.5 * sc.link_len] + inward * (sc.link_rad + 0.005)
    rows = O.contacts(osc1, SIM, 0, [*c, 1, 0, 0, 0], lp)
    assert int(rows[rows[:, 1] == middle][0][2]) == 2 * sc.n_fingers + f


def test_unit_inertia_of_sphere_grid():
    """3x3x3 grid, spacing s, radius r: J_xx = (2/5) r^2 + (2/3) 2 s^2 / 3 * 3 = 0.4 r^2 + 4 s^2 / 3."""
    side, r = 0.05, 0.0083
    s = side / 2 - r
    osc = O.OracleScene(W.ground_scene(W.box27(side, r)))
    J = O.unit_inertia(osc, 0)
    # mean of y^2 + z^2 over the grid: each coordinate is -s, 0, s with mean square 2 s^2 / 3
    np.testing.assert_allclose(J, np.eye(3) * (0.4 * r * r + 2 * (2 * s * s / 3)), rtol=1e-12, atol=1e-18)


def test_unit_inertia_of_single_ball():
    osc = O.OracleScene(W.ground_scene(np.array([[0.3, -0.1, 0.2, 0.01]])))
    np.testing.assert_allclose(O.unit_inertia(osc, 0), 0.4 * 1e-4 * np.eye(3), rtol=1e-12)


def test_add_translation_and_rotation_closed_forms():
    rows = W.cylinder64()
    osc = O.OracleScene(W.ground_scene(rows))
    a = np.array([0.01, 0.02, 0.05, 1, 0, 0, 0])
    t = np.array([0.003, -0.004, 0.012])
    b = a.copy()
    b[:3] += t
    assert abs(O.add(osc, 0, a, b) - np.linalg.norm(t)) < 1e-15
    th = 0.3
    c = a.copy()
    c[3:] = Rotation.from_rotvec([0, 0, th]).as_quat(scalar_first=True)
    rho = np.hypot(rows[:, 0], rows[:, 1])
    assert abs(O.add(osc, 0, a, c) - np.mean(2 * math.sin(th / 2) * rho)) < 1e-15


@pytest.mark.parametrize("joint", [0, 1, 2, 3])
def test_link_point_velocity_is_the_rigid_rotation_of_the_joint(joint):
    """A contact's link velocity (the kinematic hand) is the displacement over
    the substep of the link point carried rigidly from the link's start pose to
    its end pose. When only joint `joint` of finger 1 turns, by d = w h, every
    link at or after it turns rigidly by d about that joint's axis: the vertical
    axis through the finger root for the abduction joint 0, the link frame's y
    axis through the link origin (turning by -d) for a flexion joint. So
      v = (Rot(a, +-d) (p - o) + o - p) / h   exactly,
    which tends to w (a x (p - o)) with an error of (h/2) w^2 |a x (a x r)| +
    O(h^2): halving h halves it."""
    sc = _hand_scene()
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(11 + joint)
    f = 1
    q = rng.uniform(-0.3, 0.8, sc.n_joints)
    w = 2.7   # rad/s
    k = 4 * f + joint
    lp_a = O.fk(osc, q)
    if joint == 0:
        a, o, sgn = np.array([0.0, 0.0, 1.0]), sc.finger_root[f, :3], 1.0
    else:
        la = lp_a[1 + k]
        a = Rotation.from_quat(la[3:], scalar_first=True).apply([0, 1, 0])
        o, sgn = la[:3], -1.0
    errs = []
    for h in (1e-2, 5e-3, 2.5e-3):
        dq = np.zeros(sc.n_joints)
        dq[k] = w * h
        lp_b = O.fk(osc, q + dq)
        for j in range(joint, 4):
            l = 1 + 4 * f + j
            p = lp_a[l, :3] + rng.normal(scale=0.01, size=3)
            v = O.link_point_velocity(lp_a[l], lp_b[l], p, h)
            rot = Rotation.from_rotvec(sgn * w * h * a)
            v_ref = (rot.apply(p - o) + o - p) / h
            np.testing.assert_allclose(v, v_ref, rtol=0, atol=1e-12)
            if j == 3:
                r = p - o
                lim = sgn * w * np.cross(a, r)
                errs.append((np.linalg.norm(v - lim), 0.5 * h * w * w * np.linalg.norm(np.cross(a, np.cross(a, r)))))
        # links before the joint do not move
        for j in range(joint):
            l = 1 + 4 * f + j
            p = lp_a[l, :3]
            np.testing.assert_allclose(O.link_point_velocity(lp_a[l], lp_b[l], p, h), 0.0, atol=1e-12)
    for e, e_pred in errs:
        assert abs(e - e_pred) <= 0.05 * e_pred, (e, e_pred)
