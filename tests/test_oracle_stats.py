"""Pins of the oracle's random streams, initial sampling, cost and optimizer.

Philox4x32-10 is checked against its published known-answer vectors; the
normal and uniform streams against their distributions; the so(3) maps against
scipy's rotation library; the cost against hand-computed values; the
optimizer's ranking, weighted statistics and Cholesky factor against numpy and
its resampling against the defining property of systematic resampling.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2002_12160_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        np.testing.assert_array_equal(O.philox(v[0:4], v[4:6]), np.array(v[6:10], np.uint32))


def test_normal_stream_distribution():
    z = np.concatenate([O.normals(7, 1, 3, e, 8) for e in range(20000)])
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # distinct counters give distinct draws
    assert not np.array_equal(O.normals(7, 1, 3, 0, 8), O.normals(7, 1, 4, 0, 8))
    assert not np.array_equal(O.normals(7, 1, 3, 0, 8), O.normals(8, 1, 3, 0, 8))


def test_uniform_stream_distribution():
    u = np.concatenate([O.uniforms(11, 2, k, 0, 0) for k in range(20000)])
    assert u.min() > 0 and u.max() < 1
    assert stats.kstest(u, "uniform").pvalue > 1e-4


@pytest.mark.parametrize("seed", range(6))
def test_so3_exp_log_against_scipy(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=3)
    w *= rng.uniform(0.0, 3.0) / np.linalg.norm(w)
    q = O.quat_exp(w)
    ref = Rotation.from_rotvec(w).as_quat(scalar_first=True)
    if np.dot(q, ref) < 0:
        ref = -ref
    np.testing.assert_allclose(q, ref, atol=1e-15)
    np.testing.assert_allclose(O.quat_log(q), w, atol=1e-12)
    np.testing.assert_allclose(O.quat_log(-q), w, atol=1e-12)


def test_initial_sampling_distribution():
    n = 20000
    init = W.InitSampling()
    nominal = np.array([0.01, -0.02, 0.035, *Rotation.from_rotvec([0.1, 0.2, -0.3]).as_quat(scalar_first=True)])
    pose, theta = O.sample_initial(n, nominal, init, seed=5)
    dx = pose[:, :3] - nominal[:3]
    np.testing.assert_allclose(dx.mean(0), 0, atol=4 * init.sigma_p / math.sqrt(n))
    np.testing.assert_allclose(np.cov(dx.T), init.sigma_p ** 2 * np.eye(3), atol=4 * init.sigma_p ** 2 * math.sqrt(2 / n))
    r0 = Rotation.from_quat(nominal[3:], scalar_first=True)
    rel = (Rotation.from_quat(pose[:, 3:], scalar_first=True) * r0.inv()).as_rotvec()
    np.testing.assert_allclose(rel.mean(0), 0, atol=4 * init.sigma_r / math.sqrt(n))
    np.testing.assert_allclose(np.cov(rel.T), init.sigma_r ** 2 * np.eye(3), atol=4 * init.sigma_r ** 2 * math.sqrt(2 / n))
    assert theta[:, 0].min() >= init.m_range[0] and theta[:, 0].max() <= init.m_range[1]
    assert stats.kstest((theta[:, 1] - init.mu_range[0]) / (init.mu_range[1] - init.mu_range[0]), "uniform").pvalue > 1e-4


def test_cost_hand_computed():
    sim = W.SimConfig(tau=0.02, w_force=1.0, w_contact=1.0)
    forces = np.array([[[1.0, 0, 0], [0, 0, 0]],      # env 0
                       [[0, 0, 0], [0, 0.5, 0]],       # env 1 = the observation
                       [[0, 0, 0.01], [0, 0.5, 0]]])   # env 2: below threshold on pad 0
    obs = np.array([[0, 0, 0], [0, 0.5, 0]])
    c_sum = np.zeros(3)
    i, c_mean, c = O.cost(sim, forces, obs, np.zeros(3, np.int32), c_sum, 1)
    # env 0: |(1,0,0)|^2 + |(0,-0.5,0)|^2 = 1.25, plus two contact-state mismatches
    np.testing.assert_allclose(c, [1.25 + 2.0, 0.0, 1e-4], rtol=1e-15)
    assert i == 1
    # second frame: the running mean uses the window length
    i, c_mean, _ = O.cost(sim, forces, obs, np.zeros(3, np.int32), c_sum, 2)
    np.testing.assert_allclose(c_mean, [3.25, 0.0, 1e-4], rtol=1e-15)


def test_argmin_ties_nan_and_diverged():
    sim = W.SimConfig()
    forces = np.zeros((5, 1, 3))
    forces[0, 0, 0] = 0.5
    obs = np.zeros((1, 3))
    status = np.array([0, 1, 0, 0, 0], np.int32)       # env 1 diverged
    c_sum = np.array([0.0, -10.0, np.nan, 0.0, 0.0])   # env 2 NaN, envs 3 and 4 tie
    i, c_mean, _ = O.cost(sim, forces, obs, status, c_sum, 1)
    assert math.isinf(c_mean[1])
    assert i == 3


def _opt_state(n, seed):
    rng = np.random.default_rng(seed)
    pose = np.zeros((n, 7))
    pose[:, :3] = rng.normal(size=(n, 3)) * 0.01
    pose[:, 3:] = Rotation.from_rotvec(rng.normal(size=(n, 3)) * 0.2).as_quat(scalar_first=True)
    vel = rng.normal(size=(n, 6))
    theta = np.column_stack([rng.uniform(0.05, 0.3, n), rng.uniform(0.3, 1.2, n)])
    C = rng.exponential(size=n)
    return O.State(pose, vel, theta), C


def test_optimizer_elites_weights_and_statistics():
    n = 200
    st, C = _opt_state(n, 1)
    C[17] = C[3]            # a tie: index order decides
    C[50] = np.nan          # NaN ranks last
    before = O.State(st.pose, st.vel, st.theta)
    opt = W.OptConfig()
    istar, parent, s = O.optimizer(opt, st, C, seed=9, update_index=4)
    k = max(1, int(math.floor(opt.elite_frac * n)))
    key = np.where(np.isnan(C), np.inf, C)
    order = np.lexsort((np.arange(n), key))
    elites = np.sort(order[:k])
    assert s["k"] == k and istar == order[0] == s["istar"]
    # elites unchanged and their own parents
    np.testing.assert_array_equal(parent[elites], elites)
    np.testing.assert_array_equal(st.pose[elites], before.pose[elites])
    np.testing.assert_array_equal(st.theta[elites], before.theta[elites])
    # weights exp(-(C - Cmin)/s), s = population std of the elite costs
    ce = key[elites]
    sd = ce.std()
    assert abs(s["sd"] - sd) < 1e-15
    w = np.exp(-(ce - ce.min()) / sd)
    w /= w.sum()
    r_ref = Rotation.from_quat(before.pose[istar, 3:], scalar_first=True)
    rot = (Rotation.from_quat(before.pose[elites, 3:], scalar_first=True) * r_ref.inv()).as_rotvec()
    z = np.column_stack([before.pose[elites, :3], rot, before.theta[elites]])
    np.testing.assert_allclose(s["mean"], np.average(z, axis=0, weights=w), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(s["cov"], np.cov(z.T, aweights=w, bias=True), rtol=1e-10, atol=1e-16)
    A = s["cov"] + np.diag(np.array(opt.floor_std) ** 2)
    np.testing.assert_allclose(s["L"], np.linalg.cholesky(A), rtol=1e-12, atol=1e-16)
    # systematic resampling: elite j has floor(M w_j) or ceil(M w_j) children
    M = n - k
    non = np.setdiff1d(np.arange(n), elites)
    counts = np.array([(parent[non] == e).sum() for e in elites])
    assert counts.sum() == M
    assert np.all(counts >= np.floor(M * w) - 1e-9) and np.all(counts <= np.ceil(M * w) + 1e-9)
    # non-elites copy the parent's velocity and stay inside the clamps
    np.testing.assert_array_equal(st.vel[non], before.vel[parent[non]])
    assert st.theta[:, 0].min() >= opt.m_range[0] and st.theta[:, 1].max() <= opt.mu_range[1]


def test_optimizer_perturbation_has_the_floor_covariance():
    """With one elite (all mass on it), every child is parent + L eps, L L^T = Sigma_floor."""
    n = 20001
    st, C = _opt_state(n, 2)
    C[:] = 5.0
    C[123] = 0.0
    opt = W.OptConfig(elite_frac=0.5 / n)   # k = 1
    parent_pose = st.pose[123].copy()
    parent_theta = st.theta[123].copy()
    istar, parent, s = O.optimizer(opt, st, C, seed=3, update_index=1)
    assert istar == 123 and s["k"] == 1 and np.all(parent == 123)
    non = np.arange(n) != 123
    dx = st.pose[non, :3] - parent_pose[:3]
    rot = (Rotation.from_quat(st.pose[non, 3:], scalar_first=True)
           * Rotation.from_quat(parent_pose[3:], scalar_first=True).inv()).as_rotvec()
    dth = st.theta[non] - parent_theta
    d = np.column_stack([dx, rot, dth])
    sig = np.array(opt.floor_std)
    m = d.shape[0]
    np.testing.assert_allclose(d.mean(0) / sig, 0, atol=4 / math.sqrt(m))
    np.testing.assert_allclose(d.std(0) / sig, 1, atol=4 * math.sqrt(0.5 / m))
    np.testing.assert_allclose(np.corrcoef(d.T) - np.eye(8), 0, atol=4 / math.sqrt(m))


def test_optimizer_equal_costs_give_uniform_weights():
    n = 100
    st, C = _opt_state(n, 4)
    C[:] = 2.5
    before = st.pose.copy()
    istar, parent, s = O.optimizer(W.OptConfig(), st, C, seed=1, update_index=0)
    elites = np.arange(10)                    # ties -> lowest indices
    assert istar == 0
    np.testing.assert_allclose(s["mean"][:3], before[elites, :3].mean(0), rtol=1e-12)
    counts = np.array([(parent[10:] == e).sum() for e in elites])
    np.testing.assert_array_equal(counts, np.full(10, 9))


def test_cholesky_against_numpy():
    rng = np.random.default_rng(0)
    B = rng.normal(size=(8, 8))
    A = B @ B.T + 0.1 * np.eye(8)
    rc, L = O.cholesky8(A)
    assert rc == 0
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-14, atol=1e-14)
    rc, _ = O.cholesky8(-A)
    assert rc == -1
