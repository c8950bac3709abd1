"""Pins of the oracle's WRS and REPS updates (Sec. III-D, Eqs. of WRS and REPS).

- REPS temperature: eta* minimises the dual g(eta) (scipy's bounded scalar
  minimiser on log eta), and at the minimum the PMF's divergence from the
  uniform PMF over the finite-cost simulations equals epsilon (the KL bound is
  active: g'(eta*) = eps - KL).
- degenerate cases: equal costs -> uniform (eta* = +inf); eps >= log(K/n_min)
  -> all mass on the minima (eta* = 0); diverged simulations excluded.
- WRS: the PMF is the softmax of -lambda (C - C_min); each environment's
  parent is the inverse CDF (index order) of its stream-3 uniform.
- draws with replacement: parent counts over many environments follow the
  PMF (chi-square); REPS with eta* equals WRS with lambda = 1/eta*.
- exploration: per-coordinate standard deviations of the perturbations
  (pose or velocity mode); the pose is untouched in velocity mode.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2002_12160_gb300 import workloads as W

scipy_opt = pytest.importorskip("scipy.optimize")
scipy_stats = pytest.importorskip("scipy.stats")


def _state(n, rng):
    pose = np.zeros((n, 7))
    pose[:, :3] = rng.normal(0, 0.01, (n, 3))
    q = rng.normal(size=(n, 4))
    pose[:, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
    vel = rng.normal(0, 0.05, (n, 6))
    theta = np.stack([rng.uniform(0.05, 0.3, n), rng.uniform(0.3, 1.2, n)], 1)
    return O.State(pose, vel, theta)


def _opt(**kw):
    return dataclasses.replace(W.OptConfig(), **kw)


@pytest.mark.parametrize("eps", [0.05, 0.5, 1.0, 3.0])
def test_reps_eta_minimises_the_dual_and_meets_the_kl_bound(eps):
    rng = np.random.default_rng(7)
    C = rng.uniform(0.1, 5.0, 300)
    C[[3, 40]] = np.inf   # diverged simulations take no part
    fin = C[np.isfinite(C)]
    K, cmin = len(fin), fin.min()
    eta, iters = O.reps_eta(C, eps)
    assert 0 < eta < np.inf and iters < 40

    def g(t):
        e = np.exp(t)
        return e * eps + e * np.log(np.mean(np.exp((cmin - fin) / e)))

    r = scipy_opt.minimize_scalar(g, bounds=(np.log(eta) - 5, np.log(eta) + 5), method="bounded",
                                  options={"xatol": 1e-11})
    assert abs(np.exp(r.x) / eta - 1) < 1e-6
    P = np.exp((cmin - fin) / eta)
    P /= P.sum()
    assert abs(np.sum(P * np.log(P * K)) - eps) < 1e-10


def test_reps_degenerate_cases():
    eta, _ = O.reps_eta(np.full(10, 2.5), 0.5)
    assert eta == np.inf                                   # equal costs: uniform
    C = np.array([1.0, 1.0, 2.0, 3.0, np.nan, np.inf])
    eta, _ = O.reps_eta(C, np.log(4 / 2) + 1e-9)           # eps >= log(K / n_min), K = 4, n_min = 2
    assert eta == 0.0
    st = _state(6, np.random.default_rng(1))
    _, parent, stats = O.softmax_update(_opt(kind="reps", reps_epsilon=2.0), st, C, 11, 3)
    assert set(parent) <= {0, 1} and stats["n_finite"] == 4
    st = _state(5, np.random.default_rng(2))
    _, parent, stats = O.softmax_update(_opt(kind="wrs"), st, np.full(5, np.inf), 11, 3)
    assert stats["wsum"] == 5.0                            # nothing finite: uniform over all


def test_wrs_pmf_and_inverse_cdf_draws():
    rng = np.random.default_rng(3)
    n, lam, seed, upd = 2000, 0.7, 99, 5
    C = rng.uniform(0.0, 6.0, n)
    C[[10, 11]] = np.nan
    st = _state(n, rng)
    p_before = st.pose.copy()
    istar, parent, stats = O.softmax_update(_opt(kind="wrs", wrs_lambda=lam), st, C, seed, upd)
    fin = np.isfinite(C)
    w = np.where(fin, np.exp(-lam * (np.where(fin, C, 0) - C[fin].min())), 0.0)
    cum = np.cumsum(w)
    assert abs(stats["wsum"] / cum[-1] - 1) < 1e-13
    u = np.array([O.uniforms(seed, 3, upd, i, 0)[0] for i in range(n)])
    expect = np.searchsorted(cum, u * cum[-1], side="right")
    assert np.array_equal(parent, expect)
    assert not np.any(np.isin(parent, [10, 11]))
    assert istar == int(np.nanargmin(C))
    # each environment starts from its parent's pose before exploring
    d = np.linalg.norm(st.pose[:, :3] - p_before[parent, :3], axis=1)
    assert d.max() < 10 * 0.001 * np.sqrt(3)


def test_draws_follow_the_pmf_and_reps_is_wrs_at_its_temperature():
    rng = np.random.default_rng(4)
    n = 20000
    levels = np.array([0.0, 0.3, 0.7, 1.5, 3.0])
    C = levels[rng.integers(0, 5, n)]
    st = _state(n, rng)
    _, parent, stats = O.softmax_update(_opt(kind="reps", reps_epsilon=0.4), st, C, 5, 1)
    eta = stats["eta"]
    w = np.exp((C.min() - C) / eta)
    P = w / w.sum()
    groups = [C == v for v in levels]
    obs = np.array([np.sum(g[parent]) for g in groups])
    exp_ = np.array([n * P[g].sum() for g in groups])
    chi2 = np.sum((obs - exp_) ** 2 / exp_)
    assert scipy_stats.chi2.sf(chi2, len(levels) - 1) > 1e-3
    st2 = _state(n, np.random.default_rng(4))
    _, parent2, _ = O.softmax_update(_opt(kind="wrs", wrs_lambda=1.0 / eta), st2, C, 5, 1)
    assert np.mean(parent2 == parent) > 0.999


@pytest.mark.parametrize("mode", ["pose", "velocity"])
def test_exploration_standard_deviations(mode):
    n = 20000
    rng = np.random.default_rng(5)
    st = _state(n, rng)
    st.pose[:] = st.pose[0]
    st.vel[:] = st.vel[0]
    st.theta[:] = [0.2, 0.8]
    p0, v0 = st.pose[0].copy(), st.vel[0].copy()
    opt = _opt(kind="wrs", explore=mode, sigma_pose=(0.001, 0.002, 0.003, 0.01, 0.02, 0.03),
               sigma_vel=(0.01, 0.02, 0.03, 0.1, 0.2, 0.3), sigma_theta=(0.004, 0.03))
    O.softmax_update(opt, st, np.zeros(n), 8, 2)   # equal costs: uniform parents, all identical
    tol = 4 / np.sqrt(2 * n)                       # 4 sigma of a sample standard deviation
    np.testing.assert_allclose(st.theta.std(0), opt.sigma_theta, rtol=tol)
    if mode == "pose":
        np.testing.assert_allclose((st.pose[:, :3] - p0[:3]).std(0), opt.sigma_pose[:3], rtol=tol)
        rot = np.array([O.quat_log(_qmul(q, _qconj(p0[3:]))) for q in st.pose[:2000, 3:]])
        np.testing.assert_allclose(rot.std(0), opt.sigma_pose[3:], rtol=4 / np.sqrt(2 * 2000))
        assert np.allclose(st.vel, v0)
    else:
        assert np.array_equal(st.pose, np.broadcast_to(p0, st.pose.shape))
        np.testing.assert_allclose((st.vel - v0).std(0), opt.sigma_vel, rtol=tol)


def _qmul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])


def _qconj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])
