"""Pins of the FP64 adjoint oracle (oracle/adjoint.py).

1. Its forward is the C oracle's: the same frames from the same state give
   the same states and pad forces to rounding.
2. With the smoothing applied in the forward as well, the function is smooth
   along branch-stable paths, so its autograd gradient must equal central
   finite differences (FP64; steps 1e-6 and 5e-7 combined by Richardson
   extrapolation, which removes the h^2 error term) to 1e-6 relative.
   The check uses a friction-disk smoothing width of 0.2 (relative to the
   disk radius): with the default 1e-3 the smoothed clamp bends over an
   impulse change of about 1e-6 N s, the size a 1e-6 m step causes, so the
   difference quotient cannot resolve it (its higher derivatives scale as
   width^-3) although the adjoint is exact there too.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2002_12160_gb300 import workloads as W

pytest.importorskip("torch")

WIDTH = 0.2


def _case(n=4, frames=8, warm=3, name="tracking_box27"):
    wl = W.make_workload(name, n_envs=n, frames=frames)
    osc = O.OracleScene(wl.scene)
    pose, theta = O.sample_initial(n, O.pose8_to7(wl.nominal_pose), wl.init, wl.seed)
    st = O.State(pose, np.zeros((n, 6)), theta)
    O.step(osc, wl.sim, st, wl.q_traj, 0, warm)    # contacts established
    return wl, osc, st


def test_forward_equals_c_oracle():
    wl, osc, st = _case()
    H = 3
    ref = O.State(st.pose, st.vel, st.theta)
    f_ref = []
    for k in range(H):
        f, _ = O.step(osc, wl.sim, ref, wl.q_traj, 3 + k, 1)
        f_ref.append(f)
    obs = np.zeros((H, wl.scene.n_pads, 3))
    for i in range(st.n):
        cost, _, fin, forces, _ = A.horizon(wl.scene, wl.sim, st.pose[i], st.vel[i], st.theta[i], wl.q_traj,
                                            3, H, obs, delta=np.zeros(8))
        np.testing.assert_allclose(fin[:3], ref.pose[i, :3], atol=1e-12)
        q = fin[3:7]
        assert abs(abs(np.dot(q, ref.pose[i, 3:])) - 1) < 1e-12
        np.testing.assert_allclose(fin[7:10], ref.vel[i, :3], atol=1e-10)
        np.testing.assert_allclose(fin[10:13], ref.vel[i, 3:], atol=1e-9)
        for k in range(H):
            np.testing.assert_allclose(forces[k], f_ref[k][i], rtol=1e-9, atol=1e-11)


def test_smoothed_gradient_equals_central_differences():
    warm, H = 18, 5
    wl, osc, st = _case(n=4, frames=warm + H + 2, warm=warm, name="tracking_cyl64")
    obs_state = O.State(st.pose[:1], st.vel[:1], np.array([wl.theta_gt]))
    obs = []
    for k in range(H):   # observations: the ground-truth parameters from env 0's start
        f, _ = O.step(osc, wl.sim, obs_state, wl.q_traj, warm + k, 1)
        obs.append(f[0])
    obs = np.array(obs)
    h = 1e-6
    checked = 0

    def central(args, c, step, sig):
        e = np.zeros(8)
        e[c] = step
        cp, _, _, _, sp = A.horizon(*args, smooth_forward=True, width=WIDTH, delta=e)
        cm, _, _, _, sm = A.horizon(*args, smooth_forward=True, width=WIDTH, delta=-e)
        if sp != sig or sm != sig:
            return None   # a branch (membership, clamp, face, bias regime) changes within the step
        return (cp - cm) / (2 * step)

    for i in range(st.n):
        args = (wl.scene, wl.sim, st.pose[i], st.vel[i], st.theta[i], wl.q_traj, warm, H, obs)
        cost, grad, _, _, sig = A.horizon(*args, smooth_forward=True, width=WIDTH)
        assert cost > 0 and np.all(np.isfinite(grad)) and np.any(grad != 0)
        for c in range(8):
            f1, f2 = central(args, c, h, sig), central(args, c, h / 2, sig)
            if f1 is None or f2 is None:
                continue
            fd = (4 * f2 - f1) / 3
            assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), abs(fd)) + 1e-8 * max(1.0, abs(cost)), (i, c, fd, grad[c])
            checked += 1
    assert checked >= 20


def test_unsmoothed_limit_equals_finite_differences_of_the_exact_forward():
    """With the smoothing taken to its limit (beta = 1e8 (N s)^-1, width 1e-8)
    the backward-smoothed gradient is the derivative of the exact,
    non-smooth forward: on components whose contact set, clamps and every
    projection's active side (normal clamp, disk clamp, per contact and
    iteration) stay unchanged within the step, it equals central finite
    differences of the exact forward (steps 1e-7 and 5e-8, Richardson) to
    1e-5 relative."""
    warm, H = 18, 5
    wl, osc, st = _case(n=4, frames=warm + H + 2, warm=warm, name="tracking_cyl64")
    obs_state = O.State(st.pose[:1], st.vel[:1], np.array([wl.theta_gt]))
    obs = np.array([O.step(osc, wl.sim, obs_state, wl.q_traj, warm + k, 1)[0][0] for k in range(H)])
    checked = 0
    for i in (0, 3):
        args = (wl.scene, wl.sim, st.pose[i], st.vel[i], st.theta[i], wl.q_traj, warm, H, obs)
        cost, grad, _, _, sig = A.horizon(*args, beta=1e8, width=1e-8, record_regimes=True)
        for c in range(8):
            fds, stable = [], True
            for h in (1e-7, 5e-8):
                e = np.zeros(8)
                e[c] = h
                cp = A.horizon(*args, delta=e, record_regimes=True)
                cm = A.horizon(*args, delta=-e, record_regimes=True)
                stable &= cp[4] == sig and cm[4] == sig
                fds.append((cp[0] - cm[0]) / (2 * h))
            if not stable:
                continue
            fd = (4 * fds[1] - fds[0]) / 3
            assert abs(fd - grad[c]) <= 1e-5 * max(abs(grad[c]), abs(fd)) + 1e-9, (i, c, fd, grad[c])
            checked += 1
    assert checked >= 12
