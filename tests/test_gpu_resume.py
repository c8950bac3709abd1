"""Checkpoint and resume of a tracking run through the C ABI.

The tracker's whole state between two windows is what sim_get_state returns
(pose, velocity, parameters, status) plus each environment's shape and solver
iteration count: the window's cost sums start from zero after every update,
the commanded trajectory and the observations are inputs, and the optimizer's
random numbers are Philox draws keyed by the handle's seed and counted by the
update index. So a run checkpointed after window 1 -- state read back, handle
destroyed, a new handle with the same seed given that state -- and resumed at
window 2 must reproduce the uninterrupted run bit for bit: every frame's
estimate and argmin, and the final state.
"""
import numpy as np
import pytest

from paper_2002_12160_gb300 import tracking, workloads as W

from gpu_common import dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n", [("tracking_cyl64", 256), ("uneven_mixed", 300)])
def test_resume_from_checkpoint_is_bit_identical(name, n):
    dev()
    T, windows, cut = 10, 4, 2
    wl = W.make_workload(name, n_envs=n, frames=windows * T)
    ref = tracking.Tracker(wl, n_envs=n)
    ref.prepare()
    for w in range(windows):
        ref.window(w)
    ref_state = [t.clone() for t in ref.sim.sim_get_state()]
    ref_est, ref_am = ref.est.clone(), ref.argmin.clone()
    ref.close()

    run = tracking.Tracker(wl, n_envs=n)
    run.prepare()
    for w in range(cut):
        run.window(w)
    ckpt = [t.clone() for t in run.sim.sim_get_state()]
    est0, am0 = run.est[:cut * T].clone(), run.argmin[:cut * T].clone()
    run.close()
    assert torch.equal(est0, ref_est[:cut * T]) and torch.equal(am0, ref_am[:cut * T])

    res = tracking.Tracker(wl, n_envs=n)
    res.prepare()
    d = dev()
    shape = torch.from_numpy(wl.shape_id[:n].astype(np.int32)).to(d)
    iters = torch.from_numpy(wl.iters[:n].astype(np.int32)).to(d)
    assert int((ckpt[3] != 0).sum()) == 0   # every diverged env was replaced at the update
    res.sim.sim_set_state(ckpt[0], ckpt[1], ckpt[2], shape, iters)
    for w in range(cut, windows):
        res.window(w)
    got = res.sim.sim_get_state()
    assert torch.equal(res.est[cut * T:], ref_est[cut * T:])
    assert torch.equal(res.argmin[cut * T:], ref_am[cut * T:])
    for a, b in zip(got, ref_state):
        assert torch.equal(a, b)
    res.close()
