"""cost_eval_static: the allocation-free cost entry point, for callers that
may not call cudaMalloc (they cannot create a simulator handle or give us
scratch space). Called here through the C ABI with ctypes, on buffers that
the test owns, and checked against cost_eval of a simulator handle on two
consecutive frames: window means bit for bit (the same FP64 arithmetic in the
same order) and the same argmin. The file name sorts last so that a run which
stops at its first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2002_12160_gb300 import workloads as W

from gpu_common import dev, start, torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2002_12160_gb300 import inhand
    lib = C.CDLL(inhand.LIB_PATH)
    fn = lib.cost_eval_static
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_float,
                   C.c_float, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    return fn


def test_cost_eval_static_matches_cost_eval_on_two_calls():
    d = dev()
    fn = _lib()
    n = 333
    wl = W.make_workload("tracking_box27", n_envs=n, frames=20)
    sim = start(wl, n=n, frames=20)
    sim.sim_step(0, 16)   # the grasp has closed: finger pads carry force
    c_sum = torch.zeros(n, dtype=torch.float64, device=d)     # the caller's own window sums
    mean_static = torch.empty(n, dtype=torch.float64, device=d)
    am_static = torch.empty(1, dtype=torch.int32, device=d)
    mean_ref = torch.empty(n, dtype=torch.float64, device=d)
    am_ref = torch.empty(1, dtype=torch.int32, device=d)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    obs = None
    for call in (1, 2):
        sim.sim_step(15 + call, 1)
        forces, status = sim.sim_read_sensors()
        if obs is None:   # the environment with the most pad force observes itself
            me = int(forces.abs().sum(dim=(1, 2)).argmax().item())
            obs = forces[me].clone()
        sim.cost_eval(obs, mean_ref, am_ref)
        rc = fn(C.c_void_p(forces.data_ptr()), C.c_void_p(obs.data_ptr()), C.c_void_p(status.data_ptr()),
                n, wl.scene.n_pads, wl.sim.tau, wl.sim.w_force, wl.sim.w_contact,
                C.c_void_p(c_sum.data_ptr()), call, C.c_void_p(mean_static.data_ptr()),
                C.c_void_p(am_static.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(mean_static, mean_ref), float((mean_static - mean_ref).abs().max())
        assert int(am_static.item()) == int(am_ref.item())
        if call == 1:   # that environment scored against its own forces: cost 0, the unique minimum
            assert float(mean_ref[me].item()) == 0.0 and int(am_ref.item()) == me
            assert int((mean_ref == 0).sum().item()) == 1


def test_cost_eval_static_status_and_diverged_environments():
    """Without a status array every environment is scored; with one, the
    environments marked diverged score +inf (the rest unchanged, bit for bit)
    and the argmin moves to the lowest remaining window mean, lowest index on
    ties."""
    d = dev()
    fn = _lib()
    n = 300
    wl = W.make_workload("tracking_box27", n_envs=n, frames=20)
    sim = start(wl, n=n, frames=20)
    sim.sim_step(0, 17)   # finger pads carry force
    forces, status = sim.sim_read_sensors()
    assert int(status.abs().sum().item()) == 0
    me = int(forces.abs().sum(dim=(1, 2)).argmax().item())
    obs = forces[me].clone()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(st):
        c_sum = torch.zeros(n, dtype=torch.float64, device=d)
        mean = torch.empty(n, dtype=torch.float64, device=d)
        am = torch.empty(1, dtype=torch.int32, device=d)
        rc = fn(C.c_void_p(forces.data_ptr()), C.c_void_p(obs.data_ptr()),
                None if st is None else C.c_void_p(st.data_ptr()), n, wl.scene.n_pads, wl.sim.tau,
                wl.sim.w_force, wl.sim.w_contact, C.c_void_p(c_sum.data_ptr()), 1, C.c_void_p(mean.data_ptr()),
                C.c_void_p(am.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        return mean.cpu().numpy(), int(am.item())

    m_none, a_none = call(None)
    m_zero, a_zero = call(status)
    np.testing.assert_array_equal(m_none, m_zero)
    assert a_none == a_zero == me
    marked = sorted({3, me, 200, int(np.argsort(m_none, kind="stable")[1])})
    st = torch.zeros(n, dtype=torch.int32, device=d)
    st[marked] = 1   # IH_ENV_NONFINITE
    m_div, a_div = call(st)
    assert np.all(np.isinf(m_div[marked]) & (m_div[marked] > 0))
    keep = np.setdiff1d(np.arange(n), marked)
    np.testing.assert_array_equal(m_div[keep], m_none[keep])
    rest = m_none.copy()
    rest[marked] = np.inf
    assert a_div == int(np.argmin(rest)) and a_div not in marked


def test_cost_eval_static_rejects_sizes_beyond_its_scratch():
    d = dev()
    fn = _lib()
    dummy = torch.zeros(16, dtype=torch.float64, device=d)
    p = C.c_void_p(dummy.data_ptr())
    assert fn(p, p, None, 131073, 8, 0.02, 1.0, 1.0, p, 1, None, p, None) == 6   # IH_ERR_OVERFLOW
    assert fn(p, p, None, 10, 33, 0.02, 1.0, 1.0, p, 1, None, p, None) == 1      # IH_ERR_ARG
