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
    wl = W.make_workload("tracking_box27", n_envs=n, frames=6)
    sim = start(wl, n=n, frames=6)
    sim.sim_step(0, 2)
    c_sum = torch.zeros(n, dtype=torch.float64, device=d)     # the caller's own window sums
    mean_static = torch.empty(n, dtype=torch.float64, device=d)
    am_static = torch.empty(1, dtype=torch.int32, device=d)
    mean_ref = torch.empty(n, dtype=torch.float64, device=d)
    am_ref = torch.empty(1, dtype=torch.int32, device=d)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    obs = None
    for call in (1, 2):
        sim.sim_step(1 + call, 1)
        forces, status = sim.sim_read_sensors()
        if obs is None:
            obs = forces[11].clone()
        sim.cost_eval(obs, mean_ref, am_ref)
        rc = fn(C.c_void_p(forces.data_ptr()), C.c_void_p(obs.data_ptr()), C.c_void_p(status.data_ptr()),
                n, wl.scene.n_pads, wl.sim.tau, wl.sim.w_force, wl.sim.w_contact,
                C.c_void_p(c_sum.data_ptr()), call, C.c_void_p(mean_static.data_ptr()),
                C.c_void_p(am_static.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(mean_static, mean_ref), float((mean_static - mean_ref).abs().max())
        assert int(am_static.item()) == int(am_ref.item())
        assert float(mean_ref[11].item()) <= float(mean_ref.min().item()) + 0.0


def test_cost_eval_static_rejects_sizes_beyond_its_scratch():
    d = dev()
    fn = _lib()
    dummy = torch.zeros(16, dtype=torch.float64, device=d)
    p = C.c_void_p(dummy.data_ptr())
    assert fn(p, p, None, 131073, 8, 0.02, 1.0, 1.0, p, 1, None, p, None) == 6   # IH_ERR_OVERFLOW
    assert fn(p, p, None, 10, 33, 0.02, 1.0, 1.0, p, 1, None, p, None) == 1      # IH_ERR_ARG
