"""The end-to-end driver (inputs from pinned host buffers, outputs read back)
against the same windows run from device-resident inputs."""
import pytest

from paper_2002_12160_gb300 import workloads as W

from gpu_common import dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("workload,n", [("tracking_box27", 64), ("tracking_cyl64", 300)])
def test_end_to_end_windows_equal_the_device_windows(workload, n):
    """Tracker.e2e_windows -- its pipelined half (every window's packed inputs
    copied up, its commands' kinematics, the window, its outputs copied back,
    all enqueued on the handle's one stream with a single synchronisation at
    the end) and its half with the host waiting for every window -- gives the
    estimates and argmins of the same windows launched from device-resident
    commands and observations, bit for bit, and leaves the same state
    behind."""
    from paper_2002_12160_gb300 import tracking
    dev()
    count = 6
    wl = W.make_workload(workload, n_envs=n, frames=count * 10)
    a = tracking.Tracker(wl)
    b = tracking.Tracker(wl)
    a.prepare()
    b.prepare()
    T = a.T
    assert count * T <= wl.frames
    for w in range(count):
        a.window(w)
    b.e2e_windows(0, count)
    torch.cuda.synchronize()
    assert torch.equal(a.est[:count * T], b.est[:count * T])
    assert torch.equal(a.argmin[:count * T], b.argmin[:count * T])
    for x, y in zip(a.sim.sim_get_state(), b.sim.sim_get_state()):
        assert torch.equal(x, y)
    a.close()
    b.close()
