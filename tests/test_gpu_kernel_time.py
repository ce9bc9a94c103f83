"""The profiling entry points: every kernel case times to a positive duration on a problem
that uses it, the flushed form (L2 overwritten before each launch) is not faster than the
back-to-back form by more than noise, and a problem without fused first-level multigrid
kernels refuses those cases."""
import pytest

import workloads as W
from tests.gpu_helpers import gpu_problem, need_gpu, set_gpu_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return need_gpu()


def test_every_case_times(env):
    torch, iim = env
    spec = W.star_interface_1024(256)
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for name in iim.KERNELS:
        us = iim.kernel_time(P, name, reps=3)
        assert us > 0, name
    for name in ("mg_down0", "mg_up0", "mg_tail", "stencil"):
        cold = iim.kernel_time(P, name, reps=5, flush=flush)
        warm = iim.kernel_time(P, name, reps=20)
        assert cold > 0 and cold > 0.5 * warm, (name, cold, warm)


def test_fused_first_level_cases_refused_in_3d(env):
    torch, iim = env
    spec = W.perturbed_sphere(40)
    P = gpu_problem(iim, spec)
    assert iim.kernel_time(P, "mg_tail", reps=2) > 0
    for name in ("mg_down0", "mg_up0"):
        with pytest.raises(iim.IIMError):
            iim.kernel_time(P, name, reps=2)
