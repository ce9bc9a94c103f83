"""Failure paths, made on the host (no fault, trap or hang of the GPU): every one ends in
a status the caller reads, and the problem, engine or server stays usable afterwards.

* NaN in the data: the first true residual is not finite, so FGMRES stops at once with
  IIM_ERR_BREAKDOWN (graph and host-driven loops alike); clean data then solve normally.
* max_iter below the iterations needed: IIM_ERR_NOT_CONVERGED with the iteration count
  and a finite relative residual above tol in the solve info.
* A request larger than the server's budget is refused at submission with IIM_ERR_BUDGET
  and the requests behind it are still served.
* Releasing a slot of the batched engine while its solve is unfinished cancels it
  (IIM_ERR_TIMEOUT, the state of the last run's tick) and leaves the engine usable.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import dev, gpu_data, gpu_problem, need_gpu, set_gpu_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("use_graph", [1, 0])
def test_nan_in_the_data_reports_breakdown(env, use_graph):
    torch, iim = env
    spec = W.star_interface_1024(128)
    P = gpu_problem(iim, spec, use_graph=use_graph)
    f, g, j0, j1, box = gpu_data(P, spec)
    bad = f.copy()
    bad[bad.size // 2 + 7] = np.nan
    P.set_data(dev(bad), dev(g), dev(j0), dev(j1), dev(box))
    x, info = P.solve(check=False)
    assert info.status == iim.IIM_ERR_BREAKDOWN and not info.converged
    assert info.iters == 0
    # the problem stays usable: clean data converge
    P.set_data(dev(f), dev(g), dev(j0), dev(j1), dev(box))
    x, info = P.solve(check=False)
    assert info.status == iim.IIM_OK and info.converged and info.relres <= 1e-10


def test_max_iter_reports_not_converged(env):
    torch, iim = env
    spec = W.star_interface_1024(128)
    P = gpu_problem(iim, spec, max_iter=3)
    set_gpu_data(P, spec)
    x, info = P.solve(check=False)
    assert info.status == iim.IIM_ERR_NOT_CONVERGED and not info.converged
    assert info.iters == 3
    assert np.isfinite(info.relres) and 1e-10 < info.relres < 1.0
    with pytest.raises(iim.IIMError) as e:
        P.solve()
    assert e.value.status == iim.IIM_ERR_NOT_CONVERGED


def test_budget_refusal_does_not_block_the_queue(env):
    torch, iim = env
    small = [W.circle_dirichlet_64(64), W.star_interface_1024(128), W.circle_dirichlet_64(80)]
    sizes = []
    for sp in small:
        P = gpu_problem(iim, sp)
        sizes.append(P.device_bytes())
        P.close()
    budget = int(1.5 * max(sizes))
    S = iim.Server(iim.default_options(), budget_bytes=budget, max_slots=4, ticks_per_run=3)
    with pytest.raises(iim.IIMError) as e:
        S.submit(iim.desc_from_spec(W.star_interface_1024(1024)))
    assert e.value.status == iim.IIM_ERR_BUDGET
    arrivals = [(0.0, iim.desc_from_spec(sp), sp) for sp in small]
    out, wall = iim.serve(S, arrivals, lambda view, sp: set_gpu_data(view, sp), realtime=False, deadline_s=120)
    stats = S.stats()
    S.close()
    assert len(out) == len(small)
    for x, info, lat, st, sp in out.values():
        assert st == 0 and info.converged, sp.name
    assert stats["peak_bytes"] <= budget


def test_engine_release_of_a_running_slot_cancels_it(env):
    torch, iim = env
    spec = W.star_interface_1024(128)
    ref = gpu_problem(iim, spec)
    set_gpu_data(ref, spec)
    x_ref, info_ref = ref.solve()
    E = iim.Engine(iim.default_options(), max_slots=4)
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    slot = E.admit(P)
    E.run(max_ticks=3)
    done, live, ticks = E.poll(wait=True)
    assert live == 1 and slot not in done
    x = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    info = E.release(slot, x, check=False)
    assert info.status == iim.IIM_ERR_TIMEOUT and not info.converged
    assert 0 < info.iters < info_ref.iters
    # the engine is still usable: the same problem, admitted again, solves to the single-solve result
    slot = E.admit(P)
    E.solve_all()
    info = E.release(slot, x)
    assert info.converged and info.iters == info_ref.iters
    assert torch.equal(x, x_ref)
    E.close()
