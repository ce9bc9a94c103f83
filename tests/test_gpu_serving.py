"""The request loop: results are the same alone and in the mix.

A stream of mixed 2D/3D requests goes through a server whose memory budget
holds only a few of them at a time, so requests wait in the queue and enter the
engine while others are still running.  Every request's solution must equal,
bit for bit, the solution of the same request served alone (and of iim_solve),
and the budget must never be exceeded.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import gpu_problem, need_gpu, set_gpu_data

pytestmark = pytest.mark.gpu


def _trace():
    # small sizes of the serving mix: 2D 64..256, 3D ellipsoids at 64 (|kappa h| < 1/4 needs n >= 49)
    return W.serving_trace(count=10, rate=1e9, seed=5, n2_lo=64, n2_hi=256, n3_lo=64, n3_hi=64, frac_3d=0.3)


@pytest.fixture(scope="module")
def env():
    return need_gpu()


def _serve(iim, specs, budget, ticks_per_run=3, mode=0, pooling=True, pool_stats=None, data_threads=0):
    S = iim.Server(iim.default_options(), budget_bytes=budget, max_slots=8, ticks_per_run=ticks_per_run, mode=mode,
                   pooling=pooling)
    arrivals = [(0.0, iim.desc_from_spec(sp), sp) for sp in specs]
    out, wall = iim.serve(S, arrivals, lambda view, sp: set_gpu_data(view, sp), realtime=False,
                          data_threads=data_threads)
    stats = S.stats()
    if pool_stats is not None:
        pool_stats.update(S.pool_stats())
    S.close()
    return [out[rid] for rid in sorted(out)], stats


@pytest.mark.parametrize("mode", [0, 1])
def test_served_results_equal_alone_and_single_solves(env, mode):
    """mode 0: requests advance together in the batched engine; mode 1: each request's
    solve graph on its own stream."""
    torch, iim = env
    specs = [sp for _, sp in _trace()]
    assert any(sp.dim == 3 for sp in specs) and any(sp.dim == 2 for sp in specs)
    # budget: the two largest requests at a time -> queueing and admission mid-run
    sizes = []
    for sp in specs:
        P = gpu_problem(iim, sp)
        sizes.append(P.device_bytes())
        P.close()
    budget = int(2.5 * max(sizes))
    mixed, stats = _serve(iim, specs, budget, mode=mode)
    assert stats["peak_bytes"] <= budget
    assert stats["runs"] > 3 or mode == 1
    assert len(mixed) == len(specs)
    for (x, info, lat, st, sp) in mixed:
        assert st == 0 and info.converged and info.relres <= 1e-10, (sp.name, info.as_dict())
        assert lat > 0
    for (x, info, lat, st, sp) in mixed:
        (alone,), _ = _serve(iim, [sp], 1 << 36, mode=mode)
        assert np.array_equal(alone[0], x), (sp.name, sp.n, sp.dim, "alone", alone[1].as_dict(), "mixed", info.as_dict(),
                                             float(np.max(np.abs(alone[0] - x))))
        assert alone[1].iters == info.iters
    # and the plain single solve of two of them
    for (x, info, lat, st, sp) in mixed[:2]:
        P = gpu_problem(iim, sp)
        set_gpu_data(P, sp)
        xs, si = P.solve()
        assert np.array_equal(xs.cpu().numpy(), x) and si.iters == info.iters
        P.close()


def test_request_larger_than_budget_is_refused(env):
    torch, iim = env
    sp = W.circle_dirichlet_64(64)
    S = iim.Server(iim.default_options(), budget_bytes=1 << 20, max_slots=2, ticks_per_run=2)
    with pytest.raises(iim.IIMError) as e:
        S.submit(iim.desc_from_spec(sp))
    assert e.value.status == 7
    S.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_every_request_reported_with_one_id_per_step(env, mode):
    """Arrays of capacity 1: ids that do not fit are reported by later steps, each once,
    and the final state counts are all zero once every request is taken."""
    torch, iim = env
    specs = [sp for _, sp in _trace()][:6]
    S = iim.Server(iim.default_options(), budget_bytes=1 << 36, max_slots=8, ticks_per_run=3, mode=mode, cap=1)
    arrivals = [(0.0, iim.desc_from_spec(sp), sp) for sp in specs]
    out, wall = iim.serve(S, arrivals, lambda view, sp: set_gpu_data(view, sp), realtime=False, deadline_s=120)
    st = S.stats()
    S.close()
    assert len(out) == len(specs)
    assert all(o[3] == 0 for o in out.values())
    assert sum(st["states"].values()) == 0


@pytest.mark.parametrize("mode", [1, 0])
def test_kept_problems_give_the_results_of_fresh_ones(env, mode):
    """Requests of a few kinds repeated with other geometry parameters, through a budget that
    holds about two problems: finished problems are kept and taken by later requests of the
    same kind (set-up re-run in place), or freed for room.  Every result equals, bit for bit,
    the result with reuse switched off (every request created afresh)."""
    torch, iim = env
    specs = []
    for k in range(4):
        specs.append(W.ProblemSpec(n=96, geometry=W.Geometry(W.CIRCLE, (0.01 * k, -0.02, 0.45 + 0.03 * k), True),
                                   bc=W.DIRICHLET, order=4, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)))
        specs.append(W.ProblemSpec(n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.38 + 0.02 * k, 0.3, 0.2 * k),
                                                             False),
                                   bc=W.NEUMANN, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=2.0,
                                   solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)))
    sizes = []
    for sp in specs[:2]:
        P = gpu_problem(iim, sp)
        sizes.append(P.device_bytes())
        P.close()
    budget = int(2.6 * max(sizes))
    ps = {}
    kept, _ = _serve(iim, specs, budget, mode=mode, pooling=True, pool_stats=ps)
    fresh, _ = _serve(iim, specs, budget, mode=mode, pooling=False)
    assert ps["hits"] > 0
    for (xa, ia, _, sa, sp), (xb, ib, _, sb, _) in zip(kept, fresh):
        assert sa == 0 and sb == 0 and ia.converged and ib.converged, sp.name
        assert ia.iters == ib.iters and np.array_equal(xa, xb), (sp.geometry, ia.as_dict(), ib.as_dict())


@pytest.mark.parametrize("mode", [1, 0])
def test_client_data_threads_give_the_same_results(env, mode):
    """Request data set on four client threads while the loop keeps stepping: every result
    equals, bit for bit, the result with the data set on the loop's own thread."""
    torch, iim = env
    specs = [sp for _, sp in _trace()]
    threaded, _ = _serve(iim, specs, 1 << 36, mode=mode, data_threads=4)
    inline, _ = _serve(iim, specs, 1 << 36, mode=mode, data_threads=0)
    assert len(threaded) == len(inline) == len(specs)
    for (xa, ia, _, sa, sp), (xb, ib, _, sb, _) in zip(threaded, inline):
        assert sa == 0 and sb == 0 and ia.converged, sp.name
        assert ia.iters == ib.iters and np.array_equal(xa, xb), sp.name


@pytest.mark.parametrize("mode", [1, 0])
def test_cancel_in_every_state(env, mode):
    """A request cancelled while queued, one cancelled instead of receiving its data, and a
    larger one cancelled right after the step that starts its solve: each is reported with
    IIM_ERR_TIMEOUT and no solution, every other request converges, nothing is left held."""
    torch, iim = env
    specs = [sp for _, sp in _trace()][:5]
    big = W.star_interface_1024(512)
    S = iim.Server(iim.default_options(), budget_bytes=1 << 36, max_slots=8, ticks_per_run=2, mode=mode)
    ids = [S.submit(iim.desc_from_spec(sp)) for sp in specs]
    big_id = S.submit(iim.desc_from_spec(big))
    users = dict(zip(ids + [big_id], specs + [big]))
    S.cancel(ids[0])                                   # queued
    cancelled = {ids[0], ids[1], big_id}
    out, started_big = {}, False
    need_q, fin_q = [], []
    import time
    t0 = time.perf_counter()
    while len(out) < len(users):
        assert time.perf_counter() - t0 < 120, S.stats()
        need, fin = S.step()
        need_q += need
        fin_q += fin
        while need_q:
            rid = need_q.pop(0)
            if rid == ids[1]:
                S.cancel(rid)                          # waiting for its data
                continue
            set_gpu_data(S.problem(rid), users[rid])
            S.data_ready(rid)
            if rid == big_id:
                need, fin = S.step()                   # its solve starts (mode 1) or joins a run (mode 0)
                need_q += need
                fin_q += fin
                S.cancel(big_id)                       # running
                started_big = True
        while fin_q:
            rid = fin_q.pop(0)
            out[rid] = S.take(rid)
    st = S.stats()
    S.close()
    assert started_big
    for rid, (x, info, lat, status) in out.items():
        if rid in cancelled:
            assert status == iim.IIM_ERR_TIMEOUT and not info.converged, users[rid].name
        else:
            assert status == 0 and info.converged, users[rid].name
    assert sum(st["states"].values()) == 0 and st["bytes_in_use"] == 0
