"""The batched engine against single solves.

A slot's work is split into the same thread blocks as the single-problem solve,
so its iterates are the same floating-point operations in the same order: the
engine's solution and iteration count must equal iim_solve's bit for bit, for a
problem alone in the engine and for the same problem among others of other
sizes, orders, boundary conditions and dimensions, under any tile shape the
autotuner may pick.  Each single solve is itself checked against the oracle
elsewhere; here one mixed case is also checked against the manufactured solution.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import gpu_problem, need_gpu, set_gpu_data

pytestmark = pytest.mark.gpu


def _cases():
    specs = [
        W.circle_dirichlet_64(64),
        W.star_interface_1024(128),
        W.ProblemSpec(n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN,
                      order=6, box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
        W.ellipsoid_neumann_256(48),               # |kappa h| = 0.20 (n = 32 would break Eq. 3's bound)
    ]
    specs += W.batch_specs(6, seed=7, n_lo=64, n_hi=256)
    return specs


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.fixture(scope="module")
def singles(env):
    """Each case solved alone with iim_solve (reference for the engine)."""
    torch, iim = env
    out = []
    for spec in _cases():
        P = gpu_problem(iim, spec)
        set_gpu_data(P, spec)
        x, info = P.solve()
        assert info.converged, spec.name
        out.append((spec, x.cpu().numpy(), info.iters))
        P.close()
    return out


def _engine_solve(iim, torch, specs, shapes=None, tune=False):
    E = iim.Engine(iim.default_options(), max_slots=max(4, len(specs)))
    if shapes is not None:
        E.set_shapes(shapes)
    probs, slots = [], []
    for spec in specs:
        P = gpu_problem(iim, spec)
        set_gpu_data(P, spec)
        probs.append(P)
        slots.append(E.admit(P))
    if tune:
        E.autotune(reps=2)
    ticks = E.solve_all()
    res = []
    for P, sl in zip(probs, slots):
        x = torch.zeros(P.N, dtype=torch.float64, device="cuda")
        info = E.release(sl, x)
        res.append((x.cpu().numpy(), info))
    E.close()
    for P in probs:
        P.close()
    return res, ticks


def test_engine_alone_equals_single_solve(env, singles):
    torch, iim = env
    for spec, x_ref, it_ref in singles:
        (res,), ticks = _engine_solve(iim, torch, [spec])
        x, info = res
        assert info.converged and info.iters == it_ref, (spec.name, info.as_dict(), it_ref)
        assert np.array_equal(x, x_ref), (spec.name, float(np.max(np.abs(x - x_ref))))
        assert ticks >= info.iters + info.restarts + 1


def test_engine_mix_equals_single_solves(env, singles):
    torch, iim = env
    specs = [s for s, _, _ in singles]
    res, ticks = _engine_solve(iim, torch, specs)
    for (spec, x_ref, it_ref), (x, info) in zip(singles, res):
        assert info.converged and info.iters == it_ref, (spec.name, info.as_dict(), it_ref)
        assert np.array_equal(x, x_ref), spec.name
    assert ticks <= max(info.iters + info.restarts for _, info in res) + 2


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_tile_shape_does_not_change_results(env, singles, shape):
    torch, iim = env
    specs = [s for s, _, _ in singles if s.dim == 2]
    ref = [x for s, x, _ in singles if s.dim == 2]
    res, _ = _engine_solve(iim, torch, specs, shapes=[shape] * 6)
    for x_ref, (x, info) in zip(ref, res):
        assert np.array_equal(x, x_ref)


def test_autotuned_engine_and_slot_reuse(env, singles):
    torch, iim = env
    specs = [s for s, _, _ in singles]
    res, _ = _engine_solve(iim, torch, specs, tune=True)
    for (spec, x_ref, _), (x, info) in zip(singles, res):
        assert np.array_equal(x, x_ref), spec.name
    # a slot freed by one problem and reused by another, with others still running
    E = iim.Engine(iim.default_options(), max_slots=2)
    spec_a, xa_ref, _ = singles[0]
    spec_b, xb_ref, _ = singles[1]
    Pa = gpu_problem(iim, spec_a)
    set_gpu_data(Pa, spec_a)
    Pb = gpu_problem(iim, spec_b)
    set_gpu_data(Pb, spec_b)
    sa = E.admit(Pa)
    sb = E.admit(Pb)
    E.run(3)
    E.poll(wait=True)
    E.release(sa, check=False)                    # cancelled after three ticks
    Pa2 = gpu_problem(iim, spec_a)
    set_gpu_data(Pa2, spec_a)
    sa2 = E.admit(Pa2)
    assert sa2 == sa
    E.solve_all()
    xa = torch.zeros(Pa2.N, dtype=torch.float64, device="cuda")
    xb = torch.zeros(Pb.N, dtype=torch.float64, device="cuda")
    E.release(sa2, xa)
    E.release(sb, xb)
    assert np.array_equal(xa.cpu().numpy(), xa_ref)
    assert np.array_equal(xb.cpu().numpy(), xb_ref)


def test_engine_solution_error_against_manufactured(env):
    torch, iim = env
    spec = W.batch_specs(1, seed=11, n_lo=128, n_hi=128)[0]
    (res,), _ = _engine_solve(iim, torch, [spec])
    x, info = res
    P = gpu_problem(iim, spec)
    ph = P.phase().cpu().numpy().astype(bool)
    X = W.node_coords(spec.n, 2)
    ex = W.to_flat(spec.solution.u_plus(X))
    err = np.max(np.abs(x - ex)[ph])
    assert info.converged and err < 1e-5, err
