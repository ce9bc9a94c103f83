"""GPU FGMRES + SW-multigrid solves against the oracle and against the mathematics.

Converged solutions are unique (the discrete system is nonsingular), so the GPU
solve at tol 1e-12 must match the oracle's solve at tol 1e-13 to 1e-9 relative,
whatever the Krylov/multigrid rounding; the FP32-multigrid and FP64-multigrid
forms must agree with each other to the same bound; the residual the device
reports is re-computed with the oracle's own operator.
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_data, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu

SOLVE_CASES = {
    "circle_dirichlet_64": lambda: W.circle_dirichlet_64(64),
    "star_interface_6_128": lambda: W.star_interface_1024(128),
    "neumann_ext_6_80": lambda: W.ProblemSpec(
        n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN, order=6,
        box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
    "ellipsoid_neumann_48": lambda: W.ellipsoid_neumann_256(48),
}


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("case", sorted(SOLVE_CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_converged_solution_matches_oracle(env, case, prec):
    torch, iim = env
    spec = SOLVE_CASES[case]()
    P = gpu_problem(iim, spec, tol=1e-12, mg_precision=iim.MG_FP32 if prec == "fp32" else iim.MG_FP64)
    set_gpu_data(P, spec)
    x, info = P.solve()
    O = OracleProblem(spec)
    f, data = O.data()
    xo, oinfo, b = O.solve(f, data, tol=1e-13)
    xg = x.cpu().numpy()
    assert info.converged and info.relres <= 1e-12
    assert rel_err(xg, xo) < 1e-9
    # the residual recomputed by the oracle's operator
    r = b - O.op.apply(xg)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-12


def test_tolerance_1e10_and_manufactured_error(env):
    torch, iim = env
    spec = W.circle_dirichlet_64(64)
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    x, info = P.solve()
    O = OracleProblem(spec)
    xg = x.cpu().numpy()
    assert info.converged and info.relres <= 1e-10
    f, data = O.data()
    b = O.op.rhs(f, data)
    assert np.linalg.norm(b - O.op.apply(xg)) / np.linalg.norm(b) <= 1.01e-10
    assert np.max(np.abs(xg - O.exact())[O.unk_flat]) < 1e-7        # 4th order at n = 64: ~3e-8


def test_graph_and_host_loop_are_bitwise_equal(env):
    torch, iim = env
    spec = W.star_interface_1024(128)
    xs = []
    for graph in (1, 0):
        P = gpu_problem(iim, spec, use_graph=graph)
        set_gpu_data(P, spec)
        x, info = P.solve()
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


def test_resetup_in_place_equals_fresh_create(env):
    torch, iim = env
    spec = W.star_interface_1024(128)
    spec2 = W.star_interface_1024(128, phase=0.3)
    A = gpu_problem(iim, spec)
    A.setup(spec2.geometry.params)
    A.refresh_sizes()
    B = gpu_problem(iim, spec2)
    assert A.K == B.K
    for P in (A, B):
        set_gpu_data(P, spec2)
    xa, _ = A.solve()
    xb, _ = B.solve()
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())


def test_restart_from_solution_needs_no_iteration(env):
    torch, iim = env
    spec = W.circle_dirichlet_64(64)
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    x, info = P.solve()
    x2, info2 = P.solve(x.clone())
    assert info2.iters == 0 and info2.converged


def test_solve_host_equals_device_solve(env):
    torch, iim = env
    spec = W.ellipsoid_neumann_256(48)
    P = gpu_problem(iim, spec)
    f, g, j0, j1, box = gpu_data(P, spec)
    P.set_data(dev(f), dev(g), dev(j0), dev(j1), dev(box))
    xd, _ = P.solve()
    xh, info = P.solve_host(f, g, j0, j1, box)
    assert np.array_equal(xd.cpu().numpy(), xh)


def test_batch_results_equal_solo_results(env):
    torch, iim = env
    specs = W.batch_specs(count=6, seed=7, n_lo=64, n_hi=192)
    solo, probs, xs = [], [], []
    for spec in specs:
        P = gpu_problem(iim, spec)
        set_gpu_data(P, spec)
        x, _ = P.solve()
        solo.append(x.cpu().numpy())
        probs.append(P)
        xs.append(torch.zeros(P.N, dtype=torch.float64, device="cuda"))
    infos, st = iim.batch_solve(probs, xs)
    for s, x, inf in zip(solo, xs, infos):
        assert inf.converged
        assert np.array_equal(s, x.cpu().numpy())


def test_curvature_violation_is_reported(env):
    torch, iim = env
    spec = W.star_interface_1024(64)          # |kappa h| = 13.1 * 2/64 > 1/4
    with pytest.raises(iim.IIMError) as e:
        gpu_problem(iim, spec)
    assert e.value.status == 2


def test_body_touching_the_box_is_reported(env):
    torch, iim = env
    spec = W.ProblemSpec(n=64, geometry=W.Geometry(W.CIRCLE, (0.5, 0.0, 0.45), False), bc=W.NEUMANN, order=4,
                         box_bc=W.BOX_DIRICHLET, solution=W.sin_cos_2d(1, 0, 1, 0))
    with pytest.raises(iim.IIMError) as e:
        gpu_problem(iim, spec)
    assert e.value.status == 10


def test_non_power_of_two_grid(env):
    torch, iim = env
    spec = W.ProblemSpec(n=80, geometry=W.Geometry(W.STAR, (0.02, 0.0, 0.5, 0.03, 7.0, 0.2), True),
                         bc=W.DIRICHLET, order=4, solution=W.sin_cos_2d(1.7, 0.2, 2.1, 0.9))
    P = gpu_problem(iim, spec, tol=1e-12)
    set_gpu_data(P, spec)
    x, info = P.solve()
    O = OracleProblem(spec)
    f, data = O.data()
    xo, _, _ = O.solve(f, data, tol=1e-13)
    assert rel_err(x.cpu().numpy(), xo) < 1e-9
