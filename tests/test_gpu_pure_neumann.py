"""Pure-Neumann problems (no outer box) through the augmented system (Sec. 2.3) on the GPU.

* one FP64 V-cycle (augmented coarse solve) against the oracle's, 1e-12 relative;
* a polynomial of degree <= q: the solution is P minus its mean over the unknowns
  (the constraint gamma = 0), exactly up to the tolerance;
* a smooth manufactured solution: the GPU solution equals the oracle's augmented
  solution (both mean-free), 1e-9 relative, and the mean-free error is small.
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu


def _ellipse(n, order, solution=None):
    return W.ProblemSpec(n=n, geometry=W.Geometry(W.ELLIPSE, (0.01, -0.02, 0.6, 0.45, 0.3), True), bc=W.NEUMANN,
                         order=order, solution=solution)


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("order", [4, 6])
def test_pure_neumann_vcycle_and_polynomial_solution(env, order):
    torch, iim = env
    spec = _ellipse(72, order)
    spec.solution = W.Polynomial(2, order, np.random.default_rng(order)).manufactured()
    O = OracleProblem(spec)
    assert O.singular
    P = gpu_problem(iim, spec, mg_precision=iim.MG_FP64, tol=1e-13)
    v = np.random.default_rng(3).standard_normal(P.N) * O.unk_flat
    assert rel_err(P.precondition(dev(v)).cpu().numpy(), O.precondition(v)) < 1e-12
    set_gpu_data(P, spec)
    x, info = P.solve()
    assert info.converged, info.as_dict()
    unk = O.unk_flat
    ex = O.exact()
    ex0 = np.where(unk, ex - ex[unk].mean(), 0.0)
    xg = x.cpu().numpy()
    assert abs(xg[unk].sum()) < 1e-8 * np.abs(ex0).sum()
    assert rel_err(xg, ex0) < 1e-9


def test_pure_neumann_smooth_solution_matches_oracle(env):
    torch, iim = env
    spec = _ellipse(96, 4, W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))
    P = gpu_problem(iim, spec, tol=1e-12)
    set_gpu_data(P, spec)
    x, info = P.solve()
    assert info.converged, info.as_dict()
    O = OracleProblem(spec)
    f, data = O.data()
    xo, oinfo, _ = O.solve(f, data, tol=1e-13)
    unk = O.unk_flat
    xg = x.cpu().numpy()
    assert rel_err(xg - np.where(unk, xg[unk].mean(), 0), xo - np.where(unk, xo[unk].mean(), 0)) < 1e-9
    ex = O.exact()
    e = (xg - xg[unk].mean()) - (ex - ex[unk].mean())
    assert np.max(np.abs(e[unk])) < 1e-5
