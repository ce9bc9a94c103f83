"""Oracle pins for singular pure-Neumann problems (Sec. 2.3, augmented system).

* a polynomial of degree <= q with its Neumann data: the operator is exact, so the
  augmented solution is P minus its mean over the unknowns (gamma = 0) and the
  compatibility shift alpha is zero;
* gamma sets the sum of the solution over the unknowns;
* a smooth manufactured solution: the mean-free error converges at order >= n and
  alpha tends to zero (the discrete compatibility defect of the data).
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem


def _ellipse(n, order, solution=None):
    return W.ProblemSpec(n=n, geometry=W.Geometry(W.ELLIPSE, (0.0, 0.0, 0.6, 0.45, 0.3), True), bc=W.NEUMANN,
                         order=order, solution=solution)


@pytest.mark.parametrize("order", [4, 6])
def test_polynomial_solution_is_exact_up_to_its_mean(order):
    spec = _ellipse(56, order)
    spec.solution = W.Polynomial(2, order, np.random.default_rng(order)).manufactured()
    P = OracleProblem(spec)
    assert P.singular
    f, data = P.data()
    x, info, b = P.solve(f, data, tol=1e-13)
    unk = P.unk_flat
    ex = P.exact()
    ex0 = np.where(unk, ex - ex[unk].mean(), 0.0)
    assert info["converged"]
    assert np.max(np.abs(x - ex0)[unk]) < 1e-10 * np.max(np.abs(ex0))
    assert abs(info["alpha"]) < 1e-10 * np.max(np.abs(f[unk]))
    assert abs(x[unk].sum()) < 1e-9


def test_gamma_sets_the_additive_constant():
    spec = _ellipse(40, 4, W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))
    P = OracleProblem(spec)
    f, data = P.data()
    x0, i0, _ = P.solve(f, data, tol=1e-13)
    x1, i1, _ = P.solve(f, data, tol=1e-13, gamma=3.0)
    unk = P.unk_flat
    assert abs(x1[unk].sum() - 3.0) < 1e-9
    assert np.max(np.abs((x1 - x0)[unk] - 3.0 / unk.sum())) < 1e-10
    assert abs(i1["alpha"] - i0["alpha"]) < 1e-12


def test_mean_free_error_converges_and_alpha_vanishes():
    errs, alphas = [], []
    for n in (64, 128):
        P = OracleProblem(_ellipse(n, 4, W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)))
        f, data = P.data()
        x, info, _ = P.solve(f, data, tol=1e-13)
        unk = P.unk_flat
        ex = P.exact()
        e = (x - x[unk].mean()) - (ex - ex[unk].mean())
        errs.append(np.max(np.abs(e[unk])))
        alphas.append(abs(info["alpha"]))
    assert np.log2(errs[0] / errs[1]) > 4.0, errs
    assert alphas[1] < alphas[0] / 16, alphas
