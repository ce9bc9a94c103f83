"""Oracle pins for the radially perturbed sphere of the paper's 3D verification (Sec. 4.2).

The body is r(e) = rho0 + rho1 Y(e) with Y the degree-3 spherical harmonic
(e_x^2 - e_y^2) e_z scaled to max |Y| = 1 (the paper names a spherical harmonic without
giving its degree).  Pins:

* the level set's gradient and Hessian against central differences of g, a symmetric
  Hessian, curvature 1/rho0 without the perturbation, and the closed-form extremum of Y:
  the surface passes through rho0 + rho1 along (sqrt(2/3), 0, 1/sqrt(3));
* the IIM operator reproduces polynomials of degree <= q = 4 exactly on this body, for
  Dirichlet and (pure) Neumann conditions, and not degree 5;
* the manufactured solution of Sec. 4.2 (the sum of sin(4 pi x_i) on the unit cube) shows
  an error decay of order >= 3.5 for both conditions (measured: 4.6 Dirichlet, 5.0-6.3
  Neumann at n = 24, 32, 40, pre-asymptotic).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.geometry import LevelSet
from oracle.problem import OracleProblem
from tests.test_oracle_operator import _exactness_error


def _ls(rho1=0.1, c=(0.01, -0.02, 0.03)):
    return LevelSet(W.Geometry(W.PERTURBED_SPHERE, (c[0], c[1], c[2], 0.7, rho1), True))


def test_level_set_derivatives_and_closed_forms():
    ls = _ls()
    X = np.random.default_rng(0).uniform(-0.9, 0.9, (30, 3))
    e = 1e-5
    I = np.eye(3)
    G, H = ls.grad_g(X), ls.hess_g(X)
    Gfd = np.stack([(ls.g(X + e * I[k]) - ls.g(X - e * I[k])) / (2 * e) for k in range(3)], -1)
    Hfd = np.stack([(ls.grad_g(X + e * I[k]) - ls.grad_g(X - e * I[k])) / (2 * e) for k in range(3)], -1)
    assert np.max(np.abs(G - Gfd)) < 1e-8 * max(1.0, np.max(np.abs(G)))
    assert np.max(np.abs(H - Hfd)) < 1e-6 * max(1.0, np.max(np.abs(H)))
    assert np.max(np.abs(H - np.swapaxes(H, -1, -2))) < 1e-12
    flat = _ls(rho1=0.0, c=(0.0, 0.0, 0.0))
    assert np.allclose(flat.curvature(np.array([[0.7, 0, 0], [0, 0.7, 0], [0, 0, -0.7]])), 1 / 0.7, rtol=1e-12)
    e_star = np.array([math.sqrt(2.0 / 3.0), 0.0, 1.0 / math.sqrt(3.0)])
    c = np.array([0.01, -0.02, 0.03])
    assert abs(ls.g((c + 0.8 * e_star)[None])[0]) < 1e-14
    # the centre itself is inside, with the harmonic term taken as 0
    assert ls.g(c[None])[0] == -0.7


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.NEUMANN])
def test_polynomial_exactness_and_teeth(bc):
    assert _exactness_error(W.perturbed_sphere(24, bc), 4) < 5e-10
    assert _exactness_error(W.perturbed_sphere(24, bc), 5) > 1e-4


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.NEUMANN])
def test_manufactured_convergence(bc):
    errs = []
    ns = (24, 32)
    for n in ns:
        P = OracleProblem(W.perturbed_sphere(n, bc))
        f, data = P.data()
        x, info, _ = P.solve(f, data, tol=1e-12)
        assert info["converged"]
        unk = P.unk_flat
        err = x - P.exact()
        if P.singular:
            err = err - np.where(unk, err[unk].mean(), 0.0)
        errs.append(np.max(np.abs(err[unk])))
    order = math.log(errs[0] / errs[1]) / math.log(ns[1] / ns[0])
    assert order >= 3.5, (errs, order)
