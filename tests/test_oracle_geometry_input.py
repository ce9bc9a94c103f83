"""Oracle pins for geometry given as a level set on the grid or as a parametric curve
(the problem statement of Secs. 2.1-2.2: Omega+ = {phi > 0} for a level set phi; the
level-set domain of Sec. 4.4).

* The degree-5 Lagrange weights reproduce polynomials of degree <= 5 and their first two
  derivatives exactly, and not degree 6 (teeth); they sum to one.
* A grid level set sampled from a quadratic (circle, rotated ellipse, sphere, ellipsoid)
  is reproduced exactly by the interpolant, so it must give the analytic body's phase,
  control points, normals and curvatures, and the same IIM operator.
* A one-mode Fourier curve r = r0 + a cos m theta + b sin m theta is the star
  r0 + amp sin(m theta + phase) (a = amp sin phase, b = amp cos phase): same control
  points, normals, curvatures and operator.
* The Fourier curvature formula against the curvature of the parametric curve
  x(theta) = c + r(theta) (cos theta, sin theta) by central differences of x.
* A grid level set sampled from a non-polynomial field (the star) converges to the
  analytic body at the interpolant's order: control points at O(h^6).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.geometry import Crossings, LevelSet, phase_plus
from oracle.operator import IIMOperator

RNG = np.random.default_rng(2503)


def _grid_ls(values):
    return LevelSet(W.Geometry(W.LEVELSET_GRID, (), False, values=values))


@pytest.mark.parametrize("order", [0, 1, 2])
def test_lagrange_weights_exact_to_degree_5(order):
    n = 40
    ls = _grid_ls(np.zeros((n, n)))
    h = 2.0 / n
    x = np.concatenate([RNG.uniform(-1, 1, 200), -1 + (np.arange(n) + 0.5) * h])   # nodes included
    s, w = ls._lagrange(x, order)
    nodes = -1 + (s[:, None] + np.arange(6)) * h + 0.5 * h
    for deg in range(7):
        c = RNG.standard_normal(deg + 1)
        P = np.polynomial.Polynomial(c)
        exact = P.deriv(order)(x) if order <= deg else np.zeros_like(x)
        got = np.sum(w * P(nodes), axis=1)
        err = np.max(np.abs(got - exact)) / max(1.0, np.max(np.abs(exact)))
        if deg <= 5:
            assert err < 1e-9 * 10 ** order, (deg, err)
        elif order == 0:
            assert err > 1e-9, "a degree-6 polynomial must not be reproduced"
    if order == 0:
        assert np.allclose(np.sum(w, axis=1), 1.0, atol=1e-13)
        # at the nodes the weights are exactly one-hot
        wn = w[200:]
        assert np.all((wn == 0.0) | (wn == 1.0)) and np.all(np.sum(wn, axis=1) == 1.0)


def _compare(A, B, n, tol_x=1e-13, tol_n=1e-12, tol_k=1e-8):
    pa, pb = phase_plus(A, n), phase_plus(B, n)
    assert np.array_equal(pa, pb)
    ca, cb = Crossings(A, n, pa), Crossings(B, n, pb)
    assert ca.count == cb.count > 0
    assert np.array_equal(ca.axis, cb.axis) and np.array_equal(ca.lo, cb.lo)
    assert np.max(np.abs(ca.x - cb.x)) < tol_x
    assert np.max(np.abs(ca.normal - cb.normal)) < tol_n
    assert np.max(np.abs(ca.kappa - cb.kappa) / np.maximum(1.0, cb.kappa)) < tol_k


QUADRICS = [
    ("ellipse", 64, W.quadric_field((0.03, -0.02), (0.5, 0.35), 0.4),
     W.Geometry(W.ELLIPSE, (0.03, -0.02, 0.5, 0.35, 0.4), True)),
    ("circle", 48, W.quadric_field((-0.04, 0.05), (0.55, 0.55)),
     W.Geometry(W.CIRCLE, (-0.04, 0.05, 0.55), True)),
    ("sphere", 24, W.quadric_field((0.02, -0.01, 0.03), (0.6, 0.6, 0.6)),
     W.Geometry(W.SPHERE, (0.02, -0.01, 0.03, 0.6), True)),
    ("ellipsoid", 24, W.quadric_field((0.0, 0.02, -0.01), (0.6, 0.45, 0.5)),
     W.Geometry(W.ELLIPSOID, (0.0, 0.02, -0.01, 0.6, 0.45, 0.5), True)),
]


@pytest.mark.parametrize("name,n,field,analytic", QUADRICS, ids=[q[0] for q in QUADRICS])
def test_quadratic_grid_level_set_is_the_analytic_body(name, n, field, analytic):
    dim = analytic.dim
    grid = W.sampled_levelset(field, n, dim)
    _compare(LevelSet(grid), LevelSet(analytic), n)


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.NEUMANN, W.INTERFACE])
def test_quadratic_grid_level_set_gives_the_analytic_operator(bc):
    n = 48
    field = W.quadric_field((0.03, -0.02), (0.45, 0.3), 0.4)
    analytic = W.Geometry(W.ELLIPSE, (0.03, -0.02, 0.45, 0.3, 0.4), bc == W.DIRICHLET)
    grid = W.sampled_levelset(field, n, 2, plus_inside=False)
    if bc != W.DIRICHLET:      # exterior problems: Omega+ outside, phi = -field
        grid = W.Geometry(W.LEVELSET_GRID, (), True, values=grid.values)
    box = W.BOX_NONE if bc == W.DIRICHLET else W.BOX_DIRICHLET
    specs = [W.ProblemSpec(n=n, geometry=g, bc=bc, order=6, box_bc=box, beta_plus=1.0, beta_minus=2.0)
             for g in (grid, analytic)]
    A, B = IIMOperator(specs[0]), IIMOperator(specs[1])
    u = RNG.standard_normal(n * n)
    ra, rb = A.apply(u), B.apply(u)
    assert np.max(np.abs(ra - rb)) < 1e-11 * np.max(np.abs(rb))


def _star_as_fourier(cx, cy, r0, amp, m, ph):
    coef = [r0] + [0.0] * (2 * int(m))
    coef[2 * int(m) - 1] = amp * math.sin(ph)
    coef[2 * int(m)] = amp * math.cos(ph)
    return W.Geometry(W.FOURIER, (cx, cy), False, coef=tuple(coef))


def test_one_mode_fourier_curve_is_the_star():
    n = 96
    star = W.Geometry(W.STAR, (0.02, -0.01, 0.5, 0.08, 5.0, 0.3), False)
    four = _star_as_fourier(0.02, -0.01, 0.5, 0.08, 5, 0.3)
    _compare(LevelSet(four), LevelSet(star), n, tol_x=1e-14, tol_n=1e-13, tol_k=1e-12)
    specs = [W.ProblemSpec(n=n, geometry=g, bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET) for g in (four, star)]
    A, B = IIMOperator(specs[0]), IIMOperator(specs[1])
    u = RNG.standard_normal(n * n)
    assert np.max(np.abs(A.apply(u) - B.apply(u))) < 1e-11 * np.max(np.abs(B.apply(u)))


def test_fourier_curvature_matches_the_parametric_curve():
    coef = (0.5, 0.03, -0.02, 0.0, 0.025, 0.01, 0.0, 0.0, 0.008)
    ls = LevelSet(W.Geometry(W.FOURIER, (0.01, 0.02), False, coef=coef))
    th = np.linspace(0, 2 * np.pi, 97)[:-1]
    r, _, _ = ls._fourier(th)
    c = np.array([0.01, 0.02])

    def curve(t):
        rr, _, _ = ls._fourier(t)
        return c + rr[..., None] * np.stack([np.cos(t), np.sin(t)], axis=-1)
    e = 1e-4
    x0, xp, xm = curve(th), curve(th + e), curve(th - e)
    d1 = (xp - xm) / (2 * e)
    d2 = (xp - 2 * x0 + xm) / (e * e)
    kappa_fd = np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]) / np.sum(d1 * d1, axis=1) ** 1.5
    assert np.max(np.abs(ls.curvature(x0) - kappa_fd)) < 1e-5 * np.max(kappa_fd)
    # the points lie on the curve: g = 0
    assert np.max(np.abs(ls.g(x0))) < 1e-14


def test_grid_star_converges_to_the_analytic_star_at_order_6():
    star = W.Geometry(W.STAR, (0.02, -0.01, 0.5, 0.05, 5.0, 0.3), True)
    field = W.star_field(0.02, -0.01, 0.5, 0.05, 5.0, 0.3)
    errs = []
    ns = (96, 192)
    for n in ns:
        A = LevelSet(W.sampled_levelset(field, n, 2))
        B = LevelSet(star)
        pa, pb = phase_plus(A, n), phase_plus(B, n)
        assert np.array_equal(pa, pb)
        ca, cb = Crossings(A, n, pa), Crossings(B, n, pb)
        errs.append(np.max(np.abs(ca.x - cb.x)))
    slope = math.log(errs[0] / errs[1]) / math.log(ns[1] / ns[0])
    assert slope > 5.0, (errs, slope)
