"""Oracle pins: stencil coefficients (Tab. 1) and geometry (crossings, normals, curvature)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle.geometry import Crossings, LevelSet, phase_plus
from oracle.stencils import second_derivative, second_derivative_fractions, sigma, sigma_max

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_sigma():
    out = {}
    for line in open(os.path.join(GOLD, "sigma_max.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            o, v = line.split()
            out[int(o)] = Fraction(v)
    return out


@pytest.mark.parametrize("order", [2, 4, 6])
def test_sigma_max_matches_table1(order):
    gold = _golden_sigma()[order]
    assert sigma_max(order) == gold
    k = np.linspace(0, np.pi, 20001)
    assert abs(np.max(sigma(order, k)) - float(gold)) < 1e-12


def test_textbook_coefficients():
    # classical centred differences (e.g. Fornberg 1988 tables)
    assert second_derivative_fractions(2) == [Fraction(-2), Fraction(1)]
    assert second_derivative_fractions(4) == [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)]
    assert second_derivative_fractions(6) == [Fraction(-49, 18), Fraction(3, 2), Fraction(-3, 20), Fraction(1, 90)]


@pytest.mark.parametrize("order", [2, 4, 6])
def test_stencil_exact_to_degree_n_plus_1(order):
    """Moments sum_j a_j j^p equal p! [p == 2] up to p = n+1 and fail at p = n+2 (exact arithmetic)."""
    half = second_derivative_fractions(order)
    w = len(half) - 1
    a = {j: half[abs(j)] for j in range(-w, w + 1)}
    for p in range(0, order + 3):
        mom = sum(a[j] * Fraction(j) ** p for j in a if not (j == 0 and p == 0)) + (a[0] if p == 0 else 0)
        target = 2 if p == 2 else 0
        if p <= order + 1:
            assert mom == target
        else:
            assert mom != target
    # and the float version used by the operator agrees
    assert np.allclose(second_derivative(order), [float(a[j]) for j in range(-w, w + 1)], rtol=0, atol=1e-15)


def test_circle_crossings_normals():
    g = W.Geometry(W.CIRCLE, (0.01, -0.02, 0.5), plus_inside=True)
    ls = LevelSet(g)
    n = 64
    plus = phase_plus(ls, n)
    cr = Crossings(ls, n, plus)
    assert cr.count > 0
    r = np.hypot(cr.x[:, 0] - 0.01, cr.x[:, 1] + 0.02)
    assert np.max(np.abs(r - 0.5)) < 1e-13
    radial = (cr.x - np.array([0.01, -0.02])) / r[:, None]
    # Omega+ is the disc, so n points outwards
    assert np.max(np.abs(cr.normal - radial)) < 1e-12
    assert np.allclose(cr.kappa, 2.0)
    # each crossing lies on its edge, between nodes of different phase
    h = 2.0 / n
    assert np.all((cr.t >= 0) & (cr.t <= 1))
    # every phase change is represented exactly once
    changes = sum(np.count_nonzero(np.diff(plus.astype(int), axis=a)) for a in range(2))
    assert changes == cr.count


def test_star_curvature_against_level_set_differences():
    g = W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.1, 5.0, 0.0), plus_inside=False)
    ls = LevelSet(g)
    th = np.linspace(0.1, 6.0, 37)
    r = 0.5 + 0.1 * np.sin(5 * th)
    X = np.stack([r * np.cos(th), r * np.sin(th)], axis=-1)
    k = ls.curvature(X)
    # curvature as the divergence of the unit normal field, by central differences
    e = 1e-4

    def nrm(P):
        G = ls.grad_g(P)
        return G / np.linalg.norm(G, axis=-1, keepdims=True)

    div = np.zeros(th.size)
    for ax in range(2):
        dP = np.zeros(2)
        dP[ax] = e
        div += (nrm(X + dP)[:, ax] - nrm(X - dP)[:, ax]) / (2 * e)
    assert np.max(np.abs(np.abs(div) - k)) < 1e-5 * np.max(k)
    # closed form of the polar curvature at the tips: r = 0.6 (convex) and r = 0.4 (concave)
    tip = ls.curvature(np.array([[0.6 * np.cos(np.pi / 10), 0.6 * np.sin(np.pi / 10)],
                                 [0.4 * np.cos(-np.pi / 10), 0.4 * np.sin(-np.pi / 10)]]))
    assert abs(tip[0] - (0.36 + 0.6 * 2.5) / 0.6 ** 3) < 1e-12
    assert abs(tip[1] - abs(0.16 - 0.4 * 2.5) / 0.4 ** 3) < 1e-12     # 13.125


def test_ellipsoid_vertex_curvature():
    g = W.Geometry(W.ELLIPSOID, (0, 0, 0, 0.6, 0.45, 0.35), plus_inside=False)
    ls = LevelSet(g)
    k = ls.curvature(np.array([[0.6, 0.0, 0.0], [0.0, 0.0, 0.35]]))
    assert abs(k[0] - 0.6 / 0.35 ** 2) < 1e-12          # principal curvatures a/b^2, a/c^2
    assert abs(k[1] - 0.35 / 0.45 ** 2) < 1e-12
