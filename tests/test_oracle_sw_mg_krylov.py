"""Oracle pins for the preconditioner (Sec. 3) and the Krylov solver (Sec. 4.1).

* every 1D Shortley-Weller formula (Eqs. 18-19) is exact on quadratics, the
  defining property stated in Sec. 3.1; the interface wall values (Eq. 21)
  reproduce piecewise-linear flux-continuous functions exactly;
* the V-cycle iterated as a solver converges to the sparse direct solution of
  the SW system (Sec. 3.3) and contracts fast for Dirichlet;
* FGMRES: an exact preconditioner converges in one iteration; with the
  identity it solves a nonsymmetric system like a dense solve; on small grids
  the converged IIM solution equals the brute-force dense solve;
* manufactured solutions converge at order n (Sec. 2.4, Fig. 3; Sec. 2.5 interface).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle.dense import assemble
from oracle.fgmres import fgmres
from oracle.geometry import LevelSet
from oracle.mg import Multigrid, level_sizes
from oracle.problem import OracleProblem
from oracle.sw import (sw_dirichlet, sw_interface_walls, sw_neumann_both, sw_neumann_left,
                       sw_neumann_right)

RNG = np.random.default_rng(11)


def _quad(c0, c1, c2):
    return (lambda x: c0 + c1 * x + 0.5 * c2 * x * x), (lambda x: c1 + c2 * x), c2


@pytest.mark.parametrize("trial", range(20))
def test_sw_1d_formulas_exact_on_quadratics(trial):
    c0, c1, c2 = RNG.standard_normal(3)
    u, du, d2 = _quad(c0, c1, c2)
    dx = RNG.uniform(0.01, 0.3)
    pm, pp = RNG.uniform(0.05, 1.0, size=2)
    xi = RNG.uniform(-1, 1)
    # Dirichlet (c): walls on both sides
    assert abs(sw_dirichlet(u(xi - pm * dx), u(xi), u(xi + pp * dx), pm, pp, dx) - d2) < 1e-8 / dx
    # (a)/(b): one regular neighbour (psi = 1)
    assert abs(sw_dirichlet(u(xi - dx), u(xi), u(xi + pp * dx), 1.0, pp, dx) - d2) < 1e-8 / dx
    # Neumann (a): wall at xi - pm dx, regular node at xi + pp dx
    assert abs(sw_neumann_left(du(xi - pm * dx), u(xi), u(xi + pp * dx), pm, pp, dx) - d2) < 1e-8 / dx
    # Neumann (b): regular node at xi - pm dx, wall at xi + pp dx
    assert abs(sw_neumann_right(u(xi - pm * dx), u(xi), du(xi + pp * dx), pm, pp, dx) - d2) < 1e-8 / dx
    # Neumann (c): walls on both sides
    assert abs(sw_neumann_both(du(xi - pm * dx), du(xi + pp * dx), pm, pp, dx) - d2) < 1e-8 / dx


def test_sw_neumann_b_printed_form_is_not_exact():
    """The printed case (b), with psi+ in the first two denominators, fails the quadratic test."""
    u, du, d2 = _quad(0.2, -0.7, 1.3)
    dx, pm, pp, xi = 0.1, 0.7, 0.6, 0.0

    def printed(uim1, ui, dup):
        return (2 * uim1 / (pp * (pm + 2 * pp)) - 2 * ui / (pp * (pm + 2 * pp)) + 2 * dx * dup / (pm + 2 * pp)) / dx ** 2
    assert abs(printed(u(xi - pm * dx), u(xi), du(xi + pp * dx)) - d2) > 1e-3


@pytest.mark.parametrize("trial", range(10))
def test_sw_interface_walls_solve_the_discrete_jump_conditions(trial):
    """Eq. 21 returns wall values with uw+ - uw- = [u] and the flux balance of Eq. 20."""
    bm, bp = RNG.uniform(0.1, 5, size=2)
    pm, pp = RNG.uniform(0.1, 0.9, size=2)
    dx = RNG.uniform(0.01, 0.2)
    ui, uip1, J, F = RNG.standard_normal(4)
    uwp, uwm = sw_interface_walls(ui, uip1, J, F, pm, pp, bm, bp, dx)
    assert abs((uwp - uwm) - J) < 1e-12
    flux = bp * (uip1 - uwp) / (pp * dx) - bm * (uwm - ui) / (pm * dx)
    assert abs(flux - F) < 1e-9 * max(1.0, abs(F))


@pytest.mark.parametrize("trial", range(10))
def test_sw_interface_walls_reproduce_flux_continuous_linear(trial):
    """A continuous piecewise-linear profile with continuous flux is reproduced exactly."""
    bm, bp = RNG.uniform(0.1, 5, size=2)
    pm, pp = RNG.uniform(0.1, 0.9, size=2)
    dx = RNG.uniform(0.01, 0.2)
    a, s = RNG.standard_normal(2)
    t = bm * s / bp                               # slope on the plus side: bp t = bm s
    ui, uip1 = a - s * pm * dx, a + t * pp * dx   # wall at 0, x_i = -pm dx, x_{i+1} = +pp dx
    uwp, uwm = sw_interface_walls(ui, uip1, 0.0, 0.0, pm, pp, bm, bp, dx)
    assert abs(uwp - a) < 1e-12 and abs(uwm - a) < 1e-12


def _mg_problem(bc, n=64):
    if bc == W.DIRICHLET:
        g = W.Geometry(W.STAR, (0.03, 0.02, 0.55, 0.05, 5.0, 0.4), True)
        return g, W.BOX_NONE, 1.0, 1.0
    if bc == W.NEUMANN:
        return W.Geometry(W.ELLIPSE, (0.02, -0.01, 0.35, 0.25, 0.3), False), W.BOX_DIRICHLET, 1.0, 1.0
    return W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.05, 5.0, 0.0), False), W.BOX_DIRICHLET, 0.5, 1.0


@pytest.mark.parametrize("bc", [W.DIRICHLET, W.NEUMANN, W.INTERFACE])
def test_vcycle_converges_to_direct_sw_solve(bc):
    g, box, bp, bm = _mg_problem(bc)
    n = 64
    ls = LevelSet(g)
    mg = Multigrid(ls, n, bc, box, bp, bm)
    L = mg.levels[0]
    f = RNG.standard_normal(n * n)
    f[~L.unk_flat] = 0.0
    unk = np.nonzero(L.unk_flat)[0]
    A = L.A[unk][:, unk].tocsc()
    u_ref = np.zeros(n * n)
    u_ref[unk] = spla.spsolve(A, f[unk])
    u = np.zeros(n * n)
    rates = []
    r_prev = np.linalg.norm(f)
    for it in range(60):
        r = f - L.apply(u)
        r[~L.unk_flat] = 0.0
        rn = np.linalg.norm(r)
        rates.append(rn / r_prev)
        r_prev = rn
        if rn < 1e-12 * np.linalg.norm(f):
            break
        u += mg.vcycle(r)
    assert np.max(np.abs(u - u_ref)) < 1e-9 * np.max(np.abs(u_ref))
    if bc == W.DIRICHLET:
        assert np.median(rates[1:]) < 0.2


def test_level_sizes_rule():
    assert level_sizes(64, 2) == [64, 32, 16, 8]
    assert level_sizes(1024, 2) == [1024, 512, 256, 128, 64, 32, 16, 8]
    assert level_sizes(96, 2) == [96, 48, 24, 12]
    assert level_sizes(256, 3) == [256, 128, 64, 32, 16, 8, 4]


def test_fgmres_exact_preconditioner_one_iteration():
    n = 60
    A = np.eye(n) * 4 + RNG.standard_normal((n, n)) * 0.3
    b = RNG.standard_normal(n)
    Ainv = np.linalg.inv(A)
    x, info = fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, tol=1e-12)
    assert info["iters"] == 1
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)


def test_fgmres_identity_matches_dense_solve_with_restarts():
    n = 80
    A = np.diag(np.linspace(1, 10, n)) + np.triu(RNG.standard_normal((n, n)) * 0.05, 1)
    b = RNG.standard_normal(n)
    x, info = fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-12, restart=10, max_iter=2000)
    assert info["converged"] and info["iters"] > 10           # restarted at least once
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-9)


@pytest.mark.parametrize("kind", ["dirichlet4", "neumann6", "interface6"])
def test_converged_solution_equals_dense_solve(kind):
    if kind == "dirichlet4":
        spec = W.circle_dirichlet_64(32)
    elif kind == "neumann6":
        spec = W.ProblemSpec(n=40, geometry=W.Geometry(W.CIRCLE, (0.03, 0.01, 0.3), False), bc=W.NEUMANN, order=6,
                             box_bc=W.BOX_DIRICHLET, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))
    else:
        spec = W.ProblemSpec(n=40, geometry=W.Geometry(W.ELLIPSE, (0.0, 0.02, 0.35, 0.3, 0.2), False),
                             bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=0.5, beta_minus=1.0,
                             solution=W.two_phase_star_solution())
    P = OracleProblem(spec)
    f, data = P.data()
    x, info, b = P.solve(f, data, tol=1e-13)
    A, unk = assemble(P.op)
    xd = np.linalg.solve(A, b[unk])
    assert info["converged"]
    assert np.max(np.abs(x[unk] - xd)) < 1e-9 * np.max(np.abs(xd))


@pytest.mark.parametrize("which", ["dirichlet4", "interface6"])
def test_manufactured_convergence_order(which):
    if which == "dirichlet4":
        mk, ns, order = W.circle_dirichlet_64, (32, 64), 4
    else:
        mk, ns, order = W.star_interface_1024, (128, 192), 6
    errs = []
    for n in ns:
        P = OracleProblem(mk(n))
        f, data = P.data()
        x, info, _ = P.solve(f, data, tol=1e-13)
        errs.append(np.max(np.abs(x - P.exact())[P.unk_flat]))
    slope = np.log(errs[0] / errs[1]) / np.log(ns[1] / ns[0])
    assert order - 0.5 < slope < order + 1.5
