"""Oracle pins for the W-cycle (Sec. 3.3 results) and left-preconditioned GMRES (Sec. 3.2).

* on a two-level hierarchy the coarse solve is exact, so the W-cycle equals the V-cycle;
* as a solver on the Shortley-Weller system, the W-cycle converges faster than the
  V-cycle for Neumann and interface problems (2D and 3D) and its rate hardly changes
  with n (2D);
* left GMRES with the identity preconditioner is plain GMRES: after k iterations it
  equals right-preconditioned FGMRES with the identity (same minimisation problem);
  with the exact inverse as preconditioner it converges in one iteration; converged,
  it matches a dense solve;
* with a diagonal (Jacobi) preconditioner M, k iterations of left GMRES give the
  minimiser of |M (b - A x)| over the Krylov space span{Mb, (MA) Mb, ...} (brute force
  by least squares); right preconditioning would minimise |b - A x| instead.
* with one V-cycle as the preconditioner, the iteration counts of both Krylov methods
  stay nearly constant from n = 64 to 256 (Sec. 3.3).
"""
import numpy as np
import pytest

import workloads as W
from oracle.dense import assemble
from oracle.fgmres import fgmres, gmres_left
from oracle.geometry import LevelSet
from oracle.mg import Multigrid
from oracle.problem import OracleProblem


def _rate(mg, n, iters=8, seed=0):
    L0 = mg.levels[0]
    f = np.random.default_rng(seed).standard_normal(n * n)
    f[~L0.unk_flat] = 0.0
    u = np.zeros_like(f)
    rs = []
    for _ in range(iters):
        r = f - L0.apply(u)
        r[~L0.unk_flat] = 0.0
        rs.append(np.linalg.norm(r))
        u = u + mg.vcycle(r)
    r = f - L0.apply(u)
    rs.append(np.linalg.norm(r[L0.unk_flat]))
    return (rs[-1] / rs[3]) ** (1.0 / (iters - 3))


def test_w_cycle_equals_v_cycle_on_two_levels():
    geom = W.Geometry(W.CIRCLE, (0.013, -0.021, 0.52), True)
    ls = LevelSet(geom)
    mv = Multigrid(ls, 16, W.DIRICHLET, W.BOX_NONE, 1.0, 1.0, 2, 2, 1)
    mw = Multigrid(ls, 16, W.DIRICHLET, W.BOX_NONE, 1.0, 1.0, 2, 2, 2)
    assert len(mv.levels) == 2
    f = np.random.default_rng(1).standard_normal(256)
    f[~mv.levels[0].unk_flat] = 0.0
    assert np.max(np.abs(mv.vcycle(f) - mw.vcycle(f))) < 1e-12 * np.max(np.abs(mv.vcycle(f)))


@pytest.mark.parametrize("case", ["neumann", "interface"])
def test_w_cycle_faster_and_resolution_independent(case):
    if case == "neumann":
        geom, bc, box = W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), W.NEUMANN, W.BOX_DIRICHLET
    else:
        geom, bc, box = W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.1, 5.0, 0.0), False), W.INTERFACE, W.BOX_DIRICHLET
    ls = LevelSet(geom)
    rates = {}
    for n in (64, 128):
        for gamma in (1, 2):
            rates[(n, gamma)] = _rate(Multigrid(ls, n, bc, box, 1.0, 1.0, 2, 2, gamma), n)
    assert rates[(128, 2)] < rates[(128, 1)], rates
    assert rates[(128, 2)] < 1.2 * rates[(64, 2)], rates
    assert rates[(128, 2)] < 0.2, rates


def test_left_gmres_with_identity_is_plain_gmres():
    spec = W.circle_dirichlet_64(24)
    P = OracleProblem(spec)
    f, data = P.data()
    b = P.op.rhs(f, data)
    ident = lambda v: v.copy()
    k = 12
    xr, _ = fgmres(P.op.apply, ident, b, tol=1e-30, restart=k, max_iter=k)
    xl, _ = gmres_left(P.op.apply, ident, b, tol=1e-30, restart=k, max_iter=k)
    assert np.max(np.abs(xr - xl)) < 1e-9 * np.max(np.abs(xr))


def test_left_gmres_exact_preconditioner_and_dense_solution():
    spec = W.circle_dirichlet_64(24)
    P = OracleProblem(spec)
    f, data = P.data()
    b = P.op.rhs(f, data)
    A, unk = assemble(P.op)
    Ainv = np.linalg.inv(A)

    def exact(v):
        z = np.zeros_like(v)
        z[unk] = Ainv @ v[unk]
        return z

    x1, i1 = gmres_left(P.op.apply, exact, b, tol=1e-12, restart=10, max_iter=10)
    assert i1["converged"] and i1["iters"] == 1
    xd = np.zeros_like(b)
    xd[unk] = np.linalg.solve(A, b[unk])
    xl, il, _ = P.solve_left(f, data, tol=1e-13)
    assert il["converged"]
    assert np.max(np.abs(xl - xd)) < 1e-9 * np.max(np.abs(xd))


def test_left_gmres_minimises_the_preconditioned_residual():
    spec = W.circle_dirichlet_64(20)
    P = OracleProblem(spec)
    f, data = P.data()
    b = P.op.rhs(f, data)
    A, unk = assemble(P.op)
    d = np.random.default_rng(4).uniform(0.2, 3.0, unk.size) / np.abs(np.diag(A))
    Dfull = np.zeros(b.size)
    Dfull[unk] = d
    jac = lambda v: Dfull * v
    k = 5
    xl, info = gmres_left(P.op.apply, jac, b, tol=1e-30, restart=k, max_iter=k)
    assert info["iters"] == k
    MA = d[:, None] * A
    K = [d * b[unk]]
    for _ in range(k - 1):
        K.append(MA @ K[-1])
    Q, _ = np.linalg.qr(np.array(K).T)
    y = np.linalg.lstsq(MA @ Q, d * b[unk], rcond=None)[0]
    x_ref = Q @ y
    assert np.max(np.abs(xl[unk] - x_ref)) < 1e-8 * np.max(np.abs(x_ref))
    y_right = np.linalg.lstsq(A @ Q, b[unk], rcond=None)[0]
    assert np.max(np.abs(Q @ y_right - x_ref)) > 1e-4 * np.max(np.abs(x_ref))


def test_left_gmres_pure_neumann_augmented_matches_fgmres():
    """The augmented system of Sec. 2.3 is nonsingular: left GMRES and FGMRES converge to
    the same (u, alpha)."""
    spec = W.ProblemSpec(n=40, geometry=W.Geometry(W.ELLIPSE, (0.01, -0.02, 0.6, 0.45, 0.3), True),
                         bc=W.NEUMANN, order=4, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))
    P = OracleProblem(spec)
    assert P.singular
    f, data = P.data()
    xr, ir, _ = P.solve(f, data, tol=1e-13)
    xl, il, _ = P.solve_left(f, data, tol=1e-13)
    assert ir["converged"] and il["converged"]
    assert np.max(np.abs(xl - xr)) < 1e-9 * np.max(np.abs(xr))
    assert abs(il["alpha"] - ir["alpha"]) < 1e-9 * max(abs(ir["alpha"]), 1e-300) + 1e-12


@pytest.mark.parametrize("case", ["dirichlet_circle", "neumann_exterior"])
def test_iterations_nearly_independent_of_resolution(case):
    """Sec. 3.3: with one multigrid cycle as the preconditioner the iteration count varies
    only weakly with the resolution (measured: circle 18, 18, 20 right / 17, 18, 19 left;
    Neumann exterior 24, 24, 24 / 24, 26, 26 at n = 64, 128, 256)."""
    def spec(n):
        if case == "dirichlet_circle":
            return W.circle_dirichlet_64(n)
        return W.ProblemSpec(n=n, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False),
                             bc=W.NEUMANN, order=4, box_bc=W.BOX_DIRICHLET, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))
    right, left = [], []
    for n in (64, 128, 256):
        P = OracleProblem(spec(n))
        f, data = P.data()
        _, ir, _ = P.solve(f, data, tol=1e-10)
        _, il, _ = P.solve_left(f, data, tol=1e-10)
        assert ir["converged"] and il["converged"]
        right.append(ir["iters"])
        left.append(il["iters"])
    assert max(right) - min(right) <= 3, right
    assert max(left) - min(left) <= 3, left
    assert max(right) <= 30 and max(left) <= 30, (right, left)


def _rate3(mg, n, iters=8, seed=0):
    L0 = mg.levels[0]
    f = np.random.default_rng(seed).standard_normal(n ** 3)
    f[~L0.unk_flat] = 0.0
    u = np.zeros_like(f)
    rs = []
    for _ in range(iters):
        r = f - L0.apply(u)
        r[~L0.unk_flat] = 0.0
        rs.append(np.linalg.norm(r))
        u = u + mg.vcycle(r)
    r = f - L0.apply(u)
    rs.append(np.linalg.norm(r[L0.unk_flat]))
    return (rs[-1] / rs[3]) ** (1.0 / (iters - 3))


@pytest.mark.parametrize("case", ["interface_sphere", "neumann_ellipsoid"])
def test_w_cycle_faster_in_3d(case):
    """3D counterpart (measured: interface sphere V 0.132 / 0.139, W 0.089 / 0.080; Neumann
    ellipsoid V 0.194 / 0.198, W 0.177 / 0.176 at n = 24 / 48)."""
    if case == "interface_sphere":
        geom, bc = W.Geometry(W.SPHERE, (0.0, 0.0, 0.0, 0.45), False), W.INTERFACE
    else:
        geom, bc = W.Geometry(W.ELLIPSOID, (0.0, 0.0, 0.0, 0.6, 0.45, 0.35), False), W.NEUMANN
    ls = LevelSet(geom)
    n = 24
    v = _rate3(Multigrid(ls, n, bc, W.BOX_DIRICHLET, 1.0, 1.0, 2, 2, 1), n)
    w = _rate3(Multigrid(ls, n, bc, W.BOX_DIRICHLET, 1.0, 1.0, 2, 2, 2), n)
    assert w < 0.95 * v and w < 0.2, (v, w)
