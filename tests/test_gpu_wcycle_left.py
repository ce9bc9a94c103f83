"""W-cycle and left-preconditioned GMRES (Sec. 3.2, Sec. 3.3 results) on the GPU against
the oracle.

* one FP64 W-cycle, 1e-12 relative (the V-cycle's bound: identical arithmetic in
  another summation order), on every path the cycle takes: fused tile kernels (the
  second visit of a level reads its previous result with a halo of 5), the separate
  2D kernels (nu = 3, 3), the generic path (nu = 1, 2 and 3D), the single-CTA tail
  alone, and the augmented coarse solve of a pure Neumann problem;
* FGMRES with the W-cycle and left GMRES (V and W) against the oracle's solves: the
  same iteration counts within one, and the same solution;
* the batched engine refuses both (they run through the single-problem solve).
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu


def _pure_neumann(n):
    return W.ProblemSpec(n=n, geometry=W.Geometry(W.ELLIPSE, (0.01, -0.02, 0.6, 0.45, 0.3), True), bc=W.NEUMANN,
                         order=4, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))


CASES = {
    "circle_dirichlet_128": (lambda: W.circle_dirichlet_64(128), (2, 2)),
    "circle_dirichlet_ragged_72": (lambda: W.ProblemSpec(
        n=72, geometry=W.Geometry(W.CIRCLE, (0.013, -0.021, 0.52), True), bc=W.DIRICHLET, order=4,
        solution=W.harmonic_exp_sin()), (2, 2)),
    "star_interface_6_128": (lambda: W.star_interface_1024(128), (2, 2)),
    "neumann_ext_6_80_nu33": (lambda: W.ProblemSpec(
        n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN, order=6,
        box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)), (3, 3)),
    "neumann_ext_6_80_nu12": (lambda: W.ProblemSpec(
        n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN, order=6,
        box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)), (1, 2)),
    "sphere_dirichlet_40": (lambda: W.ProblemSpec(
        n=40, geometry=W.Geometry(W.SPHERE, (0.02, -0.01, 0.03, 0.62), True), bc=W.DIRICHLET, order=4,
        solution=W.sin_sin_cos_3d((1.0, 2.0, 1.5), (0.1, 0.2, 0.3))), (2, 2)),
    "tail_only_circle_32": (lambda: W.circle_dirichlet_64(32), (2, 2)),
    "pure_neumann_72": (lambda: _pure_neumann(72), (2, 2)),
}


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("case", sorted(CASES))
def test_wcycle_fp64_matches_oracle(env, case):
    torch, iim = env
    make, nu = CASES[case]
    spec = make()
    P = gpu_problem(iim, spec, mg_precision=iim.MG_FP64, nu1=nu[0], nu2=nu[1], cycle=2)
    O = OracleProblem(spec, nu1=nu[0], nu2=nu[1], cycle=2)
    v = np.random.default_rng(13).standard_normal(P.N) * O.unk_flat
    got = P.precondition(dev(v)).cpu().numpy()
    assert rel_err(got, O.precondition(v)) < 1e-12, (case, rel_err(got, O.precondition(v)))
    # and it is not the V-cycle
    assert rel_err(got, OracleProblem(spec, nu1=nu[0], nu2=nu[1]).precondition(v)) > 1e-6


def test_wcycle_fp32_matches_oracle(env):
    torch, iim = env
    spec = W.star_interface_1024(128)
    P = gpu_problem(iim, spec, cycle=2)
    O = OracleProblem(spec, cycle=2)
    v = np.random.default_rng(14).standard_normal(P.N) * O.unk_flat
    assert rel_err(P.precondition(dev(v)).cpu().numpy(), O.precondition(v)) < 1e-5


def _solve_pair(iim, spec, krylov, cycle, tol, mg=None):
    opts = dict(tol=tol, cycle=cycle, krylov=krylov, max_iter=400)
    if mg is not None:
        opts["mg_precision"] = mg
    P = gpu_problem(iim, spec, **opts)
    set_gpu_data(P, spec)
    x, info = P.solve()
    O = OracleProblem(spec, cycle=cycle)
    f, data = O.data()
    if krylov == iim.KRYLOV_GMRES_LEFT:
        xo, oinfo, _ = O.solve_left(f, data, tol=tol)
    else:
        xo, oinfo, _ = O.solve(f, data, tol=tol)
    return P, x.cpu().numpy(), info, O, xo, oinfo


@pytest.mark.parametrize("case,krylov,cycle", [
    ("circle_dirichlet_128", 1, 1),
    ("star_interface_6_128", 1, 1),
    ("star_interface_6_128", 1, 2),
    ("star_interface_6_128", 0, 2),
    ("pure_neumann_72", 1, 1),
    ("sphere_dirichlet_40", 1, 2),
])
def test_solves_match_oracle(env, case, krylov, cycle):
    """FP64 multigrid: the preconditioners agree to 1e-12, so the Krylov iterations do too
    (iteration counts within one) and the converged solutions agree to the tolerance's
    reach: tol 1e-12 of a residual measured through cond(L) ~ n^2 leaves about 1e-8."""
    torch, iim = env
    spec = CASES[case][0]()
    P, x, info, O, xo, oinfo = _solve_pair(iim, spec, krylov, cycle, 1e-12, iim.MG_FP64)
    assert info.converged and oinfo["converged"], (info.as_dict(), oinfo["iters"])
    assert abs(info.iters - oinfo["iters"]) <= 1, (info.iters, oinfo["iters"])
    assert info.relres <= 1e-12
    if O.singular:
        unk = O.unk_flat
        x = x - np.where(unk, x[unk].mean(), 0)
        xo = xo - np.where(unk, xo[unk].mean(), 0)
    assert rel_err(x, xo) < 1e-8, rel_err(x, xo)


def test_left_gmres_fp32_multigrid_default_tolerance(env):
    """The FP32 preconditioner (the default) with left GMRES: converged to 1e-10 in the
    preconditioned norm, and as close to the exact solution as the FGMRES solution (both
    reach the same discrete solution; the tolerances leave far less than the
    discretisation error)."""
    torch, iim = env
    spec = W.star_interface_1024(256)
    errs = {}
    for krylov in (iim.KRYLOV_FGMRES, iim.KRYLOV_GMRES_LEFT):
        P = gpu_problem(iim, spec, krylov=krylov)
        set_gpu_data(P, spec)
        x, info = P.solve()
        assert info.converged and info.relres <= 1e-10
        ph = P.phase().cpu().numpy().astype(bool)
        X = W.node_coords(spec.n, spec.dim)
        ex = np.where(ph, W.to_flat(spec.solution.u_plus(X)), W.to_flat(spec.solution.u_minus(X)))
        errs[krylov] = np.max(np.abs(x.cpu().numpy() - ex))
    assert errs[iim.KRYLOV_GMRES_LEFT] < 1.05 * errs[iim.KRYLOV_FGMRES] + 1e-10, errs


def test_engine_refuses_w_cycle_and_left_gmres(env):
    torch, iim = env
    eng = iim.Engine(iim.default_options(), 2)
    for kw in ({"cycle": 2}, {"krylov": iim.KRYLOV_GMRES_LEFT}):
        P = gpu_problem(iim, W.circle_dirichlet_64(64), **kw)
        set_gpu_data(P, W.circle_dirichlet_64(64))
        with pytest.raises(iim.IIMError):
            eng.admit(P)
    eng.close()
