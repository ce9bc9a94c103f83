"""Re-running a problem's set-up with other geometry parameters (iim_problem_setup) gives what
creating the problem with those parameters gives: the same phase, control points, operator,
V-cycle and converged solution, bit for bit.  The cases change the number of unknowns on the
coarsest multigrid level (checked with the oracle's levels), which the dense coarse system
must follow without a new allocation."""
import numpy as np
import pytest

import workloads as W
from oracle.geometry import LevelSet
from oracle.mg import Multigrid
from tests.gpu_helpers import dev, gpu_problem, need_gpu, set_gpu_data

pytestmark = pytest.mark.gpu


def _coarse_unknowns(spec):
    mg = Multigrid(LevelSet(spec.geometry), spec.n, spec.bc, spec.box_bc, spec.beta_plus, spec.beta_minus)
    return int(mg.levels[-1].unk_flat.sum())


CASES = {
    "dirichlet_circle_4_64": (
        W.ProblemSpec(n=64, geometry=W.Geometry(W.CIRCLE, (0.01, -0.02, 0.5), True), bc=W.DIRICHLET, order=4,
                      solution=W.harmonic_exp_sin()),
        (0.01, -0.02, 0.56)),
    "neumann_ellipse_6_96": (
        W.ProblemSpec(n=96, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN,
                      order=6, box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
        (0.02, -0.03, 0.45, 0.33, 0.6)),
}


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("case", sorted(CASES))
def test_resetup_equals_fresh_create(env, case):
    torch, iim = env
    s1, p2 = CASES[case]
    s2 = W.ProblemSpec(n=s1.n, geometry=W.Geometry(s1.geometry.kind, p2, s1.geometry.plus_inside), bc=s1.bc,
                       order=s1.order, box_bc=s1.box_bc, beta_plus=s1.beta_plus, beta_minus=s1.beta_minus,
                       solution=s1.solution)
    assert _coarse_unknowns(s1) != _coarse_unknowns(s2)
    P = gpu_problem(iim, s1)
    P.setup(p2)
    P.refresh_sizes()
    Q = gpu_problem(iim, s2)
    assert P.K == Q.K
    assert torch.equal(P.phase(), Q.phase())
    xp, npp = P.control_points()
    xq, nq = Q.control_points()
    assert torch.equal(xp, xq) and torch.equal(npp, nq)
    rng = np.random.default_rng(9)
    u = dev(rng.standard_normal(P.N))
    assert torch.equal(P.apply(u), Q.apply(u))
    v = dev(rng.standard_normal(P.N) * Q.phase().cpu().numpy())
    assert torch.equal(P.precondition(v), Q.precondition(v))
    set_gpu_data(P, s2)
    set_gpu_data(Q, s2)
    xa, ia = P.solve()
    xb, ib = Q.solve()
    assert ia.converged and ib.converged and ia.iters == ib.iters
    assert torch.equal(xa, xb)
