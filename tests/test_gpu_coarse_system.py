"""The dense coarse solve at its three working modes: one V-cycle against the oracle.

The coarsest Shortley-Weller system is factored by one CTA: with the matrix and its inverse
in shared memory when both fit the shared memory sized at creation (up to 200 KB), with the
matrix alone there and the inverse built in global memory when only the matrix fits, and
entirely in global memory otherwise.  The first mode is what most problems use (every other
parity test); these cases have coarsest levels of 196 and 225 nodes (n = 112 = 7 x 16 and
n = 120 = 15 x 8), so that in FP64 and FP32 the other two modes run.  Tolerances are those
of the parity tests: one FP64 V-cycle 1e-12 relative, one FP32 V-cycle 1e-5 relative,
converged solutions 1e-9.
"""
import numpy as np
import pytest

import workloads as W
from oracle.geometry import LevelSet
from oracle.mg import Multigrid
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu

CASES = {
    # exterior of a small circle with a Dirichlet box: 225 coarse nodes, most of them unknowns
    "circle_exterior_neumann_4_120": lambda: W.ProblemSpec(
        n=120, geometry=W.Geometry(W.CIRCLE, (0.02, -0.01, 0.3), False), bc=W.NEUMANN, order=4,
        box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
    # interface: every one of the 225 coarse nodes is an unknown
    "star_interface_6_120": lambda: W.ProblemSpec(
        n=120, geometry=W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.1, 5.0, 0.2), False), bc=W.INTERFACE, order=6,
        box_bc=W.BOX_DIRICHLET, beta_plus=1.0, beta_minus=2.0, solution=W.two_phase_star_solution()),
    # interface on 14^2 coarse nodes
    "star_interface_4_112": lambda: W.ProblemSpec(
        n=112, geometry=W.Geometry(W.STAR, (0.01, 0.02, 0.5, 0.08, 5.0, 0.0), False), bc=W.INTERFACE, order=4,
        box_bc=W.BOX_DIRICHLET, beta_plus=0.5, beta_minus=1.0, solution=W.two_phase_star_solution()),
}


def _lu_mode(nu, aug, cn, elem_bytes):
    """The working mode the LU takes (2: matrix and inverse in shared memory, 1: the matrix,
    0: neither), from the shared memory the creation sizes for nu unknowns."""
    nb = min(cn, nu + nu // 4 + 8 + aug)
    smem_elems = min(2 * nb * nb * elem_bytes, 200 * 1024) // elem_bytes
    n = nu + aug
    return 2 if 2 * n * n <= smem_elems else (1 if n * n <= smem_elems else 0)


def _coarse(spec):
    mg = Multigrid(LevelSet(spec.geometry), spec.n, spec.bc, spec.box_bc, spec.beta_plus, spec.beta_minus)
    lv = mg.levels[-1]
    return int(lv.unk_flat.sum()), int(lv.unk_flat.size)


@pytest.fixture(scope="module")
def env():
    return need_gpu()


def test_the_cases_reach_the_other_modes():
    modes = set()
    for name in CASES:
        spec = CASES[name]()
        nu, nodes = _coarse(spec)
        for esz in (8, 4):
            modes.add(_lu_mode(nu, 0, nodes, esz))
    assert modes >= {0, 1}, modes


@pytest.mark.parametrize("name", sorted(CASES))
def test_vcycle_fp64_and_fp32(env, name):
    torch, iim = env
    spec = CASES[name]()
    O = OracleProblem(spec)
    v = np.random.default_rng(11).standard_normal(O.unk_flat.size) * O.unk_flat
    z_ref = O.precondition(v)
    P64 = gpu_problem(iim, spec, mg_precision=iim.MG_FP64)
    assert rel_err(P64.precondition(dev(v)).cpu().numpy(), z_ref) < 1e-12
    P32 = gpu_problem(iim, spec, mg_precision=iim.MG_FP32)
    assert rel_err(P32.precondition(dev(v)).cpu().numpy(), z_ref) < 1e-5


def test_converged_solution_global_mode(env):
    torch, iim = env
    spec = CASES["circle_exterior_neumann_4_120"]()
    P = gpu_problem(iim, spec, mg_precision=iim.MG_FP64)
    set_gpu_data(P, spec)
    x, info = P.solve()
    assert info.converged and info.relres < 1e-10
    O = OracleProblem(spec)
    f, data = O.data()
    xo, oinfo, _ = O.solve(f, data, tol=1e-13)
    assert rel_err(x.cpu().numpy(), xo) < 1e-9
