"""GPU vs oracle, element by element, through the C ABI.

Tolerances (derived from FP64 arithmetic; the method's own sizes): control points
and normals 1e-12 absolute (roots of phi agree to a few ulps of h); phase bytes
bit-exact; the IIM operator and its data term 1e-12 relative to max|L u| (sums of
<= 13 stencil terms and <= 4 fits of ~100 terms, with coefficients ~1/h^2);
one FP64 V-cycle 1e-12 relative (identical arithmetic, other summation order);
one FP32 V-cycle 1e-5 relative (single precision, cond ~ n^2 on the coarse grids).
Sizes span several thread blocks and ragged tails (n not a multiple of 32).
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu

CASES = {
    "circle_dirichlet_64": lambda: W.circle_dirichlet_64(64),
    "circle_dirichlet_ragged_72": lambda: W.ProblemSpec(
        n=72, geometry=W.Geometry(W.CIRCLE, (0.013, -0.021, 0.52), True), bc=W.DIRICHLET, order=4,
        solution=W.harmonic_exp_sin()),
    "star_interface_6_128": lambda: W.star_interface_1024(128),
    "star_interface_contrast_4_112": lambda: W.ProblemSpec(
        n=112, geometry=W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.1, 5.0, 0.4), False), bc=W.INTERFACE, order=4,
        box_bc=W.BOX_DIRICHLET, beta_plus=0.5, beta_minus=1.0, solution=W.two_phase_star_solution()),
    "neumann_ext_6_80": lambda: W.ProblemSpec(
        n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN, order=6,
        box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
    "dirichlet_star_6_96": lambda: W.ProblemSpec(
        n=96, geometry=W.Geometry(W.STAR, (0.03, 0.01, 0.55, 0.04, 6.0, 1.0), True), bc=W.DIRICHLET, order=6,
        solution=W.sin_cos_2d(2.5, 0.1, 1.2, 0.4)),
    "ellipsoid_neumann_48": lambda: W.ellipsoid_neumann_256(48),
    "sphere_dirichlet_40": lambda: W.ProblemSpec(
        n=40, geometry=W.Geometry(W.SPHERE, (0.02, -0.01, 0.03, 0.62), True), bc=W.DIRICHLET, order=4,
        solution=W.sin_sin_cos_3d((1.0, 2.0, 1.5), (0.1, 0.2, 0.3))),
}


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request, env):
    torch, iim = env
    spec = CASES[request.param]()
    P = gpu_problem(iim, spec, mg_precision=iim.MG_FP64)
    O = OracleProblem(spec)
    return spec, P, O


def test_phase_bit_exact(pair):
    spec, P, O = pair
    assert np.array_equal(P.phase().cpu().numpy().astype(bool), O.plus_flat)


def test_control_points(pair):
    spec, P, O = pair
    assert P.K == O.op.cross.count
    xc, nc = P.control_points()
    assert np.max(np.abs(xc.cpu().numpy() - O.op.cross.x)) < 1e-12
    assert np.max(np.abs(nc.cpu().numpy() - O.op.cross.normal)) < 1e-12


def test_operator_random_input(pair):
    spec, P, O = pair
    u = np.random.default_rng(5).standard_normal(P.N)
    assert rel_err(P.apply(dev(u)).cpu().numpy(), O.op.apply(u)) < 1e-12


def test_operator_smooth_input_with_data(pair):
    spec, P, O = pair
    set_gpu_data(P, spec)
    f, data = O.data()
    u = O.exact()
    got = P.apply(dev(u), include_data=True).cpu().numpy()
    ref = O.op.apply(u, data, include_data=True)
    # L u + L_Gamma u_Gamma cancels down to the truncation error: measure the
    # difference against the size of the terms that are summed
    scale = np.max(np.abs(O.op.apply(u)))
    assert np.max(np.abs(got - ref)) < 1e-12 * scale


def test_rhs_data_term(pair):
    spec, P, O = pair
    set_gpu_data(P, spec)
    f, data = O.data()
    assert rel_err(P.rhs().cpu().numpy(), O.op.rhs(f, data)) < 1e-12


def test_vcycle_fp64(pair):
    spec, P, O = pair
    v = np.random.default_rng(7).standard_normal(P.N) * O.unk_flat
    assert rel_err(P.precondition(dev(v)).cpu().numpy(), O.precondition(v)) < 1e-12


def test_vcycle_fp32(env):
    torch, iim = env
    spec = CASES["star_interface_contrast_4_112"]()
    P = gpu_problem(iim, spec, mg_precision=iim.MG_FP32)
    O = OracleProblem(spec)
    v = np.random.default_rng(8).standard_normal(P.N)
    assert rel_err(P.precondition(dev(v)).cpu().numpy(), O.precondition(v)) < 1e-5


@pytest.mark.parametrize("nu", [(3, 3), (1, 2)])
@pytest.mark.parametrize("case", ["star_interface_6_128", "neumann_ext_6_80"])
def test_vcycle_fp64_other_sweep_counts(env, case, nu):
    """nu1 = nu2 = 2 runs two fused tile kernels per level; other sweep counts run the
    separate kernels (3, 3: with the plain-sweep kernel; 1, 2: the generic path)."""
    torch, iim = env
    spec = CASES[case]()
    P = gpu_problem(iim, spec, mg_precision=iim.MG_FP64, nu1=nu[0], nu2=nu[1])
    O = OracleProblem(spec, nu1=nu[0], nu2=nu[1])
    v = np.random.default_rng(9).standard_normal(P.N) * O.unk_flat
    assert rel_err(P.precondition(dev(v)).cpu().numpy(), O.precondition(v)) < 1e-12
