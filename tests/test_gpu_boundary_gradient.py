"""Boundary quantities and the gradient (Sec. 2.4) on the GPU against the oracle.

Tolerance 1e-11 relative to the largest value.  The fit coefficients come from two
QR implementations (LAPACK in the oracle, Householder on the device), each within its
rounding level of the exact least-squares rows (the oracle's ghost rows lie within
1.1e-13 of 40-digit rows relative to the row's size, tests/test_oracle_fits_precision.py);
unlike the Laplacian, whose diagonal term dominates, the first-derivative sums carry the
two FP64 errors undamped and with a factor 1/h (measured 4.7e-12 for the (6,7) star on a
random vector), so 1e-12 is below what two FP64 implementations can agree to here.  The inputs are a random vector and
the converged solution; the GPU's data are evaluated at its own control points,
which agree with the oracle's to a few ulps (test_gpu_parity).
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu

CASES = {
    "dir2d_circle_4_64": lambda: W.circle_dirichlet_64(64),
    "dir2d_star_6_96": lambda: W.ProblemSpec(
        n=96, geometry=W.Geometry(W.STAR, (0.03, 0.01, 0.55, 0.04, 6.0, 1.0), True), bc=W.DIRICHLET, order=6,
        solution=W.sin_cos_2d(2.5, 0.1, 1.2, 0.4)),
    "neu2d_ext_6_80": lambda: W.ProblemSpec(
        n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False), bc=W.NEUMANN, order=6,
        box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
    "iface2d_6_128": lambda: W.star_interface_1024(128),
    "dir3d_sphere_4_40": lambda: W.ProblemSpec(
        n=40, geometry=W.Geometry(W.SPHERE, (0.02, -0.01, 0.03, 0.62), True), bc=W.DIRICHLET, order=4,
        solution=W.sin_sin_cos_3d((1.0, 2.0, 1.5), (0.1, 0.2, 0.3))),
    "neu3d_ellipsoid_4_48": lambda: W.ellipsoid_neumann_256(48),
}


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("case", sorted(CASES))
def test_boundary_values_and_gradient_match_oracle(env, case):
    torch, iim = env
    spec = CASES[case]()
    P = gpu_problem(iim, spec, tol=1e-12)
    set_gpu_data(P, spec)
    O = OracleProblem(spec)
    f, data = O.data()
    u = np.random.default_rng(11).standard_normal(P.N) * O.unk_flat
    x, info = P.solve()
    assert info.converged
    for vec in (u, x.cpu().numpy()):
        g_gpu = P.gradient(dev(vec)).cpu().numpy()
        g_ora = O.op.gradient(vec, data)
        assert rel_err(g_gpu, g_ora) < 1e-11, (case, rel_err(g_gpu, g_ora))
        if spec.bc != W.INTERFACE:
            b_gpu = P.boundary_values(dev(vec)).cpu().numpy()
            b_ora = O.op.boundary_values(vec, data)
            assert b_gpu.shape == b_ora.shape
            assert rel_err(b_gpu, b_ora) < 1e-11, (case, rel_err(b_gpu, b_ora))
    if spec.bc == W.INTERFACE:
        with pytest.raises(iim.IIMError):
            P.boundary_values(x)


def test_boundary_values_of_the_solution_are_accurate(env):
    """(4,5) Dirichlet circle at n = 256: the boundary normal gradient of the GPU solution
    against the exact one (the oracle shows order-4 convergence; 1.6e-8 at n = 256)."""
    torch, iim = env
    spec = W.circle_dirichlet_64(256)
    P = gpu_problem(iim, spec, tol=1e-13)
    set_gpu_data(P, spec)
    x, info = P.solve()
    bv = P.boundary_values(x).cpu().numpy()
    xc, nc = P.control_points()
    ex = np.sum(spec.solution.grad_plus(xc.cpu().numpy()) * nc.cpu().numpy(), axis=-1)
    assert np.max(np.abs(bv - ex)) < 5e-8
