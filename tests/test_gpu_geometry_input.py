"""Geometry given as a level set on the grid or as a parametric (polar Fourier) curve:
GPU against the oracle through the C ABI, with the tolerances of the parity tests (phase
bit-exact; control points and normals 1e-12; the operator on the manufactured solution and
one FP64 V-cycle 1e-12 relative, the operator on random input 3e-12 (see test_operator);
converged solutions 1e-9).  Also the query calls of the boundary: the grid edge
of every control point and the outer-box sample points, and replacing a grid level set.
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu


def _blob2(n, inside=True):
    return W.sampled_levelset(W.blob_field((0.03, -0.02), 0.5, 0.05, 3.0), n, 2, plus_inside=not inside)


CASES = {
    # Omega+ inside the blob, Dirichlet, (4,5), ragged n
    "grid_blob_dirichlet_4_88": lambda: W.ProblemSpec(
        n=88, geometry=_blob2(88), bc=W.DIRICHLET, order=4, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
    # two-phase interface around the blob, (6,7), contrast 2
    "grid_blob_interface_6_96": lambda: W.ProblemSpec(
        n=96, geometry=_blob2(96, inside=False), bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET,
        beta_plus=1.0, beta_minus=2.0, solution=W.two_phase_star_solution()),
    # 3D: Neumann outside the blob, Dirichlet box, (4,5)
    "grid_blob3_neumann_4_40": lambda: W.ProblemSpec(
        n=40, geometry=W.sampled_levelset(W.blob_field((0.02, 0.0, -0.03), 0.55, 0.04, 2.5), 40, 3,
                                          plus_inside=True),
        bc=W.NEUMANN, order=4, box_bc=W.BOX_DIRICHLET, solution=W.sin_sin_cos_3d((1.0, 2.0, 1.5), (0.1, 0.2, 0.3))),
    # three-mode Fourier curve, interface (6,7)
    "fourier_interface_6_128": lambda: W.ProblemSpec(
        n=128, geometry=W.Geometry(W.FOURIER, (0.01, -0.02), False,
                                   coef=(0.5, 0.03, -0.02, 0.0, 0.025, 0.01, 0.0, 0.0, 0.008)),
        bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=0.5, beta_minus=1.0,
        solution=W.two_phase_star_solution()),
    # Fourier curve, exterior Neumann, (4,5)
    "fourier_neumann_4_96": lambda: W.ProblemSpec(
        n=96, geometry=W.Geometry(W.FOURIER, (0.0, 0.03), False, coef=(0.45, 0.0, 0.0, 0.02, -0.015)),
        bc=W.NEUMANN, order=4, box_bc=W.BOX_DIRICHLET, beta_plus=2.0, solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7)),
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


def test_control_points_and_edges(pair):
    spec, P, O = pair
    cr = O.op.cross
    assert P.K == cr.count
    xc, nc = P.control_points()
    assert np.max(np.abs(xc.cpu().numpy() - cr.x)) < 1e-12
    assert np.max(np.abs(nc.cpu().numpy() - cr.normal)) < 1e-12
    ax, lo, side = P.control_point_edges()
    assert np.array_equal(ax.cpu().numpy(), cr.axis)
    assert np.array_equal(lo.cpu().numpy(), cr.lo)
    assert np.array_equal(side.cpu().numpy().astype(bool), cr.lo_plus)


def test_operator(pair):
    """The manufactured solution with data at 1e-12 of the terms summed (as the operator
    parity tests).  Random input excites the ghost values, whose least-squares rows each
    FP64 implementation computes only to their rounding level (the oracle's are within
    1.1e-13 of 40-digit rows relative to the row's size, tests/test_oracle_fits_precision.py,
    and its operator within 5.6e-13 of the 40-digit one on the Fourier interface case at
    n = 128); two such results can differ by the sum of their errors, 1.4e-12 measured
    here, so random input is held to 3e-12."""
    spec, P, O = pair
    u = np.random.default_rng(5).standard_normal(P.N)
    assert rel_err(P.apply(dev(u)).cpu().numpy(), O.op.apply(u)) < 3e-12
    set_gpu_data(P, spec)
    f, data = O.data()
    ue = O.exact()
    got = P.apply(dev(ue), include_data=True).cpu().numpy()
    ref = O.op.apply(ue, data, include_data=True)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(O.op.apply(ue)))


def test_vcycle_fp64(pair):
    spec, P, O = pair
    v = np.random.default_rng(7).standard_normal(P.N) * O.unk_flat
    assert rel_err(P.precondition(dev(v)).cpu().numpy(), O.precondition(v)) < 1e-12


@pytest.mark.parametrize("name", ["grid_blob_interface_6_96", "fourier_neumann_4_96"])
def test_converged_solution(env, name):
    torch, iim = env
    spec = CASES[name]()
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    x, info = P.solve()
    assert info.converged and info.relres < 1e-10
    O = OracleProblem(spec)
    f, data = O.data()
    xo, oinfo, _ = O.solve(f, data, tol=1e-13)
    assert rel_err(x.cpu().numpy(), xo) < 1e-9
    # and it solves the manufactured problem to the scheme's accuracy
    assert np.max(np.abs(x.cpu().numpy() - O.exact())[O.unk_flat]) < 1e-4


def test_grid_star_matches_the_analytic_star(env):
    """The star sampled at the nodes: control points within the interpolation error of the
    analytic star's (about 1e-9 at n = 256), and the same operator to a few digits fewer."""
    torch, iim = env
    n = 256
    star = W.star_interface_1024(n)
    grid = W.ProblemSpec(n=n, geometry=W.sampled_levelset(W.star_field(0.0, 0.0, 0.5, 0.1, 5.0, 0.0), n, 2,
                                                          plus_inside=True),
                         bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET, solution=star.solution)
    A, B = gpu_problem(iim, grid), gpu_problem(iim, star)
    assert np.array_equal(A.phase().cpu().numpy(), B.phase().cpu().numpy())
    xa, na = A.control_points()
    xb, nb = B.control_points()
    assert np.max(np.abs(xa.cpu().numpy() - xb.cpu().numpy())) < 5e-9
    assert np.max(np.abs(na.cpu().numpy() - nb.cpu().numpy())) < 1e-6
    set_gpu_data(A, grid)
    set_gpu_data(B, star)
    xsa, ia = A.solve()
    xsb, ib = B.solve()
    assert ia.converged and ib.converged
    assert rel_err(xsa.cpu().numpy(), xsb.cpu().numpy()) < 1e-6


def test_set_phi_equals_a_fresh_problem(env):
    torch, iim = env
    n = 96
    s1 = W.ProblemSpec(n=n, geometry=_blob2(n, inside=False), bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET,
                       solution=W.two_phase_star_solution())
    g2 = W.sampled_levelset(W.blob_field((-0.04, 0.03), 0.48, 0.05, 3.0), n, 2, plus_inside=True)
    s2 = W.ProblemSpec(n=n, geometry=g2, bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET,
                       solution=W.two_phase_star_solution())
    P = gpu_problem(iim, s1)
    P.set_phi(dev(W.to_flat(g2.values)))
    P.setup()
    P.refresh_sizes()
    Q = gpu_problem(iim, s2)
    assert P.K == Q.K
    assert np.array_equal(P.phase().cpu().numpy(), Q.phase().cpu().numpy())
    xp, npp = P.control_points()
    xq, nq = Q.control_points()
    assert torch.equal(xp, xq) and torch.equal(npp, nq)
    u = dev(np.random.default_rng(3).standard_normal(n * n))
    assert torch.equal(P.apply(u), Q.apply(u))


@pytest.mark.parametrize("n,dim", [(64, 2), (72, 2), (24, 3)])
def test_box_points(env, n, dim):
    torch, iim = env
    if dim == 2:
        geom = W.Geometry(W.CIRCLE, (0.0, 0.0, 0.4), False)
    else:
        geom = W.Geometry(W.SPHERE, (0.0, 0.0, 0.0, 0.4), False)
    spec = W.ProblemSpec(n=n, geometry=geom, bc=W.NEUMANN, order=4, box_bc=W.BOX_DIRICHLET)
    P = gpu_problem(iim, spec)
    xb = P.box_points().cpu().numpy()
    ref = W.box_face_points(n, dim)
    assert xb.shape == ref.shape == (2 * dim * n ** (dim - 1), dim)
    assert np.max(np.abs(xb - ref)) < 1e-15


def test_server_refuses_a_grid_level_set(env):
    torch, iim = env
    import ctypes
    lib = iim.load()
    spec = CASES["grid_blob_dirichlet_4_88"]()
    d = iim.desc_from_spec(spec)
    srv = ctypes.c_void_p()
    o = iim.default_options()
    assert lib.iim_server_create(ctypes.byref(o), 1 << 30, 4, 4, 1, ctypes.byref(srv)) == 0
    rid = ctypes.c_int64()
    st = lib.iim_server_submit(srv, ctypes.byref(d), ctypes.byref(rid))
    lib.iim_server_destroy(srv)
    assert st == iim.IIM_ERR_INVALID_ARG
