"""Parity at full size for the 3D benchmark configuration: the 256^3 exterior of the
ellipsoid (0.6, 0.45, 0.35), Neumann on it, Dirichlet box, (4,5) scheme, FP32 multigrid.

The full oracle does not fit a test at 16.7 M nodes, so the oracle evaluates the
operator one node at a time (fits built on first use) at sampled nodes: random
nodes plus nodes next to the surface, where the fits enter.
"""
import numpy as np
import pytest

import workloads as W
from oracle.operator import IIMOperator
from tests.gpu_helpers import dev, gpu_problem, need_gpu, set_gpu_data

pytestmark = pytest.mark.gpu

N = 256


@pytest.fixture(scope="module")
def setup3d():
    torch, iim = need_gpu()
    spec = W.ellipsoid_neumann_256(N)
    P = gpu_problem(iim, spec, tol=1e-10, mg_precision=iim.MG_FP32)
    f = set_gpu_data(P, spec)
    O = IIMOperator(spec, lazy=True)
    xc, nc = O.control_points()
    g, j0, j1 = W.boundary_data(spec, xc, nc)
    data = {"g": g, "j0": j0, "j1": j1, "box": W.box_data(spec)}
    rng = np.random.default_rng(9)
    phase = O.plus.ravel(order="F")
    plus_nodes = np.nonzero(phase)[0]
    # nodes within the stencil reach of a crossing (lower nodes of cut edges and their neighbours)
    near = np.unique(np.concatenate([O.cross.lo + s for s in (-2, -1, 0, 1, 2)]))
    near = near[(near >= 0) & (near < N ** 3)]
    near = near[phase[near]]
    nodes = np.concatenate([rng.choice(plus_nodes, 1500, replace=False), rng.choice(near, 1500, replace=False)])
    return torch, iim, spec, P, O, data, f, nodes


def test_3d_control_points_and_operator(setup3d):
    torch, iim, spec, P, O, data, f, nodes = setup3d
    assert P.K == O.cross.count
    xc, nc = P.control_points()
    assert np.max(np.abs(xc.cpu().numpy() - O.cross.x)) < 1e-12
    u = np.random.default_rng(2).standard_normal(P.N)
    got = P.apply(dev(u)).cpu().numpy()[nodes]
    ref = O.apply_at(u, nodes)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    b = P.rhs().cpu().numpy()[nodes]
    bref = f[nodes] - O.apply_at(np.zeros(P.N), nodes, data, include_data=True)
    assert np.max(np.abs(b - bref)) < 1e-12 * np.max(np.abs(bref))


def test_3d_solve(setup3d):
    torch, iim, spec, P, O, data, f, nodes = setup3d
    x, info = P.solve()
    assert info.converged and info.relres <= 1e-10
    xg = x.cpu().numpy()
    # residual at the sampled nodes, evaluated by the oracle, against the device's residual there
    r_dev = (P.rhs() - P.apply(x)).cpu().numpy()[nodes]
    r_orc = (f[nodes] - O.apply_at(np.zeros(P.N), nodes, data, include_data=True)) - O.apply_at(xg, nodes)
    scale = np.max(np.abs(f[nodes]))
    assert np.max(np.abs(r_dev - r_orc)) < 1e-9 * scale
    # 4th-order accuracy at h = 1/128 against the manufactured solution
    X = W.node_coords(N, 3)
    ex = W.to_flat(spec.solution.u_plus(X))
    err = np.max(np.abs(xg - ex)[O.plus.ravel(order="F")])
    assert err < 2e-6, err
