"""Oracle pins for the IIM operator (Sec. 2).

* exactness: the ghost values come from least-squares polynomials that
  reproduce degree-q data exactly, and the centred stencils are exact to
  degree n+1, so L u + L_Gamma u_Gamma = beta lap(P) at every unknown node for
  any polynomial P of degree <= q (piecewise for interfaces);
* L 1 = 0 for a pure Neumann problem (Sec. 2.3);
* truncation error of order k-2 at the affected points (Sec. 2.4, Fig. 2);
* the closed form of the interface values (Eqs. 10-11) against a direct
  solve of the discrete jump system (Eq. 9);
* the spectrum bounds of Sec. 2.5.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle.dense import assemble
from oracle.operator import IIMOperator
from oracle.problem import OracleProblem
from oracle.stencils import sigma_max


def _exactness_error(spec, deg, seed=1):
    rng = np.random.default_rng(seed)
    if spec.bc == W.INTERFACE:
        spec.solution = W.piecewise_polynomial(spec.dim, deg, rng)
    else:
        spec.solution = W.Polynomial(spec.dim, deg, rng).manufactured()
    P = OracleProblem(spec)
    f, data = P.data()
    Au = P.op.apply(P.exact(), data, include_data=True)
    unk = P.unk_flat
    return np.max(np.abs(Au - f)[unk]) / np.max(np.abs(f[unk]))


CASES = {
    "dir2d_circle_4": lambda: W.ProblemSpec(n=40, geometry=W.Geometry(W.CIRCLE, (0.03, -0.01, 0.55), True),
                                            bc=W.DIRICHLET, order=4),
    "dir2d_star_6": lambda: W.ProblemSpec(n=64, geometry=W.Geometry(W.STAR, (0.02, 0.01, 0.5, 0.04, 5.0, 0.3), True),
                                          bc=W.DIRICHLET, order=6),
    "dir2d_ellipse_ext_4": lambda: W.ProblemSpec(n=64, geometry=W.Geometry(W.ELLIPSE, (0.0, 0.05, 0.35, 0.25, 0.4), False),
                                                 bc=W.DIRICHLET, order=4, box_bc=W.BOX_DIRICHLET),
    "neu2d_ext_6": lambda: W.ProblemSpec(n=56, geometry=W.Geometry(W.CIRCLE, (0.05, -0.02, 0.35), False),
                                         bc=W.NEUMANN, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=2.0),
    "neu2d_int_4": lambda: W.ProblemSpec(n=48, geometry=W.Geometry(W.ELLIPSE, (0.0, 0.0, 0.6, 0.45, 0.3), True),
                                         bc=W.NEUMANN, order=4),
    "iface2d_6": lambda: W.star_interface_1024(128),
    "iface2d_4_contrast": lambda: W.ProblemSpec(n=112, geometry=W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.1, 5.0, 0.0), False),
                                                bc=W.INTERFACE, order=4, box_bc=W.BOX_DIRICHLET,
                                                beta_plus=0.5, beta_minus=1.0),
    "dir3d_sphere_4": lambda: W.ProblemSpec(n=24, geometry=W.Geometry(W.SPHERE, (0.02, 0.0, -0.03, 0.6), True),
                                            bc=W.DIRICHLET, order=4),
    "neu3d_ellipsoid_4": lambda: W.ellipsoid_neumann_256(48),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_polynomial_exactness(case):
    spec = CASES[case]()
    assert _exactness_error(spec, spec.order) < 5e-10


@pytest.mark.parametrize("case", ["dir2d_star_6", "neu2d_ext_6", "iface2d_6"])
def test_exactness_has_teeth(case):
    """One degree more and the operator is no longer exact."""
    spec = CASES[case]()
    assert _exactness_error(spec, spec.order + 1) > 1e-8


def test_pure_neumann_operator_annihilates_constants():
    spec = CASES["neu2d_int_4"]()
    op = IIMOperator(spec)
    ones = op.unknown.ravel(order="F").astype(float)
    Au = op.apply(ones)
    assert np.max(np.abs(Au)) < 1e-9 * (1.0 / op.h ** 2)


def test_interface_closed_form_matches_jump_system():
    """Eqs. 10-11 equal the solution of the discrete jump system of Eq. 9 with [u] = j0."""
    spec = W.star_interface_1024(128)
    spec.beta_plus, spec.beta_minus = 0.5, 1.7
    op = IIMOperator(spec)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(op.n ** 2)
    K = op.cross.count
    data = {"g": np.zeros(K), "j0": rng.standard_normal(K), "j1": rng.standard_normal(K), "box": np.zeros(4 * op.n)}
    vals = op.control_values(u, data, include_data=True)
    bp, bm = spec.beta_plus, spec.beta_minus
    for c in range(0, K, 17):
        fp, fm = op.fits[(c, True)], op.fits[(c, False)]
        Dp, Dm = fp.deriv[1:] @ u[fp.nodes], fm.deriv[1:] @ u[fm.nodes]
        # unknowns (u+, u-):  u+ - u- = j0 ;  bp (s+_c u+ + Dp) - bm (s-_c u- + Dm) = j1
        M = np.array([[1.0, -1.0], [bp * fp.deriv[0], -bm * fm.deriv[0]]])
        rhs = np.array([data["j0"][c], data["j1"][c] - bp * Dp + bm * Dm])
        up, um = np.linalg.solve(M, rhs)
        assert abs(vals[(c, True)] - up) < 1e-9 * max(1, abs(up))
        assert abs(vals[(c, False)] - um) < 1e-9 * max(1, abs(um))


def _truncation(spec_fn, ns):
    errs = []
    for n in ns:
        spec = spec_fn(n)
        P = OracleProblem(spec)
        f, data = P.data()
        tau = P.op.apply(P.exact(), data, include_data=True) - f
        errs.append(np.max(np.abs(tau[P.unk_flat])))
    return [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]


@pytest.mark.parametrize("bc,order", [(W.DIRICHLET, 4), (W.NEUMANN, 4), (W.DIRICHLET, 6)])
def test_truncation_order_k_minus_2(bc, order):
    """Sec. 2.4: (n, n+1) discretisations have truncation error O(dx^(k-2)) = O(dx^(n-1))."""
    sol = W.sin_cos_2d(4 * np.pi / 3, 0.3, 2 * np.pi / 3, 0.1)

    def mk(n):
        return W.ProblemSpec(n=n, geometry=W.Geometry(W.STAR, (0.05, 0.03, 0.45, 0.03, 5.0, 0.2), False), bc=bc,
                             order=order, box_bc=W.BOX_DIRICHLET, solution=sol)
    slopes = _truncation(mk, (96, 192, 384))
    k = order + 1
    assert slopes[-1] > (k - 2) - 0.6
    assert slopes[-1] < (k - 2) + 1.0


def _golden_spectrum():
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "spectrum_bounds.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


@pytest.mark.parametrize("bc,order", [(W.DIRICHLET, 4), (W.NEUMANN, 4), (W.INTERFACE, 4), (W.NEUMANN, 6)])
def test_spectrum_bounds(bc, order):
    gold = _golden_spectrum()
    geom = W.Geometry(W.CIRCLE, (0.02, -0.03, 0.4), False)
    spec = W.ProblemSpec(n=36, geometry=geom, bc=bc, order=order, box_bc=W.BOX_DIRICHLET,
                         beta_plus=0.5 if bc == W.INTERFACE else 1.0, beta_minus=1.0)
    op = IIMOperator(spec)
    A, _ = assemble(op)
    beta_max = max(spec.beta_plus, spec.beta_minus) if bc == W.INTERFACE else spec.beta_plus
    lam = np.linalg.eigvals(A) * op.h ** 2 / beta_max
    assert np.max(lam.real) <= gold["re_upper"] + 1e-9
    lower = -2 * float(sigma_max(order)) * (1 + gold["neumann6_overshoot"] + 1e-3)
    assert np.min(lam.real) >= lower


@pytest.mark.parametrize("case", ["iface2d_6", "neu3d_ellipsoid_4", "dir2d_circle_4"])
def test_sampled_apply_equals_full_apply(case):
    """The lazy per-node evaluation used for full-size parity equals the full operator."""
    spec = CASES[case]()
    rng = np.random.default_rng(4)
    if spec.bc == W.INTERFACE:
        spec.solution = W.two_phase_star_solution()
    elif spec.solution is None:
        spec.solution = W.sin_cos_2d(1.3, 0.2, 0.7, 0.4)
    full = OracleProblem(spec)
    f, data = full.data()
    lazy = IIMOperator(spec, lazy=True)
    u = rng.standard_normal(spec.n ** spec.dim)
    nodes = np.concatenate([rng.choice(spec.n ** spec.dim, 200, replace=False),
                            np.array(sorted({r[0] for r in full.op.iim_rec}))[:150]])
    for incl in (False, True):
        ref = full.op.apply(u, data, incl)[nodes]
        assert np.max(np.abs(lazy.apply_at(u, nodes, data, incl) - ref)) < 1e-13 * np.max(np.abs(ref))
