"""Oracle pins for the 2D/3D Shortley-Weller assembly (paper Sec. 3.1, Eqs. 18-21, and the
red-black smoother of Sec. 3.3).

The 1D formulas are pinned elsewhere (exact on quadratics).  These tests pin how the
oracle's level operator puts them together on a grid: which side of a node a wall is on,
its distance (t from the lower node of the cut edge, so 1 - t seen from the upper node),
the shift of boundary walls to psi >= 1/2, the box faces at psi = 1/2, the Neumann cases
(a), (b), (c), the interface wall value of Eq. 21 with psi = 1/2 and its weights on the
two sides, and the colours of the Gauss-Seidel half sweeps.  Every expected value is a
property of the exact function used (its Laplacian, or 0), computed here in closed form;
wall distances come from closed-form roots, not from the oracle's crossings.

Planted mistakes each test was run against (all fail):
  * distance swap t <-> 1 - t in the per-side wall distance;
  * no shift of boundary walls to psi >= 1/2;
  * Neumann case (a) and (b) exchanged;
  * interface weights of the node and of its neighbour exchanged;
  * red and black exchanged in the half sweep.
"""
import numpy as np
import pytest

import workloads as W
from oracle.geometry import LevelSet, grid_x
from oracle.sw import SWLevel


class PlaneLevelSet:
    """phi = sign * (x_axis - x0): a flat body for the tests (the oracle's level sets
    are used through phi, normal, curvature and dim only)."""

    def __init__(self, dim, axis, x0, sign):
        self.dim, self.axis, self.x0, self.sign = dim, axis, x0, sign

    def phi(self, X):
        return self.sign * (X[..., self.axis] - self.x0)

    def normal(self, X):
        out = np.zeros(X.shape)
        out[..., self.axis] = -self.sign        # out of Omega+ = -grad(phi)
        return out

    def curvature(self, X):
        return np.zeros(X.shape[:-1])


class SlabLevelSet(PlaneLevelSet):
    """Omega+ = {a < x_axis < b} (two flat walls)."""

    def __init__(self, dim, axis, a, b):
        super().__init__(dim, axis, 0.0, 1.0)
        self.a, self.b = a, b

    def phi(self, X):
        x = X[..., self.axis]
        return np.minimum(x - self.a, self.b - x)

    def normal(self, X):
        out = np.zeros(X.shape)
        mid = 0.5 * (self.a + self.b)
        out[..., self.axis] = np.where(X[..., self.axis] < mid, -1.0, 1.0)
        return out


def _coords(n, d):
    x = grid_x(n)
    X = np.stack(np.meshgrid(*([x] * d), indexing="ij"), axis=-1)
    return X.reshape(-1, d, order="F")           # flat order, i0 fastest


def _index(n, d):
    return np.stack(np.unravel_index(np.arange(n ** d), (n,) * d, order="F"), axis=-1)


def _box_interior(n, d):
    """Nodes whose 2d neighbours are all inside the box."""
    idx = _index(n, d)
    return np.all((idx > 0) & (idx < n - 1), axis=1)


# ----------------------------------------------------------------------------- Dirichlet
def _ball_wall_distance(Xi, c, R, ax, s):
    """Distance from Xi (inside the ball) along s e_ax to the sphere |x - c| = R."""
    p = Xi - c
    return -s * p[..., ax] + np.sqrt(p[..., ax] ** 2 - np.sum(p * p, axis=-1) + R * R)


@pytest.mark.parametrize("dim", [2, 3])
def test_dirichlet_ball_quadratic_exact_where_walls_are_far(dim):
    """u = R^2 - |x - c|^2 vanishes on the circle (sphere), so the homogeneous Dirichlet
    walls carry its true value.  At every unknown whose walls all lie at least h/2 away
    (no shift), each 1D formula is exact: (A u)_i = lap u = -2 d.
    Catches: the t <-> 1 - t distance swap (wrong wall position at cut sides), and any
    side/formula mix-up at cut nodes."""
    n = 64 if dim == 2 else 24
    if dim == 2:
        c, R = np.array([0.031, -0.017]), 0.55
        geom = W.Geometry(W.CIRCLE, (c[0], c[1], R), True)
    else:
        c, R = np.array([0.021, -0.013, 0.008]), 0.6
        geom = W.Geometry(W.SPHERE, (c[0], c[1], c[2], R), True)
    L = SWLevel(LevelSet(geom), n, W.DIRICHLET, W.BOX_NONE, 1.0, 1.0)
    X = _coords(n, dim)
    h = 2.0 / n
    u = R * R - np.sum((X - c) ** 2, axis=1)
    inside = np.sum((X - c) ** 2, axis=1) <= R * R
    assert np.array_equal(inside, L.unk_flat)
    far, ncut = inside.copy(), np.zeros(n ** dim, dtype=int)
    for ax in range(dim):
        for s in (-1, 1):
            Y = X.copy()
            Y[:, ax] += s * h
            cut = inside & (np.sum((Y - c) ** 2, axis=1) > R * R)
            dist = np.full(n ** dim, h)
            dist[cut] = _ball_wall_distance(X[cut], c, R, ax, s)
            far &= ~cut | (dist >= 0.5 * h)
            ncut += cut
    sel = far & (ncut > 0)
    assert sel.sum() > 20
    Au = L.apply(u)
    assert np.max(np.abs(Au[sel] + 2 * dim)) < 1e-9 * 2 * dim


@pytest.mark.parametrize("dim", [2, 3])
def test_dirichlet_single_cut_rows_use_the_shifted_wall(dim):
    """At an unknown with exactly one cut side (axis a, direction s, true wall distance
    d h), the operator sees a zero wall at psi = max(d, 1/2): the quadratic
    q(x) = (x_a - w)(x_a - w - 1), w = x_a(i) + s max(d, 1/2) h, which vanishes there and
    is constant along the other axes, gives (A q)_i = 2 exactly.
    Catches: no shift to psi >= 1/2 (rows with d < 1/2), the t <-> 1 - t swap."""
    n = 64 if dim == 2 else 24
    if dim == 2:
        c, R = np.array([0.031, -0.017]), 0.55
        geom = W.Geometry(W.CIRCLE, (c[0], c[1], R), True)
    else:
        c, R = np.array([0.021, -0.013, 0.008]), 0.6
        geom = W.Geometry(W.SPHERE, (c[0], c[1], c[2], R), True)
    L = SWLevel(LevelSet(geom), n, W.DIRICHLET, W.BOX_NONE, 1.0, 1.0)
    X = _coords(n, dim)
    h = 2.0 / n
    inside = np.sum((X - c) ** 2, axis=1) <= R * R
    cuts = []
    for ax in range(dim):
        for s in (-1, 1):
            Y = X.copy()
            Y[:, ax] += s * h
            cut = inside & (np.sum((Y - c) ** 2, axis=1) > R * R)
            cuts.append((ax, s, cut))
    ncut = sum(cut.astype(int) for _, _, cut in cuts)
    near = far = 0
    for ax, s, cut in cuts:
        for i in np.nonzero(cut & (ncut == 1))[0]:
            d = _ball_wall_distance(X[i], c, R, ax, s) / h
            w = X[i, ax] + s * max(d, 0.5) * h
            q = (X[:, ax] - w) * (X[:, ax] - w - 1.0)
            val = L.A[i] @ q
            assert abs(val[0] - 2.0) < 1e-9, (i, ax, s, d, val)
            near += d < 0.5
            far += d >= 0.5
    assert near > 5 and far > 5


def test_box_faces_are_dirichlet_walls_at_half_a_cell():
    """Outer box (Dirichlet, faces half a cell beyond the first and last nodes): the
    product u = prod_k (1 - x_k^2) vanishes on every face and is quadratic along each
    grid line, so at every unknown with no immersed wall (A u)_i = lap u, box rows
    included.  Catches: a box wall at a distance other than h/2, or a nonzero box value."""
    n = 48
    geom = W.Geometry(W.ELLIPSE, (0.02, -0.01, 0.35, 0.25, 0.3), False)
    for bc in (W.NEUMANN, W.INTERFACE):
        L = SWLevel(LevelSet(geom), n, bc, W.BOX_DIRICHLET, 1.0, 1.0)
        X = _coords(n, 2)
        u = (1 - X[:, 0] ** 2) * (1 - X[:, 1] ** 2)
        lap = -2 * (1 - X[:, 1] ** 2) - 2 * (1 - X[:, 0] ** 2)
        plus = L.plus.ravel(order="F")
        idx = _index(n, 2)
        clean = L.unk_flat & plus
        for ax in range(2):
            for s in (-1, 1):
                j = idx[:, ax] + s
                inb = (j >= 0) & (j < n)
                nb = np.where(inb, np.arange(n * n) + s * n ** ax, 0)
                clean &= ~inb | (plus[nb] == plus)
        box_rows = clean & ~_box_interior(n, 2)
        assert box_rows.sum() > 4 * (n - 2) - 8
        Au = L.apply(u)
        assert np.max(np.abs(Au[clean] - lap[clean])) < 1e-9


# ----------------------------------------------------------------------------- Neumann
@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 2)])
@pytest.mark.parametrize("side", ["a", "b"])
@pytest.mark.parametrize("frac", [0.7, 0.3])
def test_neumann_wall_cases_a_and_b(dim, axis, side, frac):
    """A flat Neumann wall normal to ``axis``: Omega+ above it (case (a), wall on the low
    side of its first nodes) or below it (case (b)).  The first node lies frac h from the
    wall; the operator sees the wall at psi = max(frac, 1/2).  u = (x_a - w)^2 + y^2, w the
    seen wall, has zero derivative along the axis there, so (A u)_i = lap u = 4 at every
    unknown whose other neighbours are in the box.
    Catches: cases (a) and (b) exchanged, the t <-> 1 - t swap (frac = 0.7), no shift
    to 1/2 (frac = 0.3)."""
    n = 32
    h = 2.0 / n
    x = grid_x(n)
    k = n // 2
    if side == "a":      # Omega+ = {x_a >= x0}, first node k at x0 + frac h
        x0 = x[k] - frac * h
        ls = PlaneLevelSet(dim, axis, x0, 1.0)
        w = x[k] - max(frac, 0.5) * h
    else:                # Omega+ = {x_a <= x0}, last node k at x0 - frac h
        x0 = x[k] + frac * h
        ls = PlaneLevelSet(dim, axis, x0, -1.0)
        w = x[k] + max(frac, 0.5) * h
    L = SWLevel(ls, n, W.NEUMANN, W.BOX_DIRICHLET, 1.0, 1.0)
    X = _coords(n, dim)
    other = (axis + 1) % dim
    u = (X[:, axis] - w) ** 2 + X[:, other] ** 2
    sel = L.unk_flat & _box_interior(n, dim)
    idx = _index(n, dim)
    wall_rows = sel & (idx[:, axis] == k)
    assert wall_rows.sum() == (n - 2) ** (dim - 1)
    Au = L.apply(u)
    assert np.max(np.abs(Au[sel] - 4.0)) < 1e-9


@pytest.mark.parametrize("dim,axis", [(2, 0), (3, 1)])
def test_neumann_case_c_both_walls(dim, axis):
    """A slab one node thick (walls on both sides of the same node, case (c)): with zero
    flux through both walls the axis contributes nothing, so for u = y^2 (+ any function
    of x_axis) (A u)_i = 2 from the other axis alone.  Catches a case (c) row that reads
    the node's own value or a neighbour."""
    n = 32
    h = 2.0 / n
    x = grid_x(n)
    k = n // 2
    ls = SlabLevelSet(dim, axis, x[k] - 0.6 * h, x[k] + 0.7 * h)
    L = SWLevel(ls, n, W.NEUMANN, W.BOX_DIRICHLET, 1.0, 1.0)
    X = _coords(n, dim)
    other = (axis + 1) % dim
    sel = L.unk_flat & _box_interior(n, dim)
    assert sel.sum() == (n - 2) ** (dim - 1)
    for fx in (lambda t: 0 * t, lambda t: np.sin(3 * t) + t * t):
        u = X[:, other] ** 2 + fx(X[:, axis])
        Au = L.apply(u)
        assert np.max(np.abs(Au[sel] - 2.0)) < 1e-9


# ----------------------------------------------------------------------------- interface
@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 2)])
@pytest.mark.parametrize("frac", [0.5, 0.2, 0.85])
@pytest.mark.parametrize("betas", [(1.0, 1.0), (0.25, 3.0), (5.0, 0.5)])
def test_interface_reproduces_flux_continuous_piecewise_linear(dim, axis, frac, betas):
    """Flat interface normal to ``axis`` between nodes k and k+1 (at frac h above node k).
    With psi+ = psi- = 1/2 (Sec. 3.1) the operator sees the interface at the midpoint m of
    the cut edge whatever frac is.  A function linear on each side with its kink at m,
    continuous there and with continuous flux (beta- s- = beta+ s+), plus a linear term
    along the other axes, is reproduced by the Eq. 21 wall value and the exact 1D
    formulas: (A u)_i = 0 at every node whose neighbours are in the box.
    Catches: the weights of the node and of its neighbour exchanged (beta+ != beta-), an
    interface psi other than 1/2, a coupling to the wrong neighbour."""
    bp, bm = betas
    n = 24 if dim == 3 else 32
    h = 2.0 / n
    x = grid_x(n)
    k = n // 2
    ls = PlaneLevelSet(dim, axis, x[k] + frac * h, 1.0)      # Omega+ above the plane
    L = SWLevel(ls, n, W.INTERFACE, W.BOX_DIRICHLET, bp, bm)
    X = _coords(n, dim)
    m = x[k] + 0.5 * h
    s_minus = 0.7
    s_plus = bm * s_minus / bp
    xa = X[:, axis] - m
    u = 0.3 + np.where(xa > 0, s_plus * xa, s_minus * xa)
    for other in range(dim):
        if other != axis:
            u = u + (0.4 + 0.1 * other) * X[:, other]
    sel = _box_interior(n, dim)
    Au = L.apply(u)
    assert np.max(np.abs(Au[sel])) < 1e-9
    # the rows next to the interface carry the coupling
    idx = _index(n, dim)
    near = sel & ((idx[:, axis] == k) | (idx[:, axis] == k + 1))
    assert near.sum() == 2 * (n - 2) ** (dim - 1)


# ----------------------------------------------------------------------------- smoother
@pytest.mark.parametrize("bc", [W.DIRICHLET, W.NEUMANN, W.INTERFACE])
def test_gauss_seidel_colours(bc):
    """gs_colour(u, f, 0) updates exactly the unknowns with an even index sum (red) and
    leaves every other entry bit-identical; afterwards the red rows of A u = f hold
    (their neighbours are all black, interface couplings included).  Then colour 1 does
    the same for the black unknowns.  Catches red and black exchanged, and a half sweep
    that reads values it has already updated."""
    n = 48
    rng = np.random.default_rng(5)
    if bc == W.DIRICHLET:
        geom, box = W.Geometry(W.STAR, (0.03, 0.02, 0.55, 0.05, 5.0, 0.4), True), W.BOX_NONE
    elif bc == W.NEUMANN:
        geom, box = W.Geometry(W.ELLIPSE, (0.02, -0.01, 0.35, 0.25, 0.3), False), W.BOX_DIRICHLET
    else:
        geom, box = W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.05, 5.0, 0.0), False), W.BOX_DIRICHLET
    L = SWLevel(LevelSet(geom), n, bc, box, 0.5, 2.0)
    idx = _index(n, 2)
    even = (idx.sum(axis=1) % 2 == 0)
    f = rng.standard_normal(n * n)
    u0 = rng.standard_normal(n * n)
    u0[~L.unk_flat] = 0.0
    for colour, mask in ((0, even), (1, ~even)):
        u = u0.copy()
        L.gs_colour(u, f, colour)
        changed = u != u0
        assert np.all(~changed[~(mask & L.unk_flat)])
        assert changed[mask & L.unk_flat].mean() > 0.99
        r = f - L.apply(u)
        rows = mask & L.unk_flat & (L.diag != 0)
        assert np.max(np.abs(r[rows])) < 1e-9 * np.max(np.abs(f))
