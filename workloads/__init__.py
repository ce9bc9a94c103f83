"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *describes* problems and evaluates the manufactured
solutions that generate their data (source term, boundary values, jumps).
It contains none of the solver's arithmetic: no crossings, no fits, no
stencils.  Both sides evaluate the data below at the points *they* computed.

Problem statement (paper Sec. 2.1, Eq. 1 and Sec. 2.2, Eq. 8):
  div(beta grad u) = f  in Omega,   u = ubar on Gamma_D,
  beta du/dn = qbar on Gamma_N,     [u] = j0, [beta du/dn] = j1 on Gamma_M,
with n pointing out of Omega+ (towards Omega-), [.] = (+ side) - (- side).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# geometry kinds (same integer codes as the C header)
CIRCLE, ELLIPSE, STAR, SPHERE, ELLIPSOID, PERTURBED_SPHERE = 0, 1, 2, 3, 4, 5
FOURIER, LEVELSET_GRID = 6, 7
# the perturbation of PERTURBED_SPHERE: the real spherical harmonic of degree 3, order 2,
# (e_x^2 - e_y^2) e_z for the unit direction e, scaled to a maximum of 1 on the sphere
PERTURB_SCALE = 1.5 * math.sqrt(3.0)
# boundary condition kinds
DIRICHLET, NEUMANN, INTERFACE = 0, 1, 2
# outer box condition
BOX_NONE, BOX_DIRICHLET = 0, 1


@dataclass
class Geometry:
    """An immersed body.  ``plus_inside`` selects which side is Omega+.

    params by kind:
      CIRCLE    (cx, cy, R)
      ELLIPSE   (cx, cy, a0, a1, angle)          semi-axes along the rotated axes
      STAR      (cx, cy, r0, amp, m, phase)      r(theta) = r0 + amp sin(m theta + phase)
      SPHERE    (cx, cy, cz, R)
      ELLIPSOID (cx, cy, cz, a0, a1, a2)         axis-aligned
      PERTURBED_SPHERE (cx, cy, cz, rho0, rho1)  r(e) = rho0 + rho1 Y(e), Y the degree-3
                                                 harmonic above (max |Y| = 1)
      FOURIER   (cx, cy)                         r(theta) = a0 + sum_k a_k cos k theta + b_k sin k theta,
                                                 ``coef`` = (a0, a1, b1, ..., aK, bK)
      LEVELSET_GRID ()                           ``values``: the level set at the grid's nodes,
                                                 shape (n,)*d indexed [i0, i1, (i2)]
    """
    kind: int
    params: tuple
    plus_inside: bool
    coef: tuple = ()
    values: object = None

    @property
    def dim(self) -> int:
        if self.kind == LEVELSET_GRID:
            return int(np.asarray(self.values).ndim)
        return 3 if self.kind in (SPHERE, ELLIPSOID, PERTURBED_SPHERE) else 2


@dataclass
class Manufactured:
    """Piecewise manufactured solution: ``u_plus`` on Omega+, ``u_minus`` on Omega-.

    Each entry is a callable ``(X) -> value`` with ``X`` of shape (..., d);
    ``grad_*`` return (..., d); ``lap_*`` return the Laplacian.
    """
    u_plus: object
    grad_plus: object
    lap_plus: object
    u_minus: object = None
    grad_minus: object = None
    lap_minus: object = None


@dataclass
class ProblemSpec:
    n: int
    geometry: Geometry
    bc: int
    order: int                     # 4 -> (4,5), 6 -> (6,7)
    box_bc: int = BOX_NONE
    beta_plus: float = 1.0
    beta_minus: float = 1.0
    solution: Manufactured = None
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.geometry.dim


# ----------------------------------------------------------------------------
# grid coordinates (cell-centred, [-1,1]^d): x_i = -1 + (i + 1/2) h
# ----------------------------------------------------------------------------
def node_coords(n: int, dim: int) -> np.ndarray:
    """Coordinates of all nodes, shape (n,)*dim + (dim,), index order [i0, i1, (i2)]."""
    h = 2.0 / n
    x = -1.0 + (np.arange(n) + 0.5) * h
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    return np.stack(grids, axis=-1)


def to_flat(a: np.ndarray) -> np.ndarray:
    """[i0, i1, i2]-indexed grid array -> flat vector with i0 fastest."""
    return np.ascontiguousarray(a).ravel(order="F")


def from_flat(v: np.ndarray, n: int, dim: int) -> np.ndarray:
    return np.asarray(v).reshape((n,) * dim, order="F")


# ----------------------------------------------------------------------------
# manufactured solutions
# ----------------------------------------------------------------------------
def harmonic_exp_sin() -> Manufactured:
    """u = exp(x) sin(y): harmonic (Laplace problem of the 64^2 circle case)."""
    u = lambda X, xp=np: xp.exp(X[..., 0]) * xp.sin(X[..., 1])
    g = lambda X, xp=np: xp.stack([xp.exp(X[..., 0]) * xp.sin(X[..., 1]),
                                   xp.exp(X[..., 0]) * xp.cos(X[..., 1])], axis=-1)
    lap = lambda X, xp=np: 0.0 * X[..., 0]
    return Manufactured(u, g, lap)


def two_phase_star_solution() -> Manufactured:
    """u- = sin(pi x) cos(pi y) inside the star, u+ = exp(x+y)/4 outside."""
    pi = math.pi
    um = lambda X: np.sin(pi * X[..., 0]) * np.cos(pi * X[..., 1])
    gm = lambda X: np.stack([pi * np.cos(pi * X[..., 0]) * np.cos(pi * X[..., 1]),
                             -pi * np.sin(pi * X[..., 0]) * np.sin(pi * X[..., 1])], axis=-1)
    lm = lambda X: -2 * pi * pi * np.sin(pi * X[..., 0]) * np.cos(pi * X[..., 1])
    up = lambda X: np.exp(X[..., 0] + X[..., 1]) / 4
    gp = lambda X: np.stack([np.exp(X[..., 0] + X[..., 1]) / 4] * 2, axis=-1)
    lp = lambda X: np.exp(X[..., 0] + X[..., 1]) / 2
    return Manufactured(up, gp, lp, um, gm, lm)


def sin2x_sin3y_cosz() -> Manufactured:
    u = lambda X: np.sin(2 * X[..., 0]) * np.sin(3 * X[..., 1]) * np.cos(X[..., 2])
    g = lambda X: np.stack([
        2 * np.cos(2 * X[..., 0]) * np.sin(3 * X[..., 1]) * np.cos(X[..., 2]),
        3 * np.sin(2 * X[..., 0]) * np.cos(3 * X[..., 1]) * np.cos(X[..., 2]),
        -np.sin(2 * X[..., 0]) * np.sin(3 * X[..., 1]) * np.sin(X[..., 2])], axis=-1)
    lap = lambda X: -14 * np.sin(2 * X[..., 0]) * np.sin(3 * X[..., 1]) * np.cos(X[..., 2])
    return Manufactured(u, g, lap)


def sin_cos_2d(a1, b1, a2, b2) -> Manufactured:
    """u = sin(a1 x + b1) cos(a2 y + b2) (batch / serving draws).

    Every callable takes an optional array namespace ``xp`` (numpy by default, or
    torch for device tensors)."""
    u = lambda X, xp=np: xp.sin(a1 * X[..., 0] + b1) * xp.cos(a2 * X[..., 1] + b2)
    g = lambda X, xp=np: xp.stack([a1 * xp.cos(a1 * X[..., 0] + b1) * xp.cos(a2 * X[..., 1] + b2),
                                   -a2 * xp.sin(a1 * X[..., 0] + b1) * xp.sin(a2 * X[..., 1] + b2)], axis=-1)
    lap = lambda X, xp=np: -(a1 * a1 + a2 * a2) * u(X, xp)
    return Manufactured(u, g, lap)


def sin_sin_cos_3d(a, b) -> Manufactured:
    """u = sin(a0 x + b0) sin(a1 y + b1) cos(a2 z + b2) (array namespace as in sin_cos_2d)."""
    s = lambda X, xp: (xp.sin(a[0] * X[..., 0] + b[0]), xp.sin(a[1] * X[..., 1] + b[1]),
                       xp.cos(a[2] * X[..., 2] + b[2]))
    c = lambda X, xp: (xp.cos(a[0] * X[..., 0] + b[0]), xp.cos(a[1] * X[..., 1] + b[1]),
                       -xp.sin(a[2] * X[..., 2] + b[2]))

    def u(X, xp=np):
        p, q, r = s(X, xp)
        return p * q * r

    def g(X, xp=np):
        p, q, r = s(X, xp)
        dp, dq, dr = c(X, xp)
        return xp.stack([a[0] * dp * q * r, a[1] * p * dq * r, a[2] * p * q * dr], axis=-1)

    lap = lambda X, xp=np: -(a[0] ** 2 + a[1] ** 2 + a[2] ** 2) * u(X, xp)
    return Manufactured(u, g, lap)


def sin_sum_3d(k=2.0 * math.pi) -> Manufactured:
    """u = sin(k x) + sin(k y) + sin(k z).  With k = 2 pi this is the paper's 3D verification
    solution sin(4 pi x_i) summed, on the unit cube mapped to [-1,1]^3."""
    u = lambda X, xp=np: xp.sin(k * X[..., 0]) + xp.sin(k * X[..., 1]) + xp.sin(k * X[..., 2])
    g = lambda X, xp=np: xp.stack([k * xp.cos(k * X[..., 0]), k * xp.cos(k * X[..., 1]),
                                   k * xp.cos(k * X[..., 2])], axis=-1)
    lap = lambda X, xp=np: -(k * k) * u(X, xp)
    return Manufactured(u, g, lap)


def perturbed_sphere(n: int, bc: int = DIRICHLET) -> "ProblemSpec":
    """The paper's 3D verification body (a sphere of radius 0.35 perturbed by 0.05 times a
    spherical harmonic, in the unit cube), mapped to [-1,1]^3: rho0 = 0.7, rho1 = 0.1,
    centred; interior problem (no outer box), Dirichlet or Neumann, (4,5)."""
    return ProblemSpec(n=n, geometry=Geometry(PERTURBED_SPHERE, (0.0, 0.0, 0.0, 0.7, 0.1), plus_inside=True),
                       bc=bc, order=4, box_bc=BOX_NONE, solution=sin_sum_3d(),
                       name=f"perturbed_sphere_{'dir' if bc == DIRICHLET else 'neu'}_{n}")


class Polynomial:
    """Random polynomial of total degree <= deg in d variables (exactness tests)."""

    def __init__(self, dim, deg, rng, scale=1.0):
        self.dim, self.deg = dim, deg
        self.exps = [e for e in _exponents(dim, deg)]
        self.coef = rng.standard_normal(len(self.exps)) * scale

    def __call__(self, X):
        out = np.zeros(X.shape[:-1])
        for c, e in zip(self.coef, self.exps):
            t = np.full(X.shape[:-1], c)
            for k in range(self.dim):
                t = t * X[..., k] ** e[k]
            out += t
        return out

    def grad(self, X):
        out = np.zeros(X.shape)
        for c, e in zip(self.coef, self.exps):
            for k in range(self.dim):
                if e[k] == 0:
                    continue
                t = np.full(X.shape[:-1], c * e[k])
                for m in range(self.dim):
                    t = t * X[..., m] ** (e[m] - (1 if m == k else 0))
                out[..., k] += t
        return out

    def lap(self, X):
        out = np.zeros(X.shape[:-1])
        for c, e in zip(self.coef, self.exps):
            for k in range(self.dim):
                if e[k] < 2:
                    continue
                t = np.full(X.shape[:-1], c * e[k] * (e[k] - 1))
                for m in range(self.dim):
                    t = t * X[..., m] ** (e[m] - (2 if m == k else 0))
                out += t
        return out

    def manufactured(self) -> Manufactured:
        return Manufactured(self, self.grad, self.lap)


def _exponents(dim, deg):
    if dim == 1:
        for a in range(deg + 1):
            yield (a,)
        return
    for a in range(deg + 1):
        for rest in _exponents(dim - 1, deg - a):
            yield (a,) + rest


def piecewise_polynomial(dim, deg, rng) -> Manufactured:
    p, m = Polynomial(dim, deg, rng), Polynomial(dim, deg, rng)
    return Manufactured(p, p.grad, p.lap, m, m.grad, m.lap)


# ----------------------------------------------------------------------------
# data evaluation at points supplied by the caller (each side passes its own)
# ----------------------------------------------------------------------------
def source_term(spec: ProblemSpec, X: np.ndarray, phase_plus: np.ndarray) -> np.ndarray:
    """f = beta lap(u) per phase at nodes X; ``phase_plus`` marks Omega+ nodes."""
    s = spec.solution
    fp = spec.beta_plus * s.lap_plus(X)
    if spec.bc == INTERFACE:
        fm = spec.beta_minus * s.lap_minus(X)
        return np.where(phase_plus, fp, fm)
    return np.where(phase_plus, fp, 0.0)


def source_term_device(spec: ProblemSpec, phase_plus):
    """source_term on the device for the boundary problems of the batch and serving
    mixes: ``phase_plus`` is the problem's phase (torch uint8/bool, flat order); the
    result is a flat float64 torch tensor on the same device.  Needs a solution
    family written for an array namespace (harmonic_exp_sin, sin_cos_2d, sin_sin_cos_3d)."""
    import torch
    n, d = spec.n, spec.dim
    x = -1.0 + (torch.arange(n, dtype=torch.float64, device=phase_plus.device) + 0.5) * (2.0 / n)
    X = torch.stack(torch.meshgrid(*([x] * d), indexing="ij"), dim=-1)
    lap = spec.solution.lap_plus(X, torch)
    flat = lap.permute(*reversed(range(d))).reshape(-1)          # order "F": x0 fastest
    if spec.bc == INTERFACE:
        raise ValueError("source_term_device covers boundary problems only")
    return torch.where(phase_plus.bool(), spec.beta_plus * flat, torch.zeros((), dtype=flat.dtype, device=flat.device))


def boundary_data(spec: ProblemSpec, xc: np.ndarray, normal: np.ndarray):
    """Per-control-point data.  Returns (g, j0, j1):

    Dirichlet: g = u(xc);  Neumann: g = beta+ grad u . n;
    interface: j0 = u+ - u-, j1 = beta+ du+/dn - beta- du-/dn.
    ``normal`` points out of Omega+.
    """
    s = spec.solution
    k = xc.shape[0]
    z = np.zeros(k)
    if spec.bc == DIRICHLET:
        return s.u_plus(xc), z, z
    if spec.bc == NEUMANN:
        return spec.beta_plus * np.sum(s.grad_plus(xc) * normal, axis=-1), z, z
    j0 = s.u_plus(xc) - s.u_minus(xc)
    j1 = (spec.beta_plus * np.sum(s.grad_plus(xc) * normal, axis=-1)
          - spec.beta_minus * np.sum(s.grad_minus(xc) * normal, axis=-1))
    return z, j0, j1


def box_face_points(n: int, dim: int) -> np.ndarray:
    """Outer-box Dirichlet sample points, one per grid line and face.

    Order: faces (-x0, +x0, -x1, +x1, [-x2, +x2]); within a face the remaining
    node indices in flat order (lowest remaining axis fastest).  The point lies
    on the face (coordinate +-1) with the other coordinates of the grid line.
    """
    h = 2.0 / n
    x = -1.0 + (np.arange(n) + 0.5) * h
    pts = []
    for ax in range(dim):
        others = [k for k in range(dim) if k != ax]
        for side in (-1.0, 1.0):
            grids = np.meshgrid(*([x] * len(others)), indexing="ij")
            flat = [g.ravel(order="F") for g in grids]
            P = np.zeros((flat[0].size, dim))
            for k, f in zip(others, flat):
                P[:, k] = f
            P[:, ax] = side
            pts.append(P)
    return np.concatenate(pts, axis=0)


def box_data(spec: ProblemSpec) -> np.ndarray:
    if spec.box_bc != BOX_DIRICHLET:
        return np.zeros(0)
    return spec.solution.u_plus(box_face_points(spec.n, spec.dim))


# ----------------------------------------------------------------------------
# level sets given at the grid's nodes (input for LEVELSET_GRID)
# ----------------------------------------------------------------------------
def sampled_levelset(fn, n: int, dim: int, plus_inside: bool = False) -> Geometry:
    """A LEVELSET_GRID geometry from a field ``fn(X)`` evaluated at the nodes of an n^dim grid."""
    return Geometry(LEVELSET_GRID, (), plus_inside, values=np.asarray(fn(node_coords(n, dim)), dtype=float))


def quadric_field(center, axes, angle=0.0):
    """phi = 1 - sum_k (y_k / a_k)^2, y = Rot(-angle)(x - center) (2D) or y = x - center (3D):
    positive inside the ellipse (ellipsoid), a polynomial of degree 2."""
    c = np.asarray(center, dtype=float)
    a = np.asarray(axes, dtype=float)

    def fn(X):
        d = X - c
        if c.size == 2:
            cs, sn = math.cos(angle), math.sin(angle)
            y0 = cs * d[..., 0] + sn * d[..., 1]
            y1 = -sn * d[..., 0] + cs * d[..., 1]
            return 1.0 - (y0 / a[0]) ** 2 - (y1 / a[1]) ** 2
        return 1.0 - np.sum((d / a) ** 2, axis=-1)
    return fn


def star_field(cx, cy, r0, amp, m, phase):
    """phi = r0 + amp sin(m theta + phase) - |x - c|: positive inside the star curve."""
    def fn(X):
        dx, dy = X[..., 0] - cx, X[..., 1] - cy
        return r0 + amp * np.sin(m * np.arctan2(dy, dx) + phase) - np.hypot(dx, dy)
    return fn


def blob_field(center, radius, eps, k):
    """A smooth body with no closed form here: phi = R^2 - |x - c|^2 + eps prod_i sin(k x_i + i),
    positive inside (2D or 3D)."""
    c = np.asarray(center, dtype=float)

    def fn(X):
        d = X - c
        w = np.ones(X.shape[:-1])
        for i in range(c.size):
            w = w * np.sin(k * X[..., i] + i)
        return radius ** 2 - np.sum(d * d, axis=-1) + eps * w
    return fn


# ----------------------------------------------------------------------------
# the paper-shaped configurations
# ----------------------------------------------------------------------------
def circle_dirichlet_64(n: int = 64) -> ProblemSpec:
    """2D Laplace, interior of the circle R=0.5, Dirichlet, (4,5)."""
    return ProblemSpec(n=n, geometry=Geometry(CIRCLE, (0.0, 0.0, 0.5), plus_inside=True),
                       bc=DIRICHLET, order=4, box_bc=BOX_NONE,
                       solution=harmonic_exp_sin(), name=f"circle_dirichlet_{n}")


def star_interface_1024(n: int = 1024, phase: float = 0.0) -> ProblemSpec:
    """2D two-phase Poisson, star r = 0.5 + 0.1 sin(5 theta), (6,7), Dirichlet box."""
    return ProblemSpec(n=n, geometry=Geometry(STAR, (0.0, 0.0, 0.5, 0.1, 5.0, phase), plus_inside=False),
                       bc=INTERFACE, order=6, box_bc=BOX_DIRICHLET, beta_plus=1.0, beta_minus=1.0,
                       solution=two_phase_star_solution(), name=f"star_interface_{n}")


def ellipsoid_neumann_256(n: int = 256) -> ProblemSpec:
    """3D exterior of the ellipsoid (0.6,0.45,0.35), Neumann on it, Dirichlet box, (4,5)."""
    return ProblemSpec(n=n, geometry=Geometry(ELLIPSOID, (0.0, 0.0, 0.0, 0.6, 0.45, 0.35), plus_inside=False),
                       bc=NEUMANN, order=4, box_bc=BOX_DIRICHLET,
                       solution=sin2x_sin3y_cosz(), name=f"ellipsoid_neumann_{n}")


def _star_amp_limit(n, m, r0):
    """Largest star amplitude keeping |kappa h| < 1/4 with a margin.

    Curvature of r = r0 + a sin(m t) peaks near the lobe tips; scanned numerically.
    This bounds the random draw only; the solver re-checks the curvature itself.
    """
    h = 2.0 / n
    t = np.linspace(0, 2 * np.pi, 4001)
    lo, hi = 0.0, 0.5 * r0
    for _ in range(50):
        a = 0.5 * (lo + hi)
        r = r0 + a * np.sin(m * t)
        r1 = a * m * np.cos(m * t)
        r2 = -a * m * m * np.sin(m * t)
        kap = np.abs(r * r + 2 * r1 * r1 - r * r2) / (r * r + r1 * r1) ** 1.5
        if np.max(kap) * h < 0.2:
            lo = a
        else:
            hi = a
    return lo


def batch_specs(count: int = 512, seed: int = 2503, n_lo: int = 64, n_hi: int = 512, n_step: int = 32):
    """Mixed batch of independent 2D problems (ellipses / 5-7 lobe stars).

    N uniform over multiples of ``n_step`` in [n_lo, n_hi]; 50% interior Dirichlet,
    50% exterior Neumann with a Dirichlet box; 50% (4,5), 50% (6,7);
    u = sin(a1 x + b1) cos(a2 y + b2).
    """
    rng = np.random.default_rng(seed)
    ns = np.arange(n_lo, n_hi + 1, n_step)
    specs = []
    for i in range(count):
        n = int(rng.choice(ns))
        order = 4 if rng.random() < 0.5 else 6
        interior = rng.random() < 0.5
        c = rng.uniform(-0.15, 0.15, size=2)
        if rng.random() < 0.5:
            # semi-axes redrawn until the ellipse's largest curvature a_max / a_min^2 keeps
            # |kappa h| < 0.2 (the bound is 1/4, Eq. 3)
            while True:
                a0, a1 = rng.uniform(0.3, 0.55, size=2)
                if not interior:
                    a0, a1 = 0.6 * a0, 0.6 * a1 + 0.1
                if max(a0, a1) / min(a0, a1) ** 2 * (2.0 / n) < 0.2:
                    break
            geom = Geometry(ELLIPSE, (c[0], c[1], a0, a1, rng.uniform(0, np.pi)), plus_inside=interior)
        else:
            m = int(rng.choice([5, 6, 7]))
            r0 = rng.uniform(0.3, 0.55) if interior else rng.uniform(0.25, 0.4)
            amp = rng.uniform(0, 0.8) * _star_amp_limit(n, m, r0)
            geom = Geometry(STAR, (c[0], c[1], r0, amp, float(m), rng.uniform(0, 2 * np.pi)), plus_inside=interior)
        a = rng.uniform(1, 3, size=2)
        b = rng.uniform(0, 2 * np.pi, size=2)
        sol = sin_cos_2d(a[0], b[0], a[1], b[1])
        if interior:
            spec = ProblemSpec(n=n, geometry=geom, bc=DIRICHLET, order=order, box_bc=BOX_NONE,
                               solution=sol, name=f"batch{i}")
        else:
            spec = ProblemSpec(n=n, geometry=geom, bc=NEUMANN, order=order, box_bc=BOX_DIRICHLET,
                               solution=sol, name=f"batch{i}")
        specs.append(spec)
    return specs


def serving_trace(count: int = 2000, rate: float = 200.0, seed: int = 22455,
                  n2_lo=128, n2_hi=1024, n3_lo=64, n3_hi=192, frac_3d=0.25, step=32):
    """Poisson arrival stream: list of (arrival_time_s, ProblemSpec)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        order = 4 if rng.random() < 0.5 else 6
        a = rng.uniform(1, 3, size=3)
        b = rng.uniform(0, 2 * np.pi, size=3)
        if rng.random() < frac_3d:
            n = int(rng.choice(np.arange(n3_lo, n3_hi + 1, step)))
            ax = rng.uniform(0.3, 0.55, size=3)
            c = rng.uniform(-0.1, 0.1, size=3)
            interior = rng.random() < 0.5
            geom = Geometry(ELLIPSOID, (c[0], c[1], c[2], ax[0], ax[1], ax[2]), plus_inside=interior)
            sol = sin_sin_cos_3d(a, b)
            order = 4
        else:
            n = int(rng.choice(np.arange(n2_lo, n2_hi + 1, step)))
            interior = rng.random() < 0.5
            m = int(rng.choice([5, 6, 7]))
            r0 = rng.uniform(0.3, 0.5) if interior else rng.uniform(0.25, 0.4)
            amp = rng.uniform(0, 0.8) * _star_amp_limit(n, m, r0)
            c = rng.uniform(-0.15, 0.15, size=2)
            geom = Geometry(STAR, (c[0], c[1], r0, amp, float(m), rng.uniform(0, 2 * np.pi)), plus_inside=interior)
            sol = sin_cos_2d(a[0], b[0], a[1], b[1])
        if interior:
            spec = ProblemSpec(n=n, geometry=geom, bc=DIRICHLET, order=order, box_bc=BOX_NONE,
                               solution=sol, name=f"req{i}")
        else:
            spec = ProblemSpec(n=n, geometry=geom, bc=NEUMANN, order=order, box_bc=BOX_DIRICHLET,
                               solution=sol, name=f"req{i}")
        out.append((float(t[i]), spec))
    return out


def star_interface_variant(n: int, step: int, seed: int = 2503, angle: float = 0.0) -> ProblemSpec:
    """The 1024^2 star interface problem with a seeded variant of its manufactured solution.

    Same geometry (rotated by ``angle``) and coefficients as ``star_interface_1024``;
    u- = sin(pi x + a) cos(pi y + b),
    u+ = exp(x + y)/4 + c (a, b, c drawn per step), so every step solves a new system.
    """
    rng = np.random.default_rng([seed, step])
    a, b = rng.uniform(0, 2 * np.pi, size=2)
    c = rng.uniform(-0.5, 0.5)
    pi = math.pi
    um = lambda X: np.sin(pi * X[..., 0] + a) * np.cos(pi * X[..., 1] + b)
    gm = lambda X: np.stack([pi * np.cos(pi * X[..., 0] + a) * np.cos(pi * X[..., 1] + b),
                             -pi * np.sin(pi * X[..., 0] + a) * np.sin(pi * X[..., 1] + b)], axis=-1)
    lm = lambda X: -2 * pi * pi * um(X)
    up = lambda X: np.exp(X[..., 0] + X[..., 1]) / 4 + c
    gp = lambda X: np.stack([np.exp(X[..., 0] + X[..., 1]) / 4] * 2, axis=-1)
    lp = lambda X: np.exp(X[..., 0] + X[..., 1]) / 2
    spec = star_interface_1024(n, phase=angle)
    spec.solution = Manufactured(up, gp, lp, um, gm, lm)
    spec.name = f"star_interface_{n}_step{step}"
    return spec
