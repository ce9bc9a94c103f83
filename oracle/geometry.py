"""Geometry for the oracle: level set phi, crossings, normals, curvature.

Paper Sec. 2.1: a *control point* x_c is the intersection of a 1D stencil
(a grid line) with the surface Gamma; the surface must satisfy the curvature
condition |kappa dx| < 1/4 (Eq. 3), kappa being the largest principal
curvature.

Conventions (paper Eqs. 1, 8): Omega+ = {phi >= 0}; the normal n points out of
Omega+ towards Omega-, so n = -grad(phi)/|grad(phi)|.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import (CIRCLE, ELLIPSE, STAR, SPHERE, ELLIPSOID, PERTURBED_SPHERE, PERTURB_SCALE, FOURIER,
                       LEVELSET_GRID)

# D_k = prod_{j != k} (k - j) over the six stencil nodes 0..5 of the degree-5 interpolant
_LAG_DEN = np.array([-120.0, 24.0, -12.0, 12.0, -24.0, 120.0])


class LevelSet:
    """phi(x) for an analytic body, a polar Fourier curve or a level set given at the grid's
    nodes; ``g`` is negative inside the body.

    FOURIER: g = |x - c| - r(theta), r = a0 + sum_k (a_k cos k theta + b_k sin k theta).
    LEVELSET_GRID: g is the level set given at the nodes of the problem's grid and, between
    them, the tensor product of the degree-5 Lagrange interpolants through the six nodes
    around the point along each axis (the six nodes shifted inwards at the grid's edge).
    """

    def __init__(self, geometry):
        self.geom = geometry
        self.kind = geometry.kind
        self.p = tuple(float(v) for v in geometry.params)
        self.sign = -1.0 if geometry.plus_inside else 1.0   # phi = sign * g
        self.dim = geometry.dim
        if self.kind == FOURIER:
            c = np.asarray(geometry.coef, dtype=float)
            self.a0, self.fa, self.fb = c[0], c[1::2], c[2::2]
        if self.kind == LEVELSET_GRID:
            self.values = np.asarray(geometry.values, dtype=float)
            self.gn = self.values.shape[0]
            self.gh = 2.0 / self.gn

    # polar Fourier curve ------------------------------------------------------------
    def _fourier(self, th):
        """r, r', r'' of the Fourier curve at angles th."""
        k = np.arange(1, self.fa.size + 1)
        kt = th[..., None] * k
        ck, sk = np.cos(kt), np.sin(kt)
        r = self.a0 + np.sum(self.fa * ck + self.fb * sk, axis=-1)
        r1 = np.sum(k * (self.fb * ck - self.fa * sk), axis=-1)
        r2 = -np.sum(k * k * (self.fa * ck + self.fb * sk), axis=-1)
        return r, r1, r2

    # level set given at the nodes ----------------------------------------------------
    def _lagrange(self, x, order):
        """First stencil node s and the weights of the value (order 0), first (1) or second
        (2) derivative along one axis for coordinates x: the derivatives of the Lagrange
        basis l_k(t) = prod_{j != k} (t - j) / D_k, t = (x - x_s) / h, over the six nodes
        from two below the point's cell.  A coordinate within 1e-9 h of node m counts as
        that node: the stencil starts at m - 2 and t is the exact integer m - s, so that the
        interpolant returns the given value there (the two stencils holding a node agree on
        its value but not on its derivatives, so the choice must not depend on rounding)."""
        n, h = self.gn, self.gh
        tc = (x + 1.0) / h - 0.5
        m = np.floor(tc + 0.5).astype(np.int64)
        at_node = np.abs(tc - m) <= 1e-9
        s = np.clip(np.where(at_node, m, np.floor(tc).astype(np.int64)) - 2, 0, n - 6)
        t = np.where(at_node, (m - s).astype(float), tc - s)
        d = t[..., None] - np.arange(6.0)
        w = np.zeros(x.shape + (6,))
        for k in range(6):
            others = [j for j in range(6) if j != k]
            if order == 0:
                acc = np.prod(d[..., others], axis=-1)
            elif order == 1:
                acc = sum(np.prod(d[..., [l for l in others if l != j]], axis=-1) for j in others)
            else:
                acc = sum(np.prod(d[..., [q for q in others if q not in (j, l)]], axis=-1)
                          for j in others for l in others if l != j)
            w[..., k] = acc / (_LAG_DEN[k] * h ** order)
        return s, w

    def _grid_eval(self, X, orders):
        """Tensor-product interpolant (orders: derivative order along each axis)."""
        d = self.dim
        flat = X.reshape(-1, d)
        sw = [self._lagrange(flat[:, a], orders[a]) for a in range(d)]
        r6 = np.arange(6)
        if d == 2:
            (s0, w0), (s1, w1) = sw
            V = self.values[(s0[:, None, None] + r6[None, :, None]), (s1[:, None, None] + r6[None, None, :])]
            out = np.einsum("pi,pj,pij->p", w0, w1, V)
        else:
            (s0, w0), (s1, w1), (s2, w2) = sw
            V = self.values[(s0[:, None, None, None] + r6[None, :, None, None]),
                            (s1[:, None, None, None] + r6[None, None, :, None]),
                            (s2[:, None, None, None] + r6[None, None, None, :])]
            out = np.einsum("pi,pj,pk,pijk->p", w0, w1, w2, V)
        return out.reshape(X.shape[:-1])

    # body function g and its gradient / Hessian -------------------------------------
    def g(self, X):
        p = self.p
        if self.kind == CIRCLE:
            return np.hypot(X[..., 0] - p[0], X[..., 1] - p[1]) - p[2]
        if self.kind == SPHERE:
            d = X - np.array(p[:3])
            return np.sqrt(np.sum(d * d, axis=-1)) - p[3]
        if self.kind == ELLIPSE:
            y = self._ellipse_local(X)
            return (y[..., 0] / p[2]) ** 2 + (y[..., 1] / p[3]) ** 2 - 1.0
        if self.kind == ELLIPSOID:
            d = X - np.array(p[:3])
            return np.sum((d / np.array(p[3:6])) ** 2, axis=-1) - 1.0
        if self.kind == STAR:
            dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
            rho = np.hypot(dx, dy)
            th = np.arctan2(dy, dx)
            return rho - (p[2] + p[3] * np.sin(p[4] * th + p[5]))
        if self.kind == FOURIER:
            dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
            r, _, _ = self._fourier(np.arctan2(dy, dx))
            return np.hypot(dx, dy) - r
        if self.kind == LEVELSET_GRID:
            return self._grid_eval(X, [0] * self.dim)
        if self.kind == PERTURBED_SPHERE:
            # g = r - rho0 - rho1 c Q(d) / r^3 with d = x - centre, r = |d|, Q = (dx^2 - dy^2) dz:
            # Q / r^3 is the harmonic (e_x^2 - e_y^2) e_z of the direction e = d / r
            # at the centre itself (r = 0) the direction is undefined: the harmonic term is 0
            d = X - np.array(p[:3])
            r = np.sqrt(np.sum(d * d, axis=-1))
            Q = (d[..., 0] ** 2 - d[..., 1] ** 2) * d[..., 2]
            Y = np.divide(Q, r ** 3, out=np.zeros_like(r), where=r > 0)
            return r - p[3] - p[4] * PERTURB_SCALE * Y
        raise ValueError("unknown geometry kind")

    def phi(self, X):
        return self.sign * self.g(X)

    def grad_g(self, X):
        p = self.p
        if self.kind in (CIRCLE, SPHERE):
            c = np.array(p[:self.dim])
            d = X - c
            return d / np.sqrt(np.sum(d * d, axis=-1))[..., None]
        if self.kind == ELLIPSE:
            y = self._ellipse_local(X)
            gy = np.stack([2 * y[..., 0] / p[2] ** 2, 2 * y[..., 1] / p[3] ** 2], axis=-1)
            c, s = math.cos(p[4]), math.sin(p[4])
            # x = c0 + R y with R = [[c,-s],[s,c]]  ->  grad_x = R grad_y
            return np.stack([c * gy[..., 0] - s * gy[..., 1], s * gy[..., 0] + c * gy[..., 1]], axis=-1)
        if self.kind == ELLIPSOID:
            d = X - np.array(p[:3])
            return 2 * d / np.array(p[3:6]) ** 2
        if self.kind == STAR:
            dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
            rho = np.hypot(dx, dy)
            th = np.arctan2(dy, dx)
            rp = p[3] * p[4] * np.cos(p[4] * th + p[5])          # r'(theta)
            er = np.stack([dx / rho, dy / rho], axis=-1)
            et = np.stack([-dy / rho, dx / rho], axis=-1)
            return er - (rp / rho)[..., None] * et
        if self.kind == FOURIER:
            dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
            rho = np.hypot(dx, dy)
            _, rp, _ = self._fourier(np.arctan2(dy, dx))
            er = np.stack([dx / rho, dy / rho], axis=-1)
            et = np.stack([-dy / rho, dx / rho], axis=-1)
            return er - (rp / rho)[..., None] * et
        if self.kind == LEVELSET_GRID:
            return np.stack([self._grid_eval(X, [1 if b == a else 0 for b in range(self.dim)])
                             for a in range(self.dim)], axis=-1)
        if self.kind == PERTURBED_SPHERE:
            d = X - np.array(p[:3])
            r = np.sqrt(np.sum(d * d, axis=-1))[..., None]
            Q = ((d[..., 0] ** 2 - d[..., 1] ** 2) * d[..., 2])[..., None]
            gQ = np.stack([2 * d[..., 0] * d[..., 2], -2 * d[..., 1] * d[..., 2],
                           d[..., 0] ** 2 - d[..., 1] ** 2], axis=-1)
            # grad (Q r^-3) = grad Q r^-3 - 3 Q d r^-5
            return d / r - p[4] * PERTURB_SCALE * (gQ / r ** 3 - 3 * Q * d / r ** 5)
        raise ValueError

    def normal(self, X):
        """Unit normal pointing out of Omega+ (towards Omega-)."""
        gphi = self.sign * self.grad_g(X)
        return -gphi / np.linalg.norm(gphi, axis=-1, keepdims=True)

    def curvature(self, X):
        """Largest |principal curvature| of the level surface through X."""
        p = self.p
        if self.kind == CIRCLE:
            return np.full(X.shape[:-1], 1.0 / p[2])
        if self.kind == SPHERE:
            return np.full(X.shape[:-1], 1.0 / p[3])
        if self.kind == STAR:
            dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
            th = np.arctan2(dy, dx)
            r = p[2] + p[3] * np.sin(p[4] * th + p[5])
            r1 = p[3] * p[4] * np.cos(p[4] * th + p[5])
            r2 = -p[3] * p[4] ** 2 * np.sin(p[4] * th + p[5])
            # curvature of the polar curve r(theta)
            return np.abs(r * r + 2 * r1 * r1 - r * r2) / (r * r + r1 * r1) ** 1.5
        if self.kind == FOURIER:
            dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
            r, r1, r2 = self._fourier(np.arctan2(dy, dx))
            return np.abs(r * r + 2 * r1 * r1 - r * r2) / (r * r + r1 * r1) ** 1.5
        # shape operator P H P / |grad g| on the tangent space (H: Hessian of g)
        if self.kind == ELLIPSE:
            c, s = math.cos(p[4]), math.sin(p[4])
            R = np.array([[c, -s], [s, c]])
            H = np.broadcast_to(R @ np.diag([2 / p[2] ** 2, 2 / p[3] ** 2]) @ R.T, X.shape[:-1] + (2, 2))
        elif self.kind == ELLIPSOID:
            H = np.broadcast_to(np.diag(2 / np.array(p[3:6]) ** 2), X.shape[:-1] + (3, 3))
        else:
            H = self.hess_g(X)
        G = self.grad_g(X)
        gn = np.linalg.norm(G, axis=-1)
        n = G / gn[..., None]
        out = np.zeros(X.shape[:-1])
        flat_n = n.reshape(-1, self.dim)
        flat_g = gn.reshape(-1)
        flat_H = np.reshape(H, (-1, self.dim, self.dim))
        res = out.reshape(-1)
        for k in range(flat_n.shape[0]):
            P = np.eye(self.dim) - np.outer(flat_n[k], flat_n[k])
            S = P @ flat_H[k] @ P / flat_g[k]
            res[k] = np.max(np.abs(np.linalg.eigvalsh(S)))
        return res.reshape(X.shape[:-1])

    def hess_g(self, X):
        """Hessian of g for PERTURBED_SPHERE and LEVELSET_GRID; for the perturbed sphere:
        (I - e e^T) / r - rho1 c [Hess Q r^-3 - 3 r^-5 (grad Q d^T + d grad Q^T)
                                  + Q (-3 r^-5 I + 15 r^-7 d d^T)]."""
        p = self.p
        if self.kind == LEVELSET_GRID:
            d = self.dim
            H = np.zeros(X.shape[:-1] + (d, d))
            for a in range(d):
                for b in range(a, d):
                    orders = [0] * d
                    orders[a] += 1
                    orders[b] += 1
                    H[..., a, b] = H[..., b, a] = self._grid_eval(X, orders)
            return H
        if self.kind != PERTURBED_SPHERE:
            raise ValueError("hess_g: perturbed sphere or grid level set only")
        d = X - np.array(p[:3])
        r = np.sqrt(np.sum(d * d, axis=-1))[..., None, None]
        dd = d[..., :, None] * d[..., None, :]
        I = np.eye(3)
        Q = ((d[..., 0] ** 2 - d[..., 1] ** 2) * d[..., 2])[..., None, None]
        gQ = np.stack([2 * d[..., 0] * d[..., 2], -2 * d[..., 1] * d[..., 2],
                       d[..., 0] ** 2 - d[..., 1] ** 2], axis=-1)
        HQ = np.zeros(X.shape[:-1] + (3, 3))
        HQ[..., 0, 0] = 2 * d[..., 2]
        HQ[..., 1, 1] = -2 * d[..., 2]
        HQ[..., 0, 2] = HQ[..., 2, 0] = 2 * d[..., 0]
        HQ[..., 1, 2] = HQ[..., 2, 1] = -2 * d[..., 1]
        cross = gQ[..., :, None] * d[..., None, :] + d[..., :, None] * gQ[..., None, :]
        Hr = (I - dd / r ** 2) / r
        Hp = HQ / r ** 3 - 3 * cross / r ** 5 + Q * (-3 * I / r ** 5 + 15 * dd / r ** 7)
        return Hr - p[4] * PERTURB_SCALE * Hp

    def _ellipse_local(self, X):
        p = self.p
        c, s = math.cos(p[4]), math.sin(p[4])
        dx, dy = X[..., 0] - p[0], X[..., 1] - p[1]
        return np.stack([c * dx + s * dy, -s * dx + c * dy], axis=-1)


def grid_x(n):
    """Cell-centred node coordinates along one axis of [-1,1]: -1 + (i+1/2) h."""
    h = 2.0 / n
    return -1.0 + (np.arange(n) + 0.5) * h


def phase_plus(ls: LevelSet, n: int) -> np.ndarray:
    """Boolean grid, True on Omega+ = {phi >= 0} (a node with phi == 0 is in Omega+)."""
    x = grid_x(n)
    X = np.stack(np.meshgrid(*([x] * ls.dim), indexing="ij"), axis=-1)
    return ls.phi(X) >= 0.0


class Crossings:
    """Control points: one per axis-aligned grid edge whose end nodes differ in phase.

    Canonical order: by axis, then by the flat index (i0 fastest) of the lower
    node of the edge.  Fields (K = number of crossings):
      axis[K], lo[K] (flat index of the lower node), t[K] (fraction of h from
      the lower node), x[K,d], normal[K,d] (out of Omega+), kappa[K],
      lo_plus[K] (True if the lower node is in Omega+).
    """

    def __init__(self, ls: LevelSet, n: int, plus: np.ndarray):
        d = ls.dim
        h = 2.0 / n
        x = grid_x(n)
        axes, los, ts, lo_plus = [], [], [], []
        for ax in range(d):
            sl_lo = [slice(None)] * d
            sl_hi = [slice(None)] * d
            sl_lo[ax] = slice(0, n - 1)
            sl_hi[ax] = slice(1, n)
            a, b = plus[tuple(sl_lo)], plus[tuple(sl_hi)]
            cut = a != b
            idx = np.argwhere(cut)                   # lower-node multi-indices, C order
            if idx.size == 0:
                continue
            flat = np.zeros(idx.shape[0], dtype=np.int64)
            for k in range(d):
                flat += idx[:, k] * n ** k
            order = np.argsort(flat, kind="stable")
            idx, flat = idx[order], flat[order]
            P0 = x[idx]                              # lower node coordinates
            t = self._bisect(ls, P0, ax, h)
            axes.append(np.full(idx.shape[0], ax))
            los.append(flat)
            ts.append(t)
            lo_plus.append(a[tuple(idx.T)])
        if axes:
            self.axis = np.concatenate(axes)
            self.lo = np.concatenate(los)
            self.t = np.concatenate(ts)
            self.lo_plus = np.concatenate(lo_plus)
        else:
            self.axis = np.zeros(0, dtype=np.int64)
            self.lo = np.zeros(0, dtype=np.int64)
            self.t = np.zeros(0)
            self.lo_plus = np.zeros(0, dtype=bool)
        K = self.axis.size
        self.n, self.dim, self.h = n, d, h
        self.count = K
        self.lo_idx = np.stack(np.unravel_index(self.lo, (n,) * d, order="F"), axis=-1) if K else np.zeros((0, d), dtype=np.int64)
        X = x[self.lo_idx].astype(float) if K else np.zeros((0, d))
        if K:
            X[np.arange(K), self.axis] += self.t * h
        self.x = X
        self.normal = ls.normal(X) if K else np.zeros((0, d))
        self.kappa = ls.curvature(X) if K else np.zeros(0)
        # lookup: (axis, lower flat index) -> crossing id
        self.lookup = {(int(a), int(l)): k for k, (a, l) in enumerate(zip(self.axis, self.lo))}

    @staticmethod
    def _bisect(ls, P0, ax, h):
        """Root of phi on each edge [P0, P0 + h e_ax] by bisection (60 halvings)."""
        lo = np.zeros(P0.shape[0])
        hi = np.ones(P0.shape[0])

        def f(t):
            X = P0.astype(float).copy()
            X[:, ax] += t * h
            return ls.phi(X)

        f_lo = f(lo)
        s_lo = f_lo >= 0.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            s_mid = f(mid) >= 0.0
            same = s_mid == s_lo
            lo = np.where(same, mid, lo)
            hi = np.where(same, hi, mid)
        return 0.5 * (lo + hi)
