"""Least-squares boundary interpolants (paper Sec. 2.1 and 2.2).

For a control point x_c and a phase sigma, the polynomial p_c of total degree
q = k - 1 fits, in the least-squares sense, u(x_c) and u at the points of the
set X_c (Sec. 2.1): the phase-sigma nodes inside a half-ellipse (half-ellipsoid
in 3D) on the sigma side of Gamma, minus the phase-sigma node closest to x_c.

Every quantity the operator needs is a row of the pseudo-inverse V^+ = R^-1 Q^T
of the Vandermonde matrix V (one QR per control point, as remarked after
Eq. 6):
  ghost row    p_c(x_g)            = v(xi_g)^T V^+ [u_c; u_X]          (Eq. 4)
  derivative   n . grad p_c(x_c)   = (1/h) sum_k n_k (V^+)_{e_k,:} [u_c; u_X]  (Eq. 5)

Readings (the half-ellipse sizes are defined in a companion paper that is not
reproduced here; parity unpinned against the paper's numbers):
  * semi-axes in units of h: normal a_n = q + 1, tangential a_t = q/2 + 1,
    grown by 1/2 up to three times while the fit is rank-deficient;
  * basis xi^alpha, xi = (x - x_c)/h, |alpha| <= q; unweighted least squares;
  * rank test: min|R_ii| >= 1e-8 max|R_ii| and at least M rows.
"""
from __future__ import annotations

import numpy as np

RANK_TOL = 1e-8
MAX_GROW = 3


def exponents(dim: int, q: int):
    """Monomial exponents of total degree <= q, graded (degree, then lexicographic)."""
    out = []
    for deg in range(q + 1):
        if dim == 2:
            for a in range(deg, -1, -1):
                out.append((a, deg - a))
        else:
            for a in range(deg, -1, -1):
                for b in range(deg - a, -1, -1):
                    out.append((a, b, deg - a - b))
    return out


def vandermonde(xi: np.ndarray, exps) -> np.ndarray:
    V = np.ones((xi.shape[0], len(exps)))
    for m, e in enumerate(exps):
        for k, p in enumerate(e):
            if p:
                V[:, m] *= xi[:, k] ** p
    return V


class FitError(Exception):
    pass


class Fit:
    """The interpolant of one control point on one side (phase) of Gamma.

    nodes   flat indices of X_c (the control point itself is row 0 of every row)
    ghost   (w, 1 + len(nodes)) coefficients of p_c at the w ghost nodes
    deriv   (1 + len(nodes),) coefficients of n . grad p_c(x_c)
            (n = normal out of Omega+, no beta factor)
    """

    def __init__(self, nodes, ghost, deriv, axes):
        self.nodes = nodes
        self.ghost = ghost
        self.deriv = deriv
        self.axes = axes


def build_fit(xc, normal, sigma_plus, plus, n, h, q, w, edge_axis, ghost_start, step):
    """Fit for control point ``xc`` on side ``sigma_plus`` (True = Omega+).

    ghost_start: multi-index of the first node past the crossing (away from the
    sigma side), step = +-1 along edge_axis; ghosts are ghost_start + k*step*e_axis,
    k = 0..w-1.
    """
    d = xc.shape[0]
    exps = exponents(d, q)
    M = len(exps)
    n_sigma = -normal if sigma_plus else normal          # points into phase sigma
    a_n, a_t = q + 1.0, q / 2.0 + 1.0
    xg = -1.0 + (np.arange(n) + 0.5) * h
    for grow in range(MAX_GROW + 1):
        an, at = a_n + 0.5 * grow, a_t + 0.5 * grow
        rad = int(np.ceil(an)) + 1
        c_idx = np.floor((xc + 1.0) / h - 0.5).astype(int)
        rng = [np.arange(max(0, c_idx[k] - rad), min(n, c_idx[k] + rad + 2)) for k in range(d)]
        I = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, d)
        in_phase = plus[tuple(I.T)] == sigma_plus
        I = I[in_phase]
        X = xg[I]
        rel = (X - xc) / h
        dist2 = np.sum(rel * rel, axis=1)
        flat = np.zeros(I.shape[0], dtype=np.int64)
        for k in range(d):
            flat += I[:, k] * n ** k
        # exclude the phase-sigma node closest to x_c (ties: smallest flat index)
        order = np.lexsort((flat, dist2))
        nearest = order[0]
        t = rel @ n_sigma
        tau2 = np.maximum(dist2 - t * t, 0.0)
        inside = (t >= 0.0) & (tau2 / (at * at) + t * t / (an * an) <= 1.0)
        inside[nearest] = False
        sel = np.nonzero(inside)[0]
        sel = sel[np.argsort(flat[sel], kind="stable")]
        nodes = flat[sel]
        xi = np.vstack([np.zeros((1, d)), rel[sel]])
        V = vandermonde(xi, exps)
        if V.shape[0] < M:
            continue
        Q, R = np.linalg.qr(V, mode="reduced")
        rd = np.abs(np.diag(R))
        if rd.min() < RANK_TOL * rd.max():
            continue
        # V^+ = R^-1 Q^T
        Vp = np.linalg.solve(R, Q.T)
        # ghost rows
        gnodes = np.array([ghost_start + kk * step * np.eye(d, dtype=int)[edge_axis] for kk in range(w)])
        xi_g = (-1.0 + (gnodes + 0.5) * h - xc) / h
        ghost = vandermonde(xi_g, exps) @ Vp
        # derivative row: grad of xi^{e_k} is e_k / h
        deriv = np.zeros(V.shape[0])
        for k in range(d):
            e = tuple(1 if m == k else 0 for m in range(d))
            deriv += normal[k] / h * Vp[exps.index(e)]
        return Fit(nodes, ghost, deriv, (an, at))
    raise FitError("least-squares fit is rank deficient after growing the region")
