"""The (n,k) immersed-interface Laplacian L_Omega u + L_Gamma u_Gamma (paper Sec. 2.3, Eq. 12).

At every unknown node i of phase sigma the operator is the dimension-split
centred stencil (Sec. 2.1)

    (L u)_i = beta_sigma / h^2  sum_axes sum_{j=-w..w} a_j  u~_{i + j e_axis}

applied to the extended function of Eq. 2: u~ = u at nodes of phase sigma, and
at nodes outside phase sigma the ghost value p_c(x) of the *first* control
point c met when walking from i along the axis (Eq. 4).  A node further along
the walk that is back in phase sigma uses u.

Control-point values (the affine data enter here):
  Dirichlet  u_c = ubar                                               (Eq. 1)
  Neumann    u_c = (qbar - sum_i s_i u_i) / s_c, s = beta+ * derivative row (Eqs. 5-6)
  interface  u+ = ubar + (j1 - beta- s-_c j0)/S,  u- = ubar + (j1 - beta+ s+_c j0)/S,
             ubar = -(beta+ sum s+_i u_i - beta- sum s-_i u_i)/S,
             S = beta+ s+_c - beta- s-_c                               (Eqs. 9-11)

Outer box (reading; the paper's domains are periodic or unbounded): with a
Dirichlet box the faces sit half a cell outside the first/last nodes, and
ghosts beyond a face come from the degree-q 1D polynomial through the face
value and q nodes of that grid line, skipping the node nearest the face (the
same exclusion the paper applies to its least-squares sets, Sec. 2.1); with
the nearest node kept, the 1D spectrum leaves the interior bound -sigma_max.

Unknowns: Omega+ nodes for boundary problems, every node for interface problems.
"""
from __future__ import annotations

import numpy as np

from workloads import DIRICHLET, NEUMANN, INTERFACE, BOX_DIRICHLET
from .fits import build_fit
from .geometry import Crossings, LevelSet, phase_plus
from .stencils import first_derivative, second_derivative


class GeometryError(Exception):
    pass


def box_ghost_weights(q: int, w: int) -> np.ndarray:
    """Lagrange weights (w, q+1): ghost k (1..w) from [face, node_2..node_{q+1}].

    Local coordinate in units of h from the face: node m (m = 1 nearest the face)
    at -(m - 1/2), face at 0, ghost k at +(k - 1/2); node 1 is skipped.
    """
    pts = np.array([0.0] + [-(m - 0.5) for m in range(2, q + 2)])
    W = np.zeros((w, q + 1))
    for k in range(1, w + 1):
        x = k - 0.5
        for a in range(q + 1):
            num, den = 1.0, 1.0
            for b in range(q + 1):
                if b != a:
                    num *= x - pts[b]
                    den *= pts[a] - pts[b]
            W[k - 1, a] = num / den
    return W


class IIMOperator:
    def __init__(self, spec, check_curvature=True, lazy=False):
        self.spec = spec
        self.n = n = spec.n
        self.d = d = spec.dim
        self.h = h = 2.0 / n
        self.order = spec.order
        self.w = w = spec.order // 2
        self.q = q = spec.order          # k = n + 1  ->  degree q = k - 1 = n
        self.bc = spec.bc
        self.beta_p, self.beta_m = spec.beta_plus, spec.beta_minus
        self.a = second_derivative(spec.order)          # a_{-w..w}
        self.ls = LevelSet(spec.geometry)
        self.plus = phase_plus(self.ls, n)
        self.cross = Crossings(self.ls, n, self.plus)
        if check_curvature and self.cross.count and np.max(self.cross.kappa) * h >= 0.25:
            raise GeometryError("curvature condition |kappa h| < 1/4 violated")
        self.unknown = np.ones_like(self.plus) if spec.bc == INTERFACE else self.plus.copy()
        self.box_w = box_ghost_weights(q, w) if spec.box_bc == BOX_DIRICHLET else None
        self._check_box()
        self.fits = {}
        if not lazy:
            self._build_records()
            self._build_fits()

    # ------------------------------------------------------------------ records
    def _check_box(self):
        n, d = self.n, self.d
        margin = self.q + 1 + self.w
        near = np.zeros_like(self.plus)
        for ax in range(d):
            sl = [slice(None)] * d
            sl[ax] = slice(0, margin)
            near[tuple(sl)] = True
            sl[ax] = slice(n - margin, n)
            near[tuple(sl)] = True
        if self.spec.box_bc == BOX_DIRICHLET:
            if not np.all(self.plus[near]):
                raise GeometryError("body too close to the outer box")
        else:
            w_near = np.zeros_like(self.plus)
            for ax in range(d):
                sl = [slice(None)] * d
                sl[ax] = slice(0, self.w)
                w_near[tuple(sl)] = True
                sl[ax] = slice(n - self.w, n)
                w_near[tuple(sl)] = True
            if np.any(self.unknown[w_near]):
                raise GeometryError("solved region reaches the box but the box has no condition")

    def _build_records(self):
        """For every unknown node, axis and direction: the first event of the walk.

        iim records: (node flat, axis, dir, jstar, crossing id, side_plus)
        box records: (node flat, axis, dir, jstar)
        """
        n, d, w = self.n, self.d, self.w
        idx = np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"), axis=-1)
        self.iim_rec, self.box_rec = [], []
        unk = self.unknown
        for ax in range(d):
            for s in (-1, 1):
                done = ~unk.copy()
                for j in range(1, w + 1):
                    pos = idx[..., ax] + j * s
                    inb = (pos >= 0) & (pos < n)
                    nb = idx.copy()
                    nb[..., ax] = np.clip(pos, 0, n - 1)
                    nb_plus = self.plus[tuple(np.moveaxis(nb, -1, 0))]
                    out_box = ~inb & ~done
                    out_phase = inb & (nb_plus != self.plus) & ~done
                    for m in np.argwhere(out_box):
                        self.box_rec.append((self._flat(m), ax, s, j))
                    for m in np.argwhere(out_phase):
                        # edge between node at offset j-1 and j
                        a = m.copy()
                        a[ax] += (j - 1) * s
                        b = m.copy()
                        b[ax] += j * s
                        lower = a if s > 0 else b
                        c = self.cross.lookup[(ax, self._flat(lower))]
                        self.iim_rec.append((self._flat(m), ax, s, j, c, bool(self.plus[tuple(m)])))
                    done = done | out_box | out_phase

    def _flat(self, m):
        return int(sum(int(m[k]) * self.n ** k for k in range(self.d)))

    def _unflat(self, f):
        return np.array(np.unravel_index(f, (self.n,) * self.d, order="F"))

    def _build_fits(self):
        """One fit per (crossing, side) that some record needs; interface needs both sides."""
        need = set()
        for (_, _, _, _, c, side) in self.iim_rec:
            need.add((c, side))
            if self.bc == INTERFACE:
                need.add((c, not side))
        self.fits = {}
        for (c, side) in sorted(need):
            self._fit(c, side)

    def _fit(self, c, side):
        """The fit of crossing c on one side (built on first use)."""
        key = (c, side)
        if key not in self.fits:
            cr = self.cross
            ax = int(cr.axis[c])
            lo = cr.lo_idx[c]
            hi = lo.copy()
            hi[ax] += 1
            lo_side = bool(cr.lo_plus[c])
            if lo_side == side:          # sigma-side node is the lower one: ghosts go up
                start, step = hi, 1
            else:
                start, step = lo, -1
            self.fits[key] = build_fit(cr.x[c], cr.normal[c], side, self.plus, self.n, self.h,
                                       self.q, self.w, ax, start, step)
        return self.fits[key]

    # ------------------------------------------------------------------ apply
    def control_values(self, u_flat, data, include_data):
        """u_c for every needed (crossing, side)."""
        vals = {}
        bp, bm = self.beta_p, self.beta_m
        g = data.get("g") if include_data else None
        j0 = data.get("j0") if include_data else None
        j1 = data.get("j1") if include_data else None
        crossings = sorted({c for (c, _) in self.fits})
        for c in crossings:
            if self.bc == DIRICHLET:
                vals[(c, True)] = g[c] if include_data else 0.0
            elif self.bc == NEUMANN:
                f = self.fits[(c, True)]
                s = bp * f.deriv
                rhs = (g[c] if include_data else 0.0) - s[1:] @ u_flat[f.nodes]
                vals[(c, True)] = rhs / s[0]
            else:
                fp, fm = self.fits[(c, True)], self.fits[(c, False)]
                Sden = bp * fp.deriv[0] - bm * fm.deriv[0]
                ubar = -(bp * (fp.deriv[1:] @ u_flat[fp.nodes]) - bm * (fm.deriv[1:] @ u_flat[fm.nodes])) / Sden
                up, um = ubar, ubar
                if include_data:
                    up = ubar + (j1[c] - bm * fm.deriv[0] * j0[c]) / Sden
                    um = ubar + (j1[c] - bp * fp.deriv[0] * j0[c]) / Sden
                vals[(c, True)] = up
                vals[(c, False)] = um
        return vals

    def ghost_values(self, u_flat, data, include_data):
        cv = self.control_values(u_flat, data, include_data)
        G = {}
        for key, f in self.fits.items():
            G[key] = f.ghost[:, 0] * cv[key] + f.ghost[:, 1:] @ u_flat[f.nodes]
        return G

    def apply(self, u_flat, data=None, include_data=False):
        """w = L_Omega u (+ L_Gamma u_Gamma if include_data); zero at non-unknowns."""
        n, d, w = self.n, self.d, self.w
        data = data or {}
        u = u_flat.reshape((n,) * d, order="F")
        acc = np.zeros((n,) * d)
        a = self.a
        for ax in range(d):
            acc += a[w] * u
            for s in (-1, 1):
                for j in range(1, w + 1):
                    shifted = np.zeros((n,) * d)
                    same = np.zeros((n,) * d, dtype=bool)
                    src = [slice(None)] * d
                    dst = [slice(None)] * d
                    if s > 0:
                        src[ax], dst[ax] = slice(j, n), slice(0, n - j)
                    else:
                        src[ax], dst[ax] = slice(0, n - j), slice(j, n)
                    shifted[tuple(dst)] = u[tuple(src)]
                    same[tuple(dst)] = self.plus[tuple(src)] == self.plus[tuple(dst)]
                    acc += a[w + j * s] * np.where(same, shifted, 0.0)
        acc_flat = acc.ravel(order="F")
        # ghost contributions of the first control point along each walk
        G = self.ghost_values(u_flat, data, include_data)
        plus_flat = self.plus.ravel(order="F")
        for (node, ax, s, jstar, c, side) in self.iim_rec:
            m = self._unflat(node)
            for j in range(jstar, w + 1):
                p = m.copy()
                p[ax] += j * s
                if 0 <= p[ax] < n and self.plus[tuple(p)] == side:
                    continue                      # back in phase sigma: uses u
                acc_flat[node] += a[w + j * s] * G[(c, side)][j - jstar]
        if self.box_rec:
            bd = data.get("box") if include_data else None
            for (node, ax, s, jstar) in self.box_rec:
                m = self._unflat(node)
                line_nodes = []
                for mm in range(2, self.q + 2):
                    p = m.copy()
                    p[ax] = n - mm if s > 0 else mm - 1
                    line_nodes.append(self._flat(p))
                vals = u_flat[line_nodes]
                face = 0.0
                if include_data:
                    face = bd[self._box_index(m, ax, s)]
                for j in range(jstar, w + 1):
                    k = j - jstar + 1
                    gval = self.box_w[k - 1, 0] * face + self.box_w[k - 1, 1:] @ vals
                    acc_flat[node] += a[w + j * s] * gval
        beta = np.where(plus_flat, self.beta_p, self.beta_m)
        out = beta * acc_flat / (self.h * self.h)
        out[~self.unknown.ravel(order="F")] = 0.0
        return out

    def boundary_values(self, u_flat, data):
        """The boundary quantity the data do not prescribe, at every control point
        (canonical order), Sec. 2.4: Dirichlet -> n . grad u(x_c) from the fit's derivative
        row (Eq. 5 without beta; n out of Omega+); Neumann -> u(x_c) from Eq. 6."""
        if self.bc == INTERFACE:
            raise ValueError("boundary values are defined for boundary problems")
        K = self.cross.count
        out = np.zeros(K)
        if self.bc == DIRICHLET:
            g = data["g"]
            for c in range(K):
                f = self.fits[(c, True)] if (c, True) in self.fits else self._fit(c, True)
                out[c] = f.deriv[0] * g[c] + f.deriv[1:] @ u_flat[f.nodes]
            return out
        for c in range(K):
            if (c, True) not in self.fits:
                self._fit(c, True)
        cv = self.control_values(u_flat, data, True)
        for c in range(K):
            out[c] = cv[(c, True)]
        return out

    def gradient(self, u_flat, data=None, include_data=True):
        """grad u at every unknown node, shape (d, n^d): the centred first-derivative
        stencil of the scheme's order applied to the same extension of u as the Laplacian
        (u in phase, the fit's ghost values past the first crossing, box ghosts), Sec. 2.4."""
        n, d, w = self.n, self.d, self.w
        data = data or {}
        b = first_derivative(self.order)
        u = u_flat.reshape((n,) * d, order="F")
        G = self.ghost_values(u_flat, data, include_data)
        out = np.zeros((d, n ** d))
        for ax in range(d):
            acc = np.zeros((n,) * d)
            for s in (-1, 1):
                for j in range(1, w + 1):
                    shifted = np.zeros((n,) * d)
                    same = np.zeros((n,) * d, dtype=bool)
                    src = [slice(None)] * d
                    dst = [slice(None)] * d
                    if s > 0:
                        src[ax], dst[ax] = slice(j, n), slice(0, n - j)
                    else:
                        src[ax], dst[ax] = slice(0, n - j), slice(j, n)
                    shifted[tuple(dst)] = u[tuple(src)]
                    same[tuple(dst)] = self.plus[tuple(src)] == self.plus[tuple(dst)]
                    acc += b[w + j * s] * np.where(same, shifted, 0.0)
            acc_flat = acc.ravel(order="F")
            for (node, rax, s, jstar, c, side) in self.iim_rec:
                if rax != ax:
                    continue
                m = self._unflat(node)
                for j in range(jstar, w + 1):
                    p = m.copy()
                    p[ax] += j * s
                    if 0 <= p[ax] < n and self.plus[tuple(p)] == side:
                        continue
                    acc_flat[node] += b[w + j * s] * G[(c, side)][j - jstar]
            if self.box_rec:
                bd = data.get("box") if include_data else None
                for (node, rax, s, jstar) in self.box_rec:
                    if rax != ax:
                        continue
                    m = self._unflat(node)
                    line_nodes = []
                    for mm in range(2, self.q + 2):
                        p = m.copy()
                        p[ax] = n - mm if s > 0 else mm - 1
                        line_nodes.append(self._flat(p))
                    vals = u_flat[line_nodes]
                    face = bd[self._box_index(m, ax, s)] if include_data else 0.0
                    for j in range(jstar, w + 1):
                        k = j - jstar + 1
                        acc_flat[node] += b[w + j * s] * (self.box_w[k - 1, 0] * face + self.box_w[k - 1, 1:] @ vals)
            acc_flat = acc_flat / self.h
            acc_flat[~self.unknown.ravel(order="F")] = 0.0
            out[ax] = acc_flat
        return out

    def apply_at(self, u_flat, nodes, data=None, include_data=False):
        """(L u)_i (+ data) at the given flat node indices only, with the same rules
        as ``apply``; fits are built on first use, so this serves grids far too large
        for the full oracle."""
        n, d, w, a = self.n, self.d, self.w, self.a
        data = data or {}
        plus = self.plus
        out = np.zeros(len(nodes))
        for t, node in enumerate(nodes):
            m = self._unflat(int(node))
            side = bool(plus[tuple(m)])
            if not self.unknown[tuple(m)]:
                continue
            acc = d * a[w] * u_flat[node]
            for ax in range(d):
                for s in (-1, 1):
                    event = None
                    for j in range(1, w + 1):
                        p = m.copy()
                        p[ax] += j * s
                        inb = 0 <= p[ax] < n
                        if event is None and (not inb or bool(plus[tuple(p)]) != side):
                            event = (j, inb)
                        if inb and bool(plus[tuple(p)]) == side:
                            acc += a[w + j * s] * u_flat[self._flat(p)]
                    if event is None:
                        continue
                    jstar, inb = event
                    if inb:
                        # crossing on the edge between offsets jstar-1 and jstar
                        pa = m.copy()
                        pa[ax] += (jstar - 1) * s
                        pb = m.copy()
                        pb[ax] += jstar * s
                        lower = pa if s > 0 else pb
                        c = self.cross.lookup[(ax, self._flat(lower))]
                        G = self._ghosts_of(c, side, u_flat, data, include_data)
                        for j in range(jstar, w + 1):
                            p = m.copy()
                            p[ax] += j * s
                            if 0 <= p[ax] < n and bool(plus[tuple(p)]) == side:
                                continue
                            acc += a[w + j * s] * G[j - jstar]
                    else:
                        line = []
                        for mm in range(2, self.q + 2):
                            p = m.copy()
                            p[ax] = n - mm if s > 0 else mm - 1
                            line.append(self._flat(p))
                        face = data["box"][self._box_index(m, ax, s)] if include_data else 0.0
                        for j in range(jstar, w + 1):
                            k = j - jstar + 1
                            acc += a[w + j * s] * (self.box_w[k - 1, 0] * face + self.box_w[k - 1, 1:] @ u_flat[line])
            beta = self.beta_p if side else self.beta_m
            out[t] = beta * acc / (self.h * self.h)
        return out

    def _ghosts_of(self, c, side, u_flat, data, include_data):
        """Ghost values of crossing c on one side (Eqs. 4-6, 9-11)."""
        bp, bm = self.beta_p, self.beta_m
        f = self._fit(c, side)
        if self.bc == DIRICHLET:
            uc = data["g"][c] if include_data else 0.0
        elif self.bc == NEUMANN:
            sv = bp * f.deriv
            uc = ((data["g"][c] if include_data else 0.0) - sv[1:] @ u_flat[f.nodes]) / sv[0]
        else:
            fp, fm = self._fit(c, True), self._fit(c, False)
            Sden = bp * fp.deriv[0] - bm * fm.deriv[0]
            ubar = -(bp * (fp.deriv[1:] @ u_flat[fp.nodes]) - bm * (fm.deriv[1:] @ u_flat[fm.nodes])) / Sden
            uc = ubar
            if include_data:
                if side:
                    uc = ubar + (data["j1"][c] - bm * fm.deriv[0] * data["j0"][c]) / Sden
                else:
                    uc = ubar + (data["j1"][c] - bp * fp.deriv[0] * data["j0"][c]) / Sden
        return f.ghost[:, 0] * uc + f.ghost[:, 1:] @ u_flat[f.nodes]

    def _box_index(self, m, ax, s):
        """Index into the box data array (faces -x0,+x0,-x1,+x1,...; others flat)."""
        n, d = self.n, self.d
        per = n ** (d - 1)
        face = 2 * ax + (1 if s > 0 else 0)
        others = [k for k in range(d) if k != ax]
        f = 0
        for r, k in enumerate(others):
            f += int(m[k]) * n ** r
        return face * per + f

    # ------------------------------------------------------------------ data term
    def rhs(self, f_flat, data):
        """b = f - L_Gamma u_Gamma = f - apply(0, data)."""
        zero = np.zeros(self.n ** self.d)
        b = f_flat - self.apply(zero, data, include_data=True)
        b[~self.unknown.ravel(order="F")] = 0.0
        return b

    def control_points(self):
        return self.cross.x, self.cross.normal
