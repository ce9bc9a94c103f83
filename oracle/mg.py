"""Geometric multigrid V-cycle for the Shortley-Weller operators (paper Sec. 3.3).

Sec. 3.3: coarsen by two, red-black Gauss-Seidel smoothing, linear
interpolation (coarse to fine), restriction, all transfers on the full grid
with zero values outside the problem domain; Neumann problems replace the
interpolation by the average of the in-domain coarse neighbours (zero if there
is none); interface problems run multigrid on lap(u) = f/beta per phase; a
direct solve on the coarsest level.

Readings for the cell-centred grids used here:
  * restriction: mean of the 2^d children (cell-centred counterpart of the
    half-weighted restriction), fine values outside the domain count as 0;
  * interpolation: bi/trilinear cell-centred weights (3/4, 1/4 per axis) over
    the 2^d nearest coarse nodes, coarse values outside the domain or the box
    count as 0; Neumann: unweighted mean of those neighbours that are unknowns;
  * colouring: red = even index sum, red first, in both pre and post smoothing;
  * levels: coarsen while N is even and N/2 >= 8 (2D) or >= 4 (3D); dense LU on
    the coarsest level (Sec. 3.3 uses a direct coarse solve at N = 8 in 2D).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from workloads import BOX_NONE, NEUMANN
from .sw import SWLevel


def level_sizes(n: int, dim: int):
    cmin = 8 if dim == 2 else 4
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] // 2 >= cmin:
        sizes.append(sizes[-1] // 2)
    return sizes


class Multigrid:
    def __init__(self, ls, n, bc, box_bc, beta_p, beta_m, nu1=2, nu2=2, gamma=1):
        self.dim = ls.dim
        self.bc = bc
        self.nu1, self.nu2 = nu1, nu2
        self.gamma = gamma                   # 1: V-cycle, 2: W-cycle
        self.sizes = level_sizes(n, ls.dim)
        self.levels = [SWLevel(ls, m, bc, box_bc, beta_p, beta_m) for m in self.sizes]
        self.beta_p, self.beta_m = beta_p, beta_m
        c = self.levels[-1]
        self.c_unk = np.nonzero(c.unk_flat)[0]
        Ac = c.A[self.c_unk][:, self.c_unk].toarray()
        # pure Neumann (no box): the coarse operator annihilates constants; the coarsest
        # level solves the augmented system [A 1; 1^T 0] (Sec. 2.3 augmentation)
        self.augmented = bc == NEUMANN and box_bc == BOX_NONE
        if self.augmented and self.c_unk.size:
            k = self.c_unk.size
            Aa = np.zeros((k + 1, k + 1))
            Aa[:k, :k] = Ac
            Aa[:k, k] = 1.0
            Aa[k, :k] = 1.0
            Ac = Aa
        self.c_lu = sla.lu_factor(Ac) if self.c_unk.size else None

    # transfers -----------------------------------------------------------------
    def restrict(self, r_f, lf, lc):
        d, nf, nc = self.dim, lf.n, lc.n
        R = r_f.reshape((nf,) * d, order="F")
        acc = np.zeros((nc,) * d)
        for off in np.ndindex(*([2] * d)):
            sl = tuple(slice(o, nf, 2) for o in off)
            acc += R[sl]
        out = (acc / 2 ** d).ravel(order="F")
        out[~lc.unk_flat] = 0.0
        return out

    def prolong(self, e_c, lc, lf):
        d, nf, nc = self.dim, lf.n, lc.n
        E = e_c.reshape((nc,) * d, order="F")
        U = lc.unk_flat.reshape((nc,) * d, order="F")
        out = np.zeros((nf,) * d)
        neumann = self.bc == NEUMANN
        for off in np.ndindex(*([2] * d)):
            # fine nodes 2I + off; neighbours I + sel * sgn, sgn = -1 if off == 0 else +1
            acc = np.zeros((nc,) * d)
            cnt = np.zeros((nc,) * d)
            for sel in np.ndindex(*([2] * d)):
                wgt = 1.0
                shift = []
                for k in range(d):
                    sgn = -1 if off[k] == 0 else 1
                    shift.append(sgn * sel[k])
                    wgt *= 0.25 if sel[k] else 0.75
                val, valid = self._shifted(E, U, shift)
                if neumann:
                    acc += np.where(valid, val, 0.0)
                    cnt += valid
                else:
                    acc += wgt * np.where(valid, val, 0.0)
            if neumann:
                acc = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)
            out[tuple(slice(o, nf, 2) for o in off)] = acc
        out = out.ravel(order="F")
        out[~lf.unk_flat] = 0.0
        return out

    @staticmethod
    def _shifted(E, U, shift):
        """Values E[I + shift] and whether that node is an in-box unknown."""
        d = E.ndim
        n = E.shape[0]
        val = np.zeros_like(E)
        valid = np.zeros(E.shape, dtype=bool)
        src, dst = [], []
        for k in range(d):
            s = shift[k]
            if s >= 0:
                src.append(slice(s, n)); dst.append(slice(0, n - s))
            else:
                src.append(slice(0, n + s)); dst.append(slice(-s, n))
        val[tuple(dst)] = E[tuple(src)]
        valid[tuple(dst)] = U[tuple(src)]
        return val, valid

    # cycle ---------------------------------------------------------------------
    def coarse_solve(self, f):
        c = self.levels[-1]
        u = np.zeros(c.n ** self.dim)
        if self.c_unk.size:
            rhs = f[self.c_unk]
            if self.augmented:
                rhs = np.append(rhs, 0.0)
            u[self.c_unk] = sla.lu_solve(self.c_lu, rhs)[:self.c_unk.size]
        return u

    def vcycle(self, f, lev=0, u0=None):
        """One cycle on level lev for L u = f, from u0 (zero if None).  gamma = 1 is the
        V-cycle; gamma = 2 the W-cycle (Sec. 3.3 results): the coarser level is visited
        twice, the second visit starting from the first visit's result."""
        L = self.levels[lev]
        if lev == len(self.levels) - 1:
            return self.coarse_solve(f)
        u = np.zeros_like(f) if u0 is None else u0.copy()
        for _ in range(self.nu1):
            L.gs_colour(u, f, 0)
            L.gs_colour(u, f, 1)
        r = f - L.apply(u)
        r[~L.unk_flat] = 0.0
        fc = self.restrict(r, L, self.levels[lev + 1])
        ec = None
        for _ in range(self.gamma):
            ec = self.vcycle(fc, lev + 1, ec)
        u += self.prolong(ec, self.levels[lev + 1], L)
        for _ in range(self.nu2):
            L.gs_colour(u, f, 0)
            L.gs_colour(u, f, 1)
        return u

    def precondition(self, v, plus_flat):
        """z = one cycle applied to v / beta_sigma (Sec. 3.3, interface and boundary alike)."""
        f = v / np.where(plus_flat, self.beta_p, self.beta_m)
        f[~self.levels[0].unk_flat] = 0.0
        return self.vcycle(f)
