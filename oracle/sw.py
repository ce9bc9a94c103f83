"""Shortley-Weller low-order discretisation (paper Sec. 3.1).

1D formulas with psi = (distance to the wall) / dx:
  Dirichlet, Eq. 18 (case (c); a regular side uses psi = 1 and its neighbour):
     u'' = [2 uw-/(psi-(psi-+psi+)) - 2 u_i/(psi- psi+) + 2 uw+/(psi+(psi-+psi+))] / dx^2
  Neumann, Eq. 19 (a) wall on the left, (b) wall on the right, (c) both:
     (a) [-2 dx dUw-/(2psi-+psi+) - 2u_i/(psi+(2psi-+psi+)) + 2u_{i+1}/(psi+(2psi-+psi+))] / dx^2
     (b) [ 2u_{i-1}/(psi-(psi-+2psi+)) - 2u_i/(psi-(psi-+2psi+)) + 2 dx dUw+/(psi-+2psi+)] / dx^2
     (c) [dUw+ - dUw-] / (dx (psi- + psi+))
  Reading: the printed case (b) carries psi+ in the first two denominators;
  the mirror image of case (a) and exactness on quadratics (the property that
  defines these stencils) both require psi-, which is what is used here.
  Interface wall values, Eq. 21, with alpha = psi/beta and x_i on the minus side:
     uw+ = ub + alpha+ [u]/(alpha+ + alpha-),  uw- = ub - alpha- [u]/(alpha+ + alpha-),
     ub  = (alpha+ u_i + alpha- u_{i+1})/(alpha+ + alpha-)
           - dx alpha+ alpha- [beta u']/(alpha+ + alpha-),
  Reading: these values satisfy uw+ - uw- = [u], the convention of Sec. 2.2
  ([u] = u+ - u-, stated before Eq. 9), and the flux balance of Eq. 20; the
  "[u] = uw- - uw+" printed in Eq. 20 is taken as a sign slip.  Only the homogeneous form,
  the same under either sign, enters the preconditioner.
Shift (Sec. 3.1, last paragraph): boundary psi is clamped to >= 1/2; interface
psi+ = psi- = 1/2.  Multi-D: the 1D stencils are applied along each axis.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads import DIRICHLET, NEUMANN, INTERFACE, BOX_DIRICHLET
from .geometry import Crossings, grid_x, phase_plus

REG, DIR, NEU = 0, 1, 2


# --------------------------------------------------------------------------- 1D formulas
def sw_dirichlet(uwm, ui, uwp, pm, pp, dx):
    return (2 * uwm / (pm * (pm + pp)) - 2 * ui / (pm * pp) + 2 * uwp / (pp * (pm + pp))) / dx ** 2


def sw_neumann_left(dum, ui, uip1, pm, pp, dx):
    den = 2 * pm + pp
    return (-2 * dx * dum / den - 2 * ui / (pp * den) + 2 * uip1 / (pp * den)) / dx ** 2


def sw_neumann_right(uim1, ui, dup, pm, pp, dx):
    den = pm + 2 * pp
    return (2 * uim1 / (pm * den) - 2 * ui / (pm * den) + 2 * dx * dup / den) / dx ** 2


def sw_neumann_both(dum, dup, pm, pp, dx):
    return (dup - dum) / (dx * (pm + pp))


def sw_interface_walls(ui, uip1, jump_u, jump_flux, pm, pp, beta_m, beta_p, dx):
    """Wall values (uw+, uw-) of Eq. 21; x_i on the minus side, x_{i+1} on the plus side."""
    ap, am = pp / beta_p, pm / beta_m
    ub = (ap * ui + am * uip1) / (ap + am) - dx * ap * am * jump_flux / (ap + am)
    return ub + ap * jump_u / (ap + am), ub - am * jump_u / (ap + am)


def clamp_psi(psi):
    return np.maximum(psi, 0.5)


# --------------------------------------------------------------------------- one level
class SWLevel:
    """Homogeneous SW operator (the Laplacian, no beta) on one cell-centred level.

    A : scipy CSR over all n^d nodes (rows of non-unknowns are empty).
    Per node and axis the left/right side is one of: a regular neighbour
    (psi = 1), a Dirichlet wall (immersed boundary, psi clamped >= 1/2, or a box
    face at psi = 1/2, value 0), a Neumann wall (psi clamped >= 1/2, zero flux),
    or an interface wall (psi = 1/2, value = the Eq. 21 wall value, which
    couples the node with its neighbour across the interface).
    """

    def __init__(self, ls, n, bc, box_bc, beta_p, beta_m):
        self.n, self.d = n, ls.dim
        self.h = h = 2.0 / n
        self.bc = bc
        d = self.d
        N = n ** d
        self.plus = plus = phase_plus(ls, n)
        self.unknown = np.ones_like(plus) if bc == INTERFACE else plus.copy()
        cr = Crossings(ls, n, plus)
        plus_f = plus.ravel(order="F")
        unk_f = self.unknown.ravel(order="F")
        idx = np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"), axis=-1).reshape(-1, d, order="F")
        flat = np.arange(N)
        # crossing fraction t on the edge (lower node, axis)
        t_edge = np.full((d, N), np.nan)
        t_edge[cr.axis, cr.lo] = cr.t
        # interface wall weights (homogeneous Eq. 21 with psi = 1/2):
        # uw = lam_minus * u(minus node) + lam_plus * u(plus node)
        lam_minus, _ = sw_interface_walls(1.0, 0.0, 0.0, 0.0, 0.5, 0.5, beta_m, beta_p, 1.0)
        lam_plus, _ = sw_interface_walls(0.0, 1.0, 0.0, 0.0, 0.5, 0.5, beta_m, beta_p, 1.0)
        rows, cols, vals = [], [], []
        diag = np.zeros(N)
        for ax in range(d):
            kind, psi, nbr = {}, {}, {}
            for s in (-1, 1):
                pos = idx[:, ax] + s
                inb = (pos >= 0) & (pos < n)
                nb = flat + s * n ** ax
                nb = np.where(inb, nb, 0)
                same = inb & (plus_f[nb] == plus_f)
                k = np.full(N, REG)
                p = np.ones(N)
                if box_bc == BOX_DIRICHLET:
                    k[~inb] = DIR
                    p[~inb] = 0.5
                elif np.any(unk_f & ~inb):
                    raise ValueError("unknown node touches a box without condition")
                cut = inb & ~same
                lower = flat if s > 0 else nb
                t = t_edge[ax, lower]
                dist = t if s > 0 else 1.0 - t
                if bc == INTERFACE:
                    k[cut] = 3
                    p[cut] = 0.5
                else:
                    k[cut] = DIR if bc == DIRICHLET else NEU
                    p[cut] = clamp_psi(dist[cut])
                kind[s], psi[s], nbr[s] = k, p, nb
            kl, kr, pl, pr = kind[-1], kind[1], psi[-1], psi[1]
            neu_l, neu_r = kl == NEU, kr == NEU
            one, zero = np.ones(N), np.zeros(N)
            cl = np.where(~neu_l & ~neu_r, sw_dirichlet(one, zero, zero, pl, pr, h),
                          np.where(neu_r & ~neu_l, sw_neumann_right(one, zero, zero, pl, pr, h), 0.0))
            c0 = np.where(~neu_l & ~neu_r, sw_dirichlet(zero, one, zero, pl, pr, h),
                          np.where(neu_l & ~neu_r, sw_neumann_left(zero, one, zero, pl, pr, h),
                                   np.where(neu_r & ~neu_l, sw_neumann_right(zero, one, zero, pl, pr, h), 0.0)))
            cR = np.where(~neu_l & ~neu_r, sw_dirichlet(zero, zero, one, pl, pr, h),
                          np.where(neu_l & ~neu_r, sw_neumann_left(zero, zero, one, pl, pr, h), 0.0))
            diag += np.where(unk_f, c0, 0.0)
            for s, coef in ((-1, cl), (1, cR)):
                k, nb = kind[s], nbr[s]
                reg = unk_f & (k == REG)
                rows.append(flat[reg]); cols.append(nb[reg]); vals.append(coef[reg])
                itf = unk_f & (k == 3)
                lam_self = np.where(plus_f, lam_plus, lam_minus)
                lam_other = np.where(plus_f, lam_minus, lam_plus)
                diag[itf] += coef[itf] * lam_self[itf]
                rows.append(flat[itf]); cols.append(nb[itf]); vals.append(coef[itf] * lam_other[itf])
        rows.append(flat[unk_f]); cols.append(flat[unk_f]); vals.append(diag[unk_f])
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
        self.diag = self.A.diagonal()
        self.unk_flat = unk_f
        par = idx.sum(axis=1)
        self.red = (par % 2 == 0) & unk_f
        self.black = (par % 2 == 1) & unk_f

    def apply(self, u):
        out = self.A @ u
        out[~self.unk_flat] = 0.0
        return out

    def gs_colour(self, u, f, colour):
        """One red (colour 0: even index sum) or black Gauss-Seidel half sweep, in place."""
        mask = self.red if colour == 0 else self.black
        Au = self.A @ u
        dg = self.diag
        upd = mask & (dg != 0.0)
        u[upd] = u[upd] + (f[upd] - Au[upd]) / dg[upd]
        u[mask & (dg == 0.0)] = 0.0
        return u
