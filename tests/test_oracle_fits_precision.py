"""Pin of the oracle's least-squares rows against 40-digit arithmetic (Sec. 2.1, Eq. 4).

Every ghost row of the (6,7) interface operator is v(xi_g)^T V^+, the pseudo-inverse of
the control point's Vandermonde matrix.  Here each row is recomputed independently at 40
significant digits, (V^T V)^-1 V^T with mpmath, from the fit's own nodes, and the oracle's
FP64 rows (Householder QR) must agree with it to the rounding level the least-squares
problems allow.  This fixes how close any FP64 implementation of these fits can come to
the exact rows, and so the bound under which the GPU operator and the oracle's can agree
on inputs that excite the ghost values (random data): the two FP64 results each carry
an error of this size.  A mistake in the QR step (a transposed factor, a dropped row, a
wrong ghost position) would put the rows far outside it.
"""
import numpy as np
import pytest

import workloads as W
from oracle.operator import IIMOperator

mp = pytest.importorskip("mpmath")


def _exponents(dim, q):
    return [(a, deg - a) for deg in range(q + 1) for a in range(deg, -1, -1)]


def test_ghost_rows_match_40_digit_least_squares():
    mp.mp.dps = 40
    spec = W.ProblemSpec(n=64, geometry=W.Geometry(W.FOURIER, (0.01, -0.02), False,
                                                   coef=(0.5, 0.03, -0.02, 0.0, 0.025, 0.01, 0.0, 0.0, 0.008)),
                         bc=W.INTERFACE, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=0.5, beta_minus=1.0)
    op = IIMOperator(spec)
    n, h, w = op.n, op.h, op.w
    xg = -1.0 + (np.arange(n) + 0.5) * h
    # ghost node of each fit's row k, from the records that use it
    ghost_pos = {}
    for (node, ax, s, jstar, c, side) in op.iim_rec:
        m = np.array(np.unravel_index(node, (n, n), order="F"))
        for j in range(jstar, w + 1):
            p = m.copy()
            p[ax] += j * s
            ghost_pos.setdefault((c, side), {})[j - jstar] = xg[p]
    exps = _exponents(2, op.q)
    worst, checked = 0.0, 0
    keys = sorted(ghost_pos)[::4]          # every fourth fit: both sides, all axes, ~60 fits
    for key in keys:
        f = op.fits[key]
        xc = op.cross.x[key[0]]
        pts = np.vstack([xc, np.stack([xg[np.array(np.unravel_index(k, (n, n), order="F"))]
                                       for k in f.nodes])])
        xi = [[(mp.mpf(float(p[k])) - mp.mpf(float(xc[k]))) / mp.mpf(h) for k in range(2)] for p in pts]
        V = mp.matrix([[x[0] ** a * x[1] ** b for (a, b) in exps] for x in xi])
        Vp = mp.inverse(V.T * V) * V.T
        for k, xgk in ghost_pos[key].items():
            z = [(mp.mpf(float(xgk[i])) - mp.mpf(float(xc[i]))) / mp.mpf(h) for i in range(2)]
            vg = mp.matrix([[z[0] ** a * z[1] ** b for (a, b) in exps]])
            exact = np.array((vg * Vp).tolist(), dtype=float)[0]
            got = f.ghost[k]
            err = np.max(np.abs(got - exact)) / np.sum(np.abs(exact))
            worst = max(worst, err)
            checked += 1
    assert checked > 50
    # rounding level of the least-squares rows: far below any algebraic slip, above eps
    assert worst < 1e-12, worst
