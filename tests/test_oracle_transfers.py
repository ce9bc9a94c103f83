"""Oracle pins for the multigrid transfers (Sec. 3.3) on cell-centred grids.

* the prolongation with weights 3/4, 1/4 per axis reproduces bilinear (2D) and trilinear
  (3D) coarse functions exactly at every fine cell whose coarse neighbours lie in the
  grid: the fine centre sits a quarter of a coarse cell from the nearest coarse centre;
* the restriction (mean of the 2^d children) maps a linear fine function to the same
  function at the coarse centres, which are the children's centroids;
* the Neumann prolongation (unweighted mean of the in-domain coarse neighbours, Sec. 3.3)
  reproduces constants but not linear functions.
A swapped weight, a wrong neighbour direction or a sum in place of the mean fails these.
"""
import numpy as np
import pytest

import workloads as W
from oracle.geometry import LevelSet
from oracle.mg import Multigrid


def _centres(n, d):
    return W.node_coords(n, d)


def _interface_mg(d):
    if d == 2:
        geom = W.Geometry(W.STAR, (0.0, 0.0, 0.5, 0.05, 5.0, 0.0), False)
        n = 32
    else:
        geom = W.Geometry(W.SPHERE, (0.0, 0.0, 0.0, 0.45), False)
        n = 24
    return Multigrid(LevelSet(geom), n, W.INTERFACE, W.BOX_DIRICHLET, 1.0, 1.0, 2, 2, 1)


@pytest.mark.parametrize("d", [2, 3])
def test_prolongation_reproduces_multilinear_functions(d):
    mg = _interface_mg(d)
    lf, lc = mg.levels[0], mg.levels[1]
    assert lf.unk_flat.all() and lc.unk_flat.all()      # interface problems: every node
    rng = np.random.default_rng(d)
    coef = rng.standard_normal(2 ** d)

    def multilinear(X):
        out = np.zeros(X.shape[:-1])
        for k, sel in enumerate(np.ndindex(*([2] * d))):
            term = np.full(X.shape[:-1], coef[k])
            for ax in range(d):
                if sel[ax]:
                    term = term * X[..., ax]
            out += term
        return out

    ec = W.to_flat(multilinear(_centres(lc.n, d)))
    got = W.from_flat(mg.prolong(ec, lc, lf), lf.n, d)
    want = multilinear(_centres(lf.n, d))
    inner = tuple(slice(1, lf.n - 1) for _ in range(d))
    assert np.max(np.abs(got[inner] - want[inner])) < 1e-13
    # at the grid's edge a missing coarse neighbour counts as 0: not exact there
    assert np.max(np.abs(got - want)) > 1e-3


@pytest.mark.parametrize("d", [2, 3])
def test_restriction_of_linear_functions(d):
    mg = _interface_mg(d)
    lf, lc = mg.levels[0], mg.levels[1]
    a = np.random.default_rng(10 + d).standard_normal(d + 1)
    lin = lambda X: a[0] + np.tensordot(X, a[1:], axes=([-1], [0]))
    got = W.from_flat(mg.restrict(W.to_flat(lin(_centres(lf.n, d))), lf, lc), lc.n, d)
    assert np.max(np.abs(got - lin(_centres(lc.n, d)))) < 1e-13


def test_neumann_prolongation_reproduces_constants_only():
    geom = W.Geometry(W.CIRCLE, (0.02, -0.01, 0.45), False)
    mg = Multigrid(LevelSet(geom), 32, W.NEUMANN, W.BOX_DIRICHLET, 1.0, 1.0, 2, 2, 1)
    lf, lc = mg.levels[0], mg.levels[1]
    const = np.where(lc.unk_flat, 2.5, 0.0)
    got = mg.prolong(const, lc, lf)
    # every unknown fine node with an in-domain coarse neighbour gets the constant
    has = got != 0.0
    assert np.all(np.abs(got[has & lf.unk_flat] - 2.5) < 1e-14)
    assert (has & lf.unk_flat).sum() > 0.9 * lf.unk_flat.sum()
    X = _centres(lc.n, 2)
    lin = W.to_flat(1.0 + X[..., 0] + 0.5 * X[..., 1]) * lc.unk_flat
    gl = W.from_flat(mg.prolong(lin, lc, lf), lf.n, 2)
    Xf = _centres(lf.n, 2)
    want = 1.0 + Xf[..., 0] + 0.5 * Xf[..., 1]
    inner = W.from_flat(lf.unk_flat, lf.n, 2)
    assert np.max(np.abs(gl - want)[inner]) > 1e-3       # the mean is not bilinear
