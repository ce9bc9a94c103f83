"""One IIM Poisson problem end to end in the oracle: operator, data, MG, FGMRES."""
from __future__ import annotations

import numpy as np

import workloads as W
from .fgmres import fgmres
from .mg import Multigrid
from .operator import IIMOperator


class OracleProblem:
    def __init__(self, spec, nu1=2, nu2=2, check_curvature=True, cycle=1):
        self.spec = spec
        self.op = IIMOperator(spec, check_curvature=check_curvature)
        self.n, self.d = spec.n, spec.dim
        self.plus_flat = self.op.plus.ravel(order="F")
        self.unk_flat = self.op.unknown.ravel(order="F")
        self._mg = None
        self.nu1, self.nu2 = nu1, nu2
        self.cycle = cycle          # coarse visits per level: 1 V-cycle, 2 W-cycle

    @property
    def mg(self):
        if self._mg is None:
            s = self.spec
            self._mg = Multigrid(self.op.ls, s.n, s.bc, s.box_bc, s.beta_plus, s.beta_minus, self.nu1, self.nu2,
                                 self.cycle)
        return self._mg

    def data(self, spec=None):
        """Manufactured data at this oracle's own control points and box points."""
        spec = spec or self.spec
        xc, nc = self.op.control_points()
        g, j0, j1 = W.boundary_data(spec, xc, nc)
        X = W.node_coords(spec.n, spec.dim)
        f = W.to_flat(W.source_term(spec, X, self.op.plus))
        return f, {"g": g, "j0": j0, "j1": j1, "box": W.box_data(spec)}

    def exact(self, spec=None):
        spec = spec or self.spec
        X = W.node_coords(spec.n, spec.dim)
        up = spec.solution.u_plus(X)
        if spec.bc == W.INTERFACE:
            u = np.where(self.op.plus, up, spec.solution.u_minus(X))
        else:
            u = np.where(self.op.plus, up, 0.0)
        return W.to_flat(u)

    def apply(self, u):
        return self.op.apply(u)

    def precondition(self, v):
        return self.mg.precondition(v, self.plus_flat)

    @property
    def singular(self):
        """Pure Neumann problem (no outer box): L 1 = 0, solution defined up to a constant."""
        return self.spec.bc == W.NEUMANN and self.spec.box_bc == W.BOX_NONE

    def system(self, f, data, gamma=0.0):
        """(apply, precondition, right-hand side, N) of the Krylov iteration.  Singular (pure
        Neumann) problems take the augmented system of Sec. 2.3, [L 1; 1^T 0][u; alpha] =
        [b; gamma] with 1 over the unknowns, preconditioned by the cycle on u and the
        identity on alpha; N is then the index of alpha, else None."""
        b = self.op.rhs(f, data)
        if not self.singular:
            return self.op.apply, self.precondition, b, None
        unk = self.unk_flat.astype(float)
        N = b.size

        def apply_aug(z):
            out = np.empty(N + 1)
            out[:N] = self.op.apply(z[:N]) + z[N] * unk
            out[N] = unk @ z[:N]
            return out

        def precond_aug(v):
            out = np.empty(N + 1)
            out[:N] = self.precondition(v[:N])
            out[N] = v[N]
            return out

        return apply_aug, precond_aug, np.append(b, gamma), N

    @staticmethod
    def _split(x, info, rhs, N):
        if N is None:
            return x, info, rhs
        info["alpha"] = x[N]
        return x[:N], info, rhs[:N]

    def solve(self, f, data, tol=1e-13, restart=10, max_iter=1000, gamma=0.0):
        """Solve L u = b by right-preconditioned FGMRES(m) (Sec. 4.1); singular problems
        through the augmented system (info["alpha"]: the shift that makes b + alpha 1
        compatible)."""
        A, M, rhs, N = self.system(f, data, gamma)
        x, info = fgmres(A, M, rhs, tol=tol, restart=restart, max_iter=max_iter)
        return self._split(x, info, rhs, N)

    def solve_left(self, f, data, tol=None, restart=10, max_iter=1000, gamma=0.0):
        """Left-preconditioned GMRES(m) (the 2D solver of Sec. 3.2) with its stopping rule
        |M r| <= tol |M b|, tol = 1e-6 / n by default; singular problems as in solve."""
        from .fgmres import gmres_left
        tol = 1e-6 / self.n if tol is None else tol
        A, M, rhs, N = self.system(f, data, gamma)
        x, info = gmres_left(A, M, rhs, tol=tol, restart=restart, max_iter=max_iter)
        return self._split(x, info, rhs, N)
