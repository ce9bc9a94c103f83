"""Right-preconditioned flexible GMRES(m) (paper Sec. 4.1; Saad 1993).

Sec. 4.1 uses FGMRES with right preconditioning and restart 10 because the
preconditioner may vary between applications.  Per cycle:
    v_1 = r/|r|;  for j: z_j = M_j(v_j), w = A z_j, orthogonalise w against
    v_1..v_j (modified Gram-Schmidt here), v_{j+1} = w/h_{j+1,j};
    Givens rotations keep the least-squares residual |g_{j+1}|;
    at the end x += Z y with H y = g.
Stopping reading: the true relative residual |b - A x| / |b| <= tol, checked
whenever the Arnoldi estimate drops below tol and at every restart.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, precond, b, tol=1e-10, restart=10, max_iter=500, x0=None):
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    hist = []
    if nb == 0.0:
        return x, {"iters": 0, "relres": 0.0, "converged": True, "hist": hist}
    r = b - apply_A(x)
    beta = np.linalg.norm(r)
    iters = 0
    while True:
        rel = beta / nb
        hist.append(rel)
        if rel <= tol:
            return x, {"iters": iters, "relres": rel, "converged": True, "hist": hist}
        if iters >= max_iter:
            return x, {"iters": iters, "relres": rel, "converged": False, "hist": hist}
        m = restart
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            iters += 1
            if abs(g[j + 1]) / nb <= tol or iters >= max_iter or breakdown:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + y @ Z[:k]
        r = b - apply_A(x)
        beta = np.linalg.norm(r)


def gmres_left(apply_A, precond, b, tol=1e-6, restart=10, max_iter=500, x0=None):
    """Left-preconditioned GMRES(m) (the 2D solver of Sec. 3.2; Saad 2003): GMRES on
    M A x = M b with modified Gram-Schmidt; the residual it minimises and tests is the
    preconditioned one, |M (b - A x)| <= tol |M b|, checked on the Arnoldi estimate and on
    the true preconditioned residual at every restart."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    mb = np.linalg.norm(precond(b))
    hist = []
    if mb == 0.0:
        return x, {"iters": 0, "relres": 0.0, "converged": True, "hist": hist}
    iters = 0
    while True:
        r = precond(b - apply_A(x))
        beta = np.linalg.norm(r)
        rel = beta / mb
        hist.append(rel)
        if rel <= tol:
            return x, {"iters": iters, "relres": rel, "converged": True, "hist": hist}
        if iters >= max_iter:
            return x, {"iters": iters, "relres": rel, "converged": False, "hist": hist}
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = precond(apply_A(V[j]))
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            if abs(g[j + 1]) / mb <= tol or iters >= max_iter or breakdown:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + V[:k].T @ y
