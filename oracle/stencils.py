"""Centred second-derivative stencils (paper Sec. 2.1 and Sec. 2.5).

The n-th order stencil a_{-w..w} (w = n/2) is the unique symmetric stencil with
sum_j a_j j^p / p! = [p == 2] for p = 0..2w, i.e. exact for polynomials of
degree <= n+1.  Its symbol is sigma(k) = 2 sum_{j>=1} a_j (1 - cos(j k)) and
sigma_max = max sigma (Tab. 1: 4, 16/3, 272/45 for orders 2, 4, 6).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np


def second_derivative_fractions(order: int):
    """Exact coefficients (a_0, a_1, ..., a_w) as Fractions."""
    w = order // 2
    # unknowns a_0..a_w; equations for even p = 0, 2, ..., 2w
    rows = []
    rhs = []
    for p in range(0, 2 * w + 1, 2):
        row = [Fraction(1 if p == 0 else 0)]           # j = 0 contributes 0^p
        for j in range(1, w + 1):
            row.append(Fraction(2 * j ** p, factorial(p)))
        rows.append(row)
        rhs.append(Fraction(1 if p == 2 else 0))
    # Gauss-Jordan in exact arithmetic
    m = len(rows)
    A = [r[:] + [b] for r, b in zip(rows, rhs)]
    for c in range(m):
        piv = next(r for r in range(c, m) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(m):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [v - f * u for v, u in zip(A[r], A[c])]
    return [A[r][m] for r in range(m)]


def second_derivative(order: int) -> np.ndarray:
    """Full stencil a_{-w..w} as float64."""
    half = [float(v) for v in second_derivative_fractions(order)]
    w = len(half) - 1
    return np.array(half[:0:-1] + half)


def sigma(order: int, k):
    a = second_derivative_fractions(order)
    k = np.asarray(k, dtype=float)
    return sum(2 * float(a[j]) * (1 - np.cos(j * k)) for j in range(1, len(a)))


def sigma_max(order: int) -> Fraction:
    """sigma(pi) for these stencils (the maximum is attained at k = pi)."""
    a = second_derivative_fractions(order)
    return sum(2 * a[j] * (1 - (-1) ** j) for j in range(1, len(a)))


def first_derivative_fractions(order: int):
    """Exact coefficients (b_1, ..., b_w) of the centred first-derivative stencil of the
    given order: b_{-j} = -b_j, b_0 = 0, sum_j b_j j^p / p! = [p == 1] for odd p <= 2w - 1,
    so the stencil is exact for polynomials of degree <= 2w = order (the gradient of the
    paper's Sec. 2.4 results uses the centred stencil of the scheme's order)."""
    w = order // 2
    rows, rhs = [], []
    for p in range(1, 2 * w, 2):
        rows.append([Fraction(2 * j ** p, factorial(p)) for j in range(1, w + 1)])
        rhs.append(Fraction(1 if p == 1 else 0))
    m = len(rows)
    A = [r[:] + [b] for r, b in zip(rows, rhs)]
    for c in range(m):
        piv = next(r for r in range(c, m) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(m):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [v - f * u for v, u in zip(A[r], A[c])]
    return [A[r][m] for r in range(m)]


def first_derivative(order: int) -> np.ndarray:
    """Full stencil b_{-w..w} as float64 (b_0 = 0, odd)."""
    half = [float(v) for v in first_derivative_fractions(order)]
    return np.array([-v for v in half[::-1]] + [0.0] + half)
