"""Dense multivariate polynomials for the oracle (test infrastructure only).

A polynomial in ``dim`` variables is a numpy array ``c`` of ``np.longdouble``
with ``c[a, b, ...]`` the coefficient of ``x^a y^b ...``.  Products are
discrete convolutions, derivatives shift one axis.  Jacobi polynomials are
expanded with exact rational arithmetic (their three-term recurrence) before
conversion, so the only rounding is in extended precision.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

LD = np.longdouble


def zeros(dim: int, size: int) -> np.ndarray:
    return np.zeros((size,) * dim, dtype=LD)


def const(dim: int, value) -> np.ndarray:
    c = zeros(dim, 1)
    c[(0,) * dim] = LD(value)
    return c


def linear(dim: int, c0, coeffs) -> np.ndarray:
    """c0 + sum_i coeffs[i] x_i."""
    c = zeros(dim, 2)
    c[(0,) * dim] = LD(c0)
    for i, a in enumerate(coeffs):
        idx = [0] * dim
        idx[i] = 1
        c[tuple(idx)] = LD(a)
    return c


def _pad(c: np.ndarray, size: int) -> np.ndarray:
    if c.shape[0] == size:
        return c
    out = zeros(c.ndim, size)
    out[tuple(slice(0, s) for s in c.shape)] = c
    return out


def add(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    size = max(p.shape[0], q.shape[0])
    return _pad(p, size) + _pad(q, size)


def scale(p: np.ndarray, s) -> np.ndarray:
    return p * LD(s)


def mul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    dim = p.ndim
    size = p.shape[0] + q.shape[0] - 1
    out = zeros(dim, size)
    for idx in zip(*np.nonzero(p)):
        sl = tuple(slice(i, i + q.shape[0]) for i in idx)
        out[sl] += p[idx] * q
    return out


def power(p: np.ndarray, n: int) -> np.ndarray:
    out = const(p.ndim, 1)
    for _ in range(n):
        out = mul(out, p)
    return out


def deriv(p: np.ndarray, axis: int) -> np.ndarray:
    size = p.shape[0]
    if size == 1:
        return zeros(p.ndim, 1)
    n = np.arange(size, dtype=LD)
    shape = [1] * p.ndim
    shape[axis] = size
    q = p * n.reshape(shape)
    q = np.roll(q, -1, axis=axis)
    idx = [slice(None)] * p.ndim
    idx[axis] = size - 1
    q[tuple(idx)] = 0
    return q


def evaluate(p: np.ndarray, pts, dtype=np.float64) -> np.ndarray:
    """Evaluate at points [M, dim] (summed in long double); returns ``dtype`` [M]."""
    pts = np.asarray(pts, dtype=LD)
    dim = p.ndim
    size = p.shape[0]
    powers = [np.stack([pts[:, i] ** a for a in range(size)], axis=1) for i in range(dim)]
    if dim == 1:
        val = powers[0] @ p
    elif dim == 2:
        val = np.einsum("ma,mb,ab->m", powers[0], powers[1], p)
    else:
        val = np.einsum("ma,mb,mc,abc->m", powers[0], powers[1], powers[2], p)
    return np.asarray(val, dtype=dtype)


def compose_1d(coeffs, arg: np.ndarray) -> np.ndarray:
    """sum_m coeffs[m] * arg^m for a univariate coefficient list and a polynomial arg."""
    out = zeros(arg.ndim, 1)
    pw = const(arg.ndim, 1)
    for m, a in enumerate(coeffs):
        if m > 0:
            pw = mul(pw, arg)
        if a != 0:
            out = add(out, scale(pw, LD(a.numerator) / LD(a.denominator)))
    return out


def homogenised(coeffs, u: np.ndarray, v: np.ndarray, n: int) -> np.ndarray:
    """v^n P(u/v) = sum_m coeffs[m] u^m v^(n-m) (a polynomial when deg P <= n)."""
    out = zeros(u.ndim, 1)
    for m, a in enumerate(coeffs):
        if a != 0:
            term = mul(power(u, m), power(v, n - m))
            out = add(out, scale(term, LD(a.numerator) / LD(a.denominator)))
    return out


def jacobi_coeffs(n: int, alpha: int, beta: int):
    """Monomial coefficients (in t) of the Jacobi polynomial P_n^{(alpha,beta)}(t), exact.

    Standard normalisation P_n(1) = binom(n + alpha, n); three-term recurrence.
    """
    a, b = Fraction(alpha), Fraction(beta)
    P = [[Fraction(1)]]
    if n == 0:
        return P[0]
    # P_1 = (alpha+1) + (alpha+beta+2)(t-1)/2
    P.append([(a + 1) - (a + b + 2) / 2, (a + b + 2) / 2])
    for m in range(2, n + 1):
        c1 = 2 * m * (m + a + b) * (2 * m + a + b - 2)
        c2 = (2 * m + a + b - 1) * (a * a - b * b)
        c3 = (2 * m + a + b - 1) * (2 * m + a + b) * (2 * m + a + b - 2)
        c4 = 2 * (m + a - 1) * (m + b - 1) * (2 * m + a + b)
        new = [Fraction(0)] * (m + 1)
        for i, x in enumerate(P[m - 1]):
            new[i] += c2 * x / c1
            new[i + 1] += c3 * x / c1
        for i, x in enumerate(P[m - 2]):
            new[i] -= c4 * x / c1
        P.append(new)
    return P[n]
