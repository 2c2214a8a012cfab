"""Exact brute force with Python integers and fractions, for tiny inputs.

Used only to pin the oracle. Each function writes out a definition from the
paper with exact arithmetic and no residues, so that a mistake in the oracle's
residue, CRT or rounding steps shows up as a mismatch here.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def to_float(q: Fraction) -> float:
    """Correctly rounded binary64 value of an exact rational (CPython's int true
    division rounds once, to nearest even, with gradual underflow)."""
    try:
        return q.numerator / q.denominator
    except OverflowError:
        return math.inf if q > 0 else -math.inf


def shift(vec, beta: int) -> int:
    """eq. convert: the largest s with every |x| 2^s < 2^beta; 0 for a zero vector."""
    mx = max((abs(float(x)) for x in vec), default=0.0)
    if mx == 0.0:
        return 0
    return beta - math.frexp(mx)[1]


def trunc_scaled(x: float, s: int) -> int:
    q = Fraction(float(x)) * (Fraction(2) ** int(s))
    return int(q)          # int() of a Fraction rounds toward zero


def emulated(A: np.ndarray, B: np.ndarray, beta: int):
    """C = fl(diag(mu)^-1 (A'B') diag(nu)^-1) with A'B' exact; also returns X = A'B', s, t."""
    M, K = A.shape
    _, N = B.shape
    s = [shift(A[i, :], beta) for i in range(M)]
    t = [shift(B[:, j], beta) for j in range(N)]
    Ap = [[trunc_scaled(A[i, h], s[i]) for h in range(K)] for i in range(M)]
    Bp = [[trunc_scaled(B[h, j], t[j]) for j in range(N)] for h in range(K)]
    X = [[sum(Ap[i][h] * Bp[h][j] for h in range(K)) for j in range(N)] for i in range(M)]
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            C[i, j] = to_float(Fraction(X[i][j]) * Fraction(2) ** (-(s[i] + t[j])))
    return C, X, s, t


def exact_product(A: np.ndarray, B: np.ndarray):
    """(AB)_ij as exact Fractions."""
    M, K = A.shape
    _, N = B.shape
    FA = [[Fraction(float(A[i, h])) for h in range(K)] for i in range(M)]
    FB = [[Fraction(float(B[h, j])) for j in range(N)] for h in range(K)]
    return [[sum(FA[i][h] * FB[h][j] for h in range(K)) for j in range(N)] for i in range(M)]


def balanced(x: int, m: int) -> int:
    r = x % m
    return r - m if r >= (m + 1) // 2 else r
