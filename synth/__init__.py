"""Seeded synthetic operands for the emulated-DGEMM workloads.

This module draws random numbers only; it holds none of the emulation's
arithmetic, so both the CUDA path's tests and the CPU oracle can take their
inputs from it.

Workloads:

* ``phi_pair(m, n, k, phi, seed)``: entries (U(-0.5, 0.5)) * exp(phi * N(0, 1)),
  the operand family whose exponent spread grows with phi. Generator: numpy
  PCG64 ``default_rng(seed)``; draw order U for A, N for A, U for B, N for B,
  each in row-major order.
* ``row_scaled_pair(n, seed)``: the paper's timing operands (Table tab:setup):
  row i of each operand is N(0, 1) times 2^{e_i}, e_i an integer drawn
  uniformly from [-20, 20), separately for A and B.
* ``batch_shapes(count, lo, hi, seed)``: m, n, k each log-uniform on [lo, hi].
"""
from __future__ import annotations

import numpy as np


def phi_matrix(rng: np.random.Generator, rows: int, cols: int, phi: float) -> np.ndarray:
    u = rng.random((rows, cols)) - 0.5
    g = rng.standard_normal((rows, cols))
    return u * np.exp(phi * g)


def phi_pair(m: int, n: int, k: int, phi: float, seed: int = 0):
    """A (m x k) and B (k x n), float64, row-major."""
    rng = np.random.default_rng(seed)
    A = phi_matrix(rng, m, k, phi)
    B = phi_matrix(rng, k, n, phi)
    return A, B


def row_scaled_pair(n: int, seed: int = 0, m: int | None = None, k: int | None = None):
    m = n if m is None else m
    k = n if k is None else k
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * np.ldexp(1.0, rng.integers(-20, 20, size=m))[:, None]
    B = rng.standard_normal((k, n)) * np.ldexp(1.0, rng.integers(-20, 20, size=k))[:, None]
    return A, B


def batch_shapes(count: int = 256, lo: int = 64, hi: int = 4096, seed: int = 0):
    """count (m, n, k) triples, each dimension log-uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(count, 3)))
    return np.clip(np.rint(x).astype(np.int64), lo, hi)


def sample_entries(m: int, n: int, count: int, seed: int = 1):
    """count distinct-ish (row, col) pairs, uniform, plus the four corners."""
    rng = np.random.default_rng(seed)
    r = rng.integers(0, m, size=count)
    c = rng.integers(0, n, size=count)
    corners_r = np.array([0, 0, m - 1, m - 1])
    corners_c = np.array([0, n - 1, 0, n - 1])
    return np.concatenate([corners_r, r]).astype(np.int64), np.concatenate([corners_c, c]).astype(np.int64)
