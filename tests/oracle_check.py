"""Reference results for the GPU tests, from the CPU oracle.

Every path of the library returns C = fl(2^-(s_i + t_j) (A'B')_ij), one
rounding of the exact product of the truncated operands (Sec. "Emulation
Problem"), so the oracle's C at the plan's bit budget is the expected result
bit for bit, whatever the path (batched, grouped, host operands, the static
scratch, the autograd products). Small products are compared entry by entry;
large ones on a fixed sample of entries that includes the first and last row
and column.
"""
from __future__ import annotations

import numpy as np

import oracle

FULL_LIMIT = 3e8          # m n k up to which every entry is computed


def sample_entries(m: int, n: int, count: int = 512, seed: int = 0):
    """(rows, cols) of `count` random entries, up to 64 entries of the last row
    and of the last column, and the four corners."""
    rng = np.random.default_rng(seed)
    rows = [rng.integers(0, m, count), np.full(min(n, 64), m - 1), rng.integers(0, m, min(m, 64)),
            np.array([0, 0, m - 1, m - 1])]
    cols = [rng.integers(0, n, count), rng.integers(0, n, min(n, 64)), np.full(min(m, 64), n - 1),
            np.array([0, n - 1, 0, n - 1])]
    return np.concatenate(rows).astype(np.int64), np.concatenate(cols).astype(np.int64)


def assert_oracle_bits(C, A, B, moduli, bits, what: str = "", full_limit: float = FULL_LIMIT, count: int = 512,
                       seed: int = 0):
    """C (m x n, host array or tensor) equals the oracle's product of A (m x k)
    and B (k x n) at the given moduli and bit budget, bit for bit: every entry
    when m n k <= full_limit, else the entries of sample_entries."""
    if hasattr(C, "detach"):
        C = C.detach().cpu().numpy()
    if hasattr(A, "detach"):
        A = A.detach().cpu().numpy()
    if hasattr(B, "detach"):
        B = B.detach().cpu().numpy()
    C = np.ascontiguousarray(C, dtype=np.float64)
    m, k = A.shape
    n = B.shape[1]
    assert C.shape == (m, n), (what, C.shape, (m, n))
    if m == 0 or n == 0:
        return
    if m * n * max(k, 1) <= full_limit:
        ref = oracle.dgemm(A, B, moduli, bits)
        bad = np.argwhere(C.view(np.uint64) != ref.view(np.uint64))
        assert bad.size == 0, (f"{what}: {len(bad)} of {m * n} entries differ from the oracle "
                               f"(m={m} n={n} k={k} bits={bits}); first at {tuple(bad[0])}: "
                               f"{C[tuple(bad[0])]!r} vs {ref[tuple(bad[0])]!r}")
    else:
        r, c = sample_entries(m, n, count, seed)
        ref = oracle.dgemm_entries(A, B, moduli, bits, r, c)
        got = C[r, c]
        bad = np.flatnonzero(got.view(np.uint64) != ref.view(np.uint64))
        assert bad.size == 0, (f"{what}: {len(bad)} of {len(r)} sampled entries differ from the oracle "
                               f"(m={m} n={n} k={k} bits={bits}); first at ({r[bad[0]]}, {c[bad[0]]}): "
                               f"{got[bad[0]]!r} vs {ref[bad[0]]!r}")
