"""Configuration search for the low-precision float alphabets (host side).

A configuration (Sec. "Forms and Channels") is a set of pairwise-coprime
moduli, each with a form whose tables take values in the format's alphabet S.
This module builds, for an alphabet and an inner dimension K, the pool of
least-rank candidate forms per modulus (Sec. "Solving the Program", reduced
program eq. ov-reduced) and finds a set of least total rank whose product
exceeds the CRT window 2 K (2^beta - 1)^2 (eq. ov-crtgen).

Candidate forms (all with one accumulator per GEMM, so eq. ov-accgen holds
when every plane value is at most r = r_max(1) = floor(sqrt(Lambda / K)),
eq. rmax, with Lambda = 2^24 for FP32 accumulation):
  * one limb, rank 1: every class mod m has a member of S within r;
  * schoolbook, two limbs at base b with m | b^2, rank 3 (the group of weight
    b^2 vanishes, eq. qm): planes A0, A1;
  * Toom (Karatsuba) at points {0, 1, inf}, two limbs, rank 3: planes A0,
    A0 + A1, A1, weights (1 - b, b, b^2 - b);
  * schoolbook, two limbs, rank 4.
Each class is encoded by the tuple whose largest plane magnitude is least
(Sec. "Forms Built from Limbs"); ties go to the smaller |a1|, then the smaller
a1, then the smaller a0. A channel takes the first base b = 2, 3, ... that
admits m (its plane values are all within r by construction).

The exact search follows the structure of the paper's five-step method: the
moduli are grouped by their prime factor above a cutoff tau (every pool member
has at most one such factor, so a group contributes at most one member), and a
dynamic program over the subsets of the primes up to tau maximises log2 P for
every total rank; the set is recovered by replaying the program from
checkpoints.

This is product code: it writes the frozen configuration tables of the C
library (csrc/gen_fp_configs.py) and shares nothing with the oracle.
"""
from __future__ import annotations

import math

import numpy as np

FP32_LAMBDA = 2**24

# (exponent bits, mantissa bits, bias, reserved top exponent (IEEE inf/NaN), top code is NaN only)
FORMATS = {
    "E4M3": (4, 3, 7, False, True),
    "E5M2": (5, 2, 15, True, False),
    "E2M3": (2, 3, 1, False, False),
    "E3M2": (3, 2, 3, False, False),
    "E2M1": (2, 1, 1, False, False),
}

FORM_ONE, FORM_SCHOOL3, FORM_TOOM3, FORM_SCHOOL4 = 1, 2, 3, 4
RANK = {FORM_ONE: 1, FORM_SCHOOL3: 3, FORM_TOOM3: 3, FORM_SCHOOL4: 4}


def codes(fmt: str):
    """{code: value} of the finite values of an OCP low-precision float format."""
    e_bits, m_bits, bias, ieee_top, nan_top_code = FORMATS[fmt]
    out = {}
    for sign in (0, 1):
        for e in range(1 << e_bits):
            for m in range(1 << m_bits):
                if ieee_top and e == (1 << e_bits) - 1:
                    continue
                if nan_top_code and e == (1 << e_bits) - 1 and m == (1 << m_bits) - 1:
                    continue
                if e == 0:
                    v = m * 2.0**(1 - bias - m_bits)
                else:
                    v = ((1 << m_bits) + m) * 2.0**(e - bias - m_bits)
                code = (sign << (e_bits + m_bits)) | (e << m_bits) | m
                out[code] = -v if sign else v
    return out


def alphabet(fmt: str):
    """(S, e_S): the finite values scaled by 2^e_S, the least power of two
    making them all integers (Sec. "Forms and Channels")."""
    vals = set(codes(fmt).values())
    smallest = min(abs(v) for v in vals if v != 0)
    e_s = -int(math.log2(smallest))
    S = sorted({int(round(v * 2.0**e_s)) for v in vals})
    return S, e_s


def r_max1(K: int, lam: int = FP32_LAMBDA) -> int:
    return math.isqrt(lam // K)


def _first_per_class(keys_order_res, m):
    """Given residues in key order, the index of the first occurrence per class
    (or -1) as an array of length m."""
    first = np.full(m, -1, dtype=np.int64)
    idx = np.arange(keys_order_res.size)
    # reverse assignment keeps the first occurrence
    first[keys_order_res[::-1]] = idx[::-1]
    return first


class Pool:
    """Least-rank candidate form per modulus for an alphabet at inner dimension K."""

    def __init__(self, fmt: str, K: int, lam: int = FP32_LAMBDA, m_max: int | None = None):
        S, e_s = alphabet(fmt)
        self.fmt, self.K, self.e_s = fmt, K, e_s
        self.r = r_max1(K, lam)
        Sr = np.array([s for s in S if abs(s) <= self.r], dtype=np.int64)
        self.Sr = Sr
        Sset = set(int(x) for x in Sr)
        a0, a1 = np.meshgrid(Sr, Sr, indexing="ij")
        a0, a1 = a0.ravel(), a1.ravel()
        # schoolbook tuples ordered by (max |limb|, |a1|, a1, a0)
        key = np.lexsort((a0, a1, np.abs(a1), np.maximum(np.abs(a0), np.abs(a1))))
        self.sb0, self.sb1 = a0[key], a1[key]
        # Toom tuples: the sum plane must lie in S within r too
        ok = np.array([int(x + y) in Sset for x, y in zip(a0, a1)])
        t0, t1 = a0[ok], a1[ok]
        key = np.lexsort((t0, t1, np.abs(t1), np.maximum(np.maximum(np.abs(t0), np.abs(t1)), np.abs(t0 + t1))))
        self.tm0, self.tm1 = t0[key], t1[key]
        one = np.array(sorted(Sr.tolist(), key=lambda v: (abs(v), v)), dtype=np.int64)
        self.one = one
        top = m_max or (len(Sr) ** 2)
        self.form, self.base = {}, {}
        for m in range(2, top + 1):
            f, b = self._best(m)
            if f:
                self.form[m], self.base[m] = f, b

    def _covers(self, x0, x1, m, bases):
        """bool per base: do the tuples reach every class of m."""
        if x0.size < m:
            return np.zeros(len(bases), dtype=bool)
        R = (x0[:, None] + np.asarray(bases)[None, :] * x1[:, None]) % m
        seen = np.zeros((len(bases), m), dtype=bool)
        seen[np.repeat(np.arange(len(bases)), R.shape[0]), R.T.ravel()] = True
        return seen.all(axis=1)

    def _best(self, m):
        if np.unique(self.one % m).size == m:
            return FORM_ONE, 0
        squares = [b for b in range(2, m) if (b * b) % m == 0]
        if squares:
            cov = self._covers(self.sb0, self.sb1, m, squares)
            if cov.any():
                return FORM_SCHOOL3, int(squares[int(np.argmax(cov))])
        for lo in range(2, m, 256):
            bases = list(range(lo, min(m, lo + 256)))
            cov = self._covers(self.tm0, self.tm1, m, bases)
            if cov.any():
                return FORM_TOOM3, int(bases[int(np.argmax(cov))])
        for lo in range(2, m, 256):
            bases = list(range(lo, min(m, lo + 256)))
            cov = self._covers(self.sb0, self.sb1, m, bases)
            if cov.any():
                return FORM_SCHOOL4, int(bases[int(np.argmax(cov))])
        return 0, 0

    def cost(self, m):
        return RANK[self.form[m]]


def _primes_upto(n):
    return [p for p in range(2, n + 1) if all(p % d for d in range(2, math.isqrt(p) + 1))]


def _factor(n):
    f, p = [], 2
    while p * p <= n:
        while n % p == 0:
            f.append(p)
            n //= p
        p += 1
    if n > 1:
        f.append(n)
    return f


def search(pool: Pool, K: int, beta: int = 53, max_cost: int = 96, checkpoint: int = 24):
    """Least total rank of a pairwise-coprime set of pool moduli with
    P > 2 K (2^beta - 1)^2; among those, the largest P. Returns (Q, moduli)."""
    need = math.log2(2 * K) + 2 * math.log2(2**beta - 1)
    ms = sorted(pool.form)
    # cutoff: every member has at most one prime factor above tau
    tau = 1
    for m in ms:
        big = sorted(set(_factor(m)))
        if len(big) >= 2:
            tau = max(tau, big[-2])
    small = [p for p in _primes_upto(tau)]
    bit = {p: 1 << i for i, p in enumerate(small)}
    groups = {}
    for m in ms:
        mask, rest = 0, m
        for p in small:
            if rest % p == 0:
                mask |= bit[p]
                while rest % p == 0:
                    rest //= p
        # what is left is a power of the one prime above tau; members sharing
        # that prime form one group, of which at most one is taken
        key = _factor(rest)[0] if rest > 1 else -m
        groups.setdefault(key, []).append((m, mask, pool.cost(m)))
    order = list(groups.values())
    nm = 1 << len(small)
    masks = np.arange(nm)
    NEG = -1e300

    def step(dp, grp):
        new = dp.copy()
        for m, mk, c in grp:
            free = (masks & mk) == 0
            src = dp[free, : max_cost + 1 - c] + math.log2(m)
            tgt = masks[free] | mk
            new[tgt, c:] = np.maximum(new[tgt, c:], src)
        return new

    dp = np.full((nm, max_cost + 1), NEG)
    dp[0, 0] = 0.0
    saved = {0: dp.copy()}
    for g, grp in enumerate(order):
        dp = step(dp, grp)
        if (g + 1) % checkpoint == 0:
            saved[g + 1] = dp.copy()
    best_c = None
    for c in range(max_cost + 1):
        if dp[:, c].max() > need + 1e-9:
            best_c = c
            break
    if best_c is None:
        raise ValueError("no configuration within max_cost")
    mask = int(np.argmax(dp[:, best_c]))
    value = dp[mask, best_c]
    # replay: walk the groups backwards, rebuilding each segment's tables
    chosen = []
    c = best_c
    g = len(order)
    while g > 0:
        start = max(k for k in saved if k < g)
        tables = [saved[start]]
        for h in range(start, g):
            tables.append(step(tables[-1], order[h]))
        for h in range(g - 1, start - 1, -1):
            prev = tables[h - start]
            if abs(prev[mask, c] - value) < 1e-9:
                continue                                  # group h unused
            for m, mk, cc in order[h]:
                if (mask & mk) == mk and cc <= c:
                    pm = mask & ~mk
                    if abs(prev[pm, c - cc] + math.log2(m) - value) < 1e-9:
                        chosen.append(m)
                        mask, c, value = pm, c - cc, prev[pm, c - cc]
                        break
            else:
                raise RuntimeError("replay failed")
        g = start
    chosen.sort(reverse=True)
    return best_c, chosen


def encode_tables(pool: Pool, m: int):
    """Per class c in [0, m): the limb tuple of the channel's form, as arrays
    (a0, a1) of length m (a1 = 0 for one limb)."""
    f, b = pool.form[m], pool.base[m]
    if f == FORM_ONE:
        first = _first_per_class(pool.one % m, m)
        return pool.one[first], np.zeros(m, dtype=np.int64)
    x0, x1 = (pool.tm0, pool.tm1) if f == FORM_TOOM3 else (pool.sb0, pool.sb1)
    first = _first_per_class((x0 + b * x1) % m, m)
    assert (first >= 0).all()
    return x0[first], x1[first]
