"""Oracle for the float-format configurations: alphabets, channel pools, the
exact least-GEMM-count search of Sec. "Solving the Program", and form tables.

TEST INFRASTRUCTURE, like the rest of oracle/: only tests/ use it, and it
shares no code with the CUDA library or its planner.

Definitions followed (paper sections):
* Alphabet S (Sec. "Forms and Channels"): the finite values of the format
  scaled by the least power of two that makes them all integers.
* Form of rank r modulo m (eq. ov-form); the one-limb, schoolbook (eq. qm) and
  Toom forms of Sec. "Forms Built from Limbs"; a class is encoded by the tuple
  whose largest plane value is least in magnitude (ties, which the paper leaves
  open: smaller |a1|, then smaller a1, then smaller a0).
* Accumulator exactness (eq. ov-accgen) with one GEMM per accumulator: every
  plane value within r_max(1) = floor(sqrt(Lambda / K)) (eq. rmax).
* Window (eq. ov-crtgen) with B_A = B_B = 2^53 - 1.
* The search, in the five steps of Sec. "Solving the Program": cutoff tau,
  products over H (primes above tau), products over L by a program over the
  subsets of P, combination, and re-runs on a shared prime above tau.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

LAMBDA_FP32 = 2**24
LAMBDA_INT32 = 2**31 - 1

# name: (exponent bits, mantissa bits, bias, style); style "ieee" reserves the top
# exponent (inf/NaN), "fn" reserves only the all-ones code (NaN), "none" neither
SPECS = {"E4M3": (4, 3, 7, "fn"), "E5M2": (5, 2, 15, "ieee"), "E2M3": (2, 3, 1, "none"),
         "E3M2": (3, 2, 3, "none"), "E2M1": (2, 1, 1, "none")}


def float_values(name):
    """All finite values of an OCP low-precision float format, as Fractions."""
    eb, mb, bias, style = SPECS[name]
    out = set()
    for e in range(2**eb):
        for mt in range(2**mb):
            if style == "ieee" and e == 2**eb - 1:
                continue
            if style == "fn" and e == 2**eb - 1 and mt == 2**mb - 1:
                continue
            if e == 0:
                v = Fraction(mt, 2**mb) * Fraction(2) ** (1 - bias)
            else:
                v = (1 + Fraction(mt, 2**mb)) * Fraction(2) ** (e - bias)
            out.add(v)
            out.add(-v)
    return out


def alphabet(name):
    """(sorted integer alphabet S, e_S). INT8 / INT4 are the two's-complement ranges."""
    if name == "INT8":
        return list(range(-128, 128)), 0
    if name == "INT4":
        return list(range(-8, 8)), 0
    vals = float_values(name)
    e = 0
    while any((v * 2**e).denominator != 1 for v in vals):
        e += 1
    return sorted(int(v * 2**e) for v in vals), e


def rmax1(K, lam):
    return math.isqrt(lam // K)


def _cover(values, m):
    return len({v % m for v in values}) == m


class Pools:
    """Least-rank candidate form per modulus, over one-limb, schoolbook (two
    limbs, rank 4, or 3 when m | b^2) and Toom (two limbs, rank 3) forms."""

    def __init__(self, name, K, lam=LAMBDA_FP32, m_top=None):
        S, self.e_s = alphabet(name)
        self.r = rmax1(K, lam)
        self.Sr = [s for s in S if abs(s) <= self.r]
        Sset = set(self.Sr)
        self.pairs = [(x, y) for x in self.Sr for y in self.Sr]
        self.toom_pairs = [(x, y) for (x, y) in self.pairs if x + y in Sset]
        A0 = np.array([p[0] for p in self.pairs])
        A1 = np.array([p[1] for p in self.pairs])
        T0 = np.array([p[0] for p in self.toom_pairs])
        T1 = np.array([p[1] for p in self.toom_pairs])
        top = m_top or len(self.Sr) ** 2
        self.rank, self.kind, self.base = {}, {}, {}
        for m in range(2, top + 1):
            if _cover(self.Sr, m):
                self.rank[m], self.kind[m], self.base[m] = 1, "one", None
                continue
            found = False
            for b in range(2, m):
                if (b * b) % m == 0 and np.unique((A0 + b * A1) % m).size == m:
                    self.rank[m], self.kind[m], self.base[m] = 3, "school3", b
                    found = True
                    break
            if found:
                continue
            for kind, X0, X1, rank in (("toom", T0, T1, 3), ("school4", A0, A1, 4)):
                if X0.size < m:
                    continue
                for b in range(2, m):
                    if np.unique((X0 + b * X1) % m).size == m:
                        self.rank[m], self.kind[m], self.base[m] = rank, kind, b
                        found = True
                        break
                if found:
                    break


def _prime_factors(n):
    out, d = set(), 2
    while d * d <= n:
        while n % d == 0:
            out.add(d)
            n //= d
        d += 1
    if n > 1:
        out.add(n)
    return out


def least_q(rank, K, beta=53):
    """The reduced program eq. ov-reduced by the five steps; returns (Q, moduli)."""
    need = 2 * K * (2**beta - 1) ** 2

    def solve(members):
        fac = {m: _prime_factors(m) for m in members}
        tau = 1
        for m in members:
            big = sorted(fac[m])
            if len(big) >= 2:
                tau = max(tau, big[-2])
        # step 1
        H = [m for m in members if len(fac[m]) == 1 and m == max(fac[m]) and m > tau]
        L = [m for m in members if m not in set(H)]
        P = sorted({p for m in L for p in fac[m] if p <= tau})
        pbit = {p: 1 << i for i, p in enumerate(P)}
        # step 2: 0/1 knapsack over H by cost, largest product
        bestH = {0: (1, ())}
        for m in H:
            for c, (prod, sel) in sorted(bestH.items(), reverse=True):
                nc = c + rank[m]
                cand = (prod * m, sel + (m,))
                if nc not in bestH or cand[0] > bestH[nc][0]:
                    bestH[nc] = cand
        # monotone: a larger budget may use fewer
        # step 3: program over subsets of P
        state = {(0, 0): (1, ())}
        for m in L:
            mk = 0
            for p in fac[m]:
                if p <= tau:
                    mk |= pbit[p]
            for (mask, c), (prod, sel) in list(state.items()):
                if mask & mk:
                    continue
                key = (mask | mk, c + rank[m])
                cand = (prod * m, sel + (m,))
                if key not in state or cand[0] > state[key][0]:
                    state[key] = cand
        bestL = {}
        for (mask, c), val in state.items():
            if c not in bestL or val[0] > bestL[c][0]:
                bestL[c] = val
        # step 4
        best = None
        for ch, (ph, sh) in bestH.items():
            for cl, (pl, sl) in bestL.items():
                if ph * pl > need:
                    key = (ch + cl, -(ph * pl))
                    if best is None or key < best[0]:
                        best = (key, sh + sl)
        if best is None:
            return None
        chosen = best[1]
        # step 5: a prime above tau shared by two chosen members
        for i, a in enumerate(chosen):
            for b2 in chosen[i + 1:]:
                shared = {p for p in fac[a] & fac[b2] if p > tau}
                if shared:
                    r1 = solve([m for m in members if m != a])
                    r2 = solve([m for m in members if m != b2])
                    cands = [r for r in (r1, r2) if r is not None]
                    return min(cands, key=lambda r: (r[0], -math.prod(r[1])))
        return (best[0][0], tuple(sorted(chosen, reverse=True)))

    return solve(sorted(rank))


def tables(name, K, m, kind, b, lam=LAMBDA_FP32):
    """Plane value tables [plane][class] of one channel, by enumeration."""
    S, _ = alphabet(name)
    r = rmax1(K, lam)
    Sr = [s for s in S if abs(s) <= r]
    if kind == "one":
        out = [None] * m
        for v in sorted(Sr, key=lambda v: (abs(v), v)):
            if out[v % m] is None:
                out[v % m] = v
        assert None not in out
        return [out]
    Sset = set(Sr)
    best = [None] * m
    for a0 in Sr:
        for a1 in Sr:
            if kind == "toom" and (a0 + a1) not in Sset:
                continue
            size = max(abs(a0), abs(a1), abs(a0 + a1)) if kind == "toom" else max(abs(a0), abs(a1))
            key = (size, abs(a1), a1, a0)
            c = (a0 + b * a1) % m
            if best[c] is None or key < best[c][0]:
                best[c] = (key, a0, a1)
    assert None not in best
    if kind == "toom":
        return [[x[1] for x in best], [x[1] + x[2] for x in best], [x[2] for x in best]]
    return [[x[1] for x in best], [x[2] for x in best]]


def weights(kind, b):
    """(plane of A, plane of B, lambda) per GEMM of a channel's form."""
    if kind == "one":
        return [(0, 0, 1)]
    if kind == "school3":
        return [(0, 0, 1), (0, 1, b), (1, 0, b)]
    if kind == "toom":
        return [(0, 0, 1 - b), (1, 1, b), (2, 2, b * b - b)]
    return [(0, 0, 1), (0, 1, b), (1, 0, b), (1, 1, b * b)]


def code_values(name):
    """{code: scaled alphabet value} for every finite code of an OCP format:
    sign bit on top, then the exponent field, then the mantissa field; the
    value is (-1)^sign 2^(1 - bias) (mantissa / 2^m_bits) for a zero exponent
    field and (-1)^sign 2^(e - bias) (1 + mantissa / 2^m_bits) otherwise,
    times 2^e_S."""
    eb, mb, bias, style = SPECS[name]
    _, e_s = alphabet(name)
    out = {}
    for sign in (0, 1):
        for e in range(2**eb):
            for mt in range(2**mb):
                if style == "ieee" and e == 2**eb - 1:
                    continue
                if style == "fn" and e == 2**eb - 1 and mt == 2**mb - 1:
                    continue
                mag = Fraction(mt, 2**mb) * Fraction(2) ** (1 - bias) if e == 0 else \
                    (1 + Fraction(mt, 2**mb)) * Fraction(2) ** (e - bias)
                v = mag * 2**e_s
                assert v.denominator == 1
                out[(sign << (eb + mb)) | (e << mb) | mt] = -int(v) if sign else int(v)
    return out
