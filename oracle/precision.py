"""Error tables of the emulated product, from the oracle alone (no GPU).

TEST INFRASTRUCTURE, like the rest of oracle/: a report tool, run by hand.

    python -m oracle.precision --n 8192 16384
    python -m oracle.precision --n 8192 --operands paper --q 14 15 16 17 18 19 20
    python -m oracle.precision --n 1024 4096 8192 --operands phi0.5 phi1 phi2 phi4 --q 10 12 14 16 18 20

Every configuration of the library returns the oracle's bits at its modulus
set and bit budget (the GPU parity tests check this entry by entry, at 8192
too), and within the window the result depends on beta alone, not on the
moduli or the alphabet (Sec. "Emulation Problem": C = fl(2^-(s+t) A'B')). So
these are the errors of the GPU results, for the INT8 path and every float
format at the same beta. Row i of op(A) and column j of op(B) hold everything
entry (i, j) depends on (its shifts included), so the sampled rows of A and
columns of B are multiplied on their own. For each sampled entry the error is
|C_ij - (AB)_ij|, formed exactly and rounded once, in units of u (|A||B|)_ij
with u = 2^-53.

Operand families (synth):
* phiX: entries U(-0.5, 0.5) exp(X N(0, 1));
* paper: the paper's timing operands (Table tab:setup), row i of each operand
  N(0, 1) 2^e_i with e_i an integer drawn from [-20, 20).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import synth  # noqa: E402


def errors(A, B, mods, beta, rows, cols):
    """|C - AB| / (u |A||B|) on the grid rows x cols (row-major)."""
    As = np.ascontiguousarray(A[rows, :])
    Bs = np.ascontiguousarray(B[:, cols])
    C = oracle.dgemm(As, Bs, mods, beta)
    r, c = np.divmod(np.arange(len(rows) * len(cols)), len(cols))
    err, ab = oracle.exact_error(As, Bs, C, r, c)
    return err / (2.0**-53 * ab)


def operands(name, n):
    if name == "paper":
        return synth.row_scaled_pair(n, seed=0)
    return synth.phi_pair(n, n, n, float(name[3:]), seed=0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[8192, 16384])
    ap.add_argument("--operands", nargs="+", default=["phi0.5", "paper"])
    ap.add_argument("--q", type=int, nargs="+", default=[16])
    ap.add_argument("--rows", type=int, default=256)
    ap.add_argument("--cols", type=int, default=256)
    args = ap.parse_args()
    print("| n | operands | Q | beta | entries | max error / u(|A||B|) | median | share above 2 |")
    print("|---|---|---|---|---|---|---|---|")
    for n in args.n:
        rng = np.random.default_rng(2)
        rows = np.sort(rng.choice(n, size=min(args.rows, n), replace=False))
        cols = np.sort(rng.choice(n, size=min(args.cols, n), replace=False))
        for ops in args.operands:
            A, B = operands(ops, n)
            for q in args.q:
                mods = oracle.max_product_moduli(q, 239)
                bmax = min(oracle.beta_max(mods, n), 80)
                # the paper's 53 where the window admits it, and the widest beta
                for beta in sorted({b for b in (53, bmax) if b <= bmax}):
                    t = time.time()
                    rel = errors(A, B, mods, beta, rows, cols)
                    print(f"| {n} | {ops} | {q} | {beta} | {rel.size} | {rel.max():.3g} | {np.median(rel):.3g} | "
                          f"{np.mean(rel > 2):.3g} |", flush=True)
                    print(f"  ({time.time() - t:.1f} s)", file=sys.stderr)
            del A, B


if __name__ == "__main__":
    main()
