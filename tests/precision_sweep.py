"""Precision / throughput sweep of the emulated product.

For every size n, exponent spread phi and modulus count Q it reports the
error against the exact product, max and median of
|C - AB|_ij / (u (|A||B|)_ij) with u = 2^-53 over sampled entries (the exact
difference comes from the oracle's fixed-point accumulator), the emulated
TFLOP/s (2 n^3 / time) and cuBLAS DGEMM's TFLOP/s on the same operands. Each Q
runs at the largest bit budget its window allows at K = n, and also at the
paper's 53 bits where the window holds.

    python tests/precision_sweep.py --n 1024 4096 8192 16384 --phi 0.5 1 2 4 \
        --q 10 11 12 13 14 15 16 17 18 19 20 --out sweep.jsonl --md sweep.md

Operands: U(-0.5, 0.5) * exp(phi * N(0, 1)), seed 0 (synth.phi_pair).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

U = 2.0**-53


def time_call(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def sweep(ns, phis, qs, samples, reps=3, dgemm=True, log=print):
    import torch

    import oracle
    import paper_2609_37693_gb300 as oz
    import synth
    rows = []
    for n in ns:
        for phi in phis:
            A, B = synth.phi_pair(n, n, n, phi, seed=0)
            Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            r, c = synth.sample_entries(n, n, samples, seed=7)
            dg = None
            if dgemm:
                ms = time_call(lambda: Ad @ Bd, 2)
                dg = 2.0 * n**3 / (ms * 1e-3) / 1e12
            for q in qs:
                mods = oracle.max_product_moduli(q, 239)
                bmax = min(oracle.beta_max(mods, n), oz.OZ_MAX_BITS)
                betas = [bmax] + ([53] if 53 < bmax else [])
                for beta in betas:
                    try:
                        plan = oz.Plan(q, beta, n)
                    except oz.OzError as e:
                        log(f"n={n} phi={phi} Q={q} beta={beta}: {e}")
                        continue
                    ws = oz.workspace(plan, n, n, n)
                    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
                    ms = time_call(lambda: oz.dgemm(Ad, Bd, plan, out=C, ws=ws), reps)
                    Ch = C.cpu().numpy()
                    err, ab = oracle.exact_error(A, B, Ch, r, c)
                    rel = np.where(ab > 0, err / (U * np.where(ab > 0, ab, 1.0)), np.where(err > 0, np.inf, 0.0))
                    row = {"n": n, "phi": phi, "q": q, "bits": beta, "max_err_u": float(rel.max()),
                           "median_err_u": float(np.median(rel)), "tflops": 2.0 * n**3 / (ms * 1e-3) / 1e12,
                           "ms": ms, "dgemm_tflops": dg, "samples": int(len(r))}
                    rows.append(row)
                    log(json.dumps(row))
                    del C, ws
            del Ad, Bd
            torch.cuda.empty_cache()
    return rows


def markdown(rows):
    out = ["| n | phi | Q | bits | max err [u·(|A||B|)] | median err | TFLOP/s | DGEMM TFLOP/s |",
           "|---|---|---|---|---|---|---|---|"]
    for r in rows:
        dg = f"{r['dgemm_tflops']:.2f}" if r["dgemm_tflops"] else "-"
        out.append(f"| {r['n']} | {r['phi']} | {r['q']} | {r['bits']} | {r['max_err_u']:.3g} | "
                   f"{r['median_err_u']:.3g} | {r['tflops']:.1f} | {dg} |")
    return "\n".join(out) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[1024, 4096, 8192])
    ap.add_argument("--phi", type=float, nargs="+", default=[0.5, 1.0, 2.0, 4.0])
    ap.add_argument("--q", type=int, nargs="+", default=list(range(10, 21)))
    ap.add_argument("--samples", type=int, default=16384)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None)
    ap.add_argument("--md", default=None)
    a = ap.parse_args()
    t0 = time.time()
    rows = sweep(a.n, a.phi, a.q, a.samples, a.reps)
    if a.out:
        with open(a.out, "w") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")
    if a.md:
        with open(a.md, "w") as f:
            f.write(markdown(rows))
    print(f"done in {time.time() - t0:.0f} s", file=sys.stderr)


if __name__ == "__main__":
    main()
