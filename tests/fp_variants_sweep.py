"""Per-format report of the float-format configurations (E4M3, E5M2, E2M3,
E3M2, E2M1) next to the INT8 path: GEMM count Q, channels, bit budget beta,
error against the exact product, emulated TFLOP/s, time of the GEMM phase and
cuBLAS DGEMM on the same operands.

Error: max and median over sampled entries of |C - AB|_ij / (u (|A||B|)_ij),
u = 2^-53 (exact difference from the oracle's fixed-point accumulator). Each
timed product is first checked bit for bit against the oracle on the sampled
entries. Each format runs at the largest beta its window allows at K = n and
at the paper's 53 bits.

    python tests/fp_variants_sweep.py --n 8192 --phi 0.5 2 --md fp.md

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
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from precision_sweep import U, time_call  # noqa: E402

FORMATS = ["E4M3", "E5M2", "E2M3", "E3M2", "E2M1"]


def sweep(ns, phis, formats, samples, reps=5, log=print):
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
            ms = time_call(lambda: Ad @ Bd, 2)
            dg = 2.0 * n**3 / (ms * 1e-3) / 1e12
            for fmt in ["INT8"] + list(formats):
                for bits in (0, 53):
                    plan = oz.Plan(16, bits, n) if fmt == "INT8" else oz.PlanFP(fmt, n, bits)
                    ws = oz.workspace(plan, n, n, n)
                    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
                    oz.dgemm(Ad, Bd, plan, out=C, ws=ws)
                    Ch = C.cpu().numpy()
                    ref = oracle.dgemm_entries(A, B, plan.moduli, plan.bits, r, c)
                    exact = bool(np.array_equal(Ch[r, c].view(np.uint64), ref.view(np.uint64)))
                    ms = time_call(lambda: oz.dgemm(Ad, Bd, plan, out=C, ws=ws), reps)
                    lay = oz.oz_workspace_layout(plan.handle, n, n, n)[1]
                    base = ws.data_ptr()
                    gms = time_call(lambda: oz.oz_residue_gemm(
                        plan.handle, n, n, lay["m_pad"], lay["n_pad"], lay["k_pad"], base + lay["u"],
                        base + lay["v"], base + lay["y"], 0, base + lay["flag"], oz._stream_handle()), reps)
                    err, ab = oracle.exact_error(A, B, Ch, r, c)
                    rel = np.where(ab > 0, err / (U * np.where(ab > 0, ab, 1.0)), np.where(err > 0, np.inf, 0.0))
                    row = {"n": n, "phi": phi, "format": fmt, "q": plan.q,
                           "channels": getattr(plan, "channels", plan.q), "bits": plan.bits,
                           "bit_exact_vs_oracle": exact, "max_err_u": float(rel.max()),
                           "median_err_u": float(np.median(rel)), "ms": ms,
                           "tflops": 2.0 * n**3 / (ms * 1e-3) / 1e12, "gemm_ms": gms,
                           "gemm_lp_tflops": 2.0 * n**3 * plan.q / (gms * 1e-3) / 1e12,
                           "dgemm_tflops": dg, "samples": int(len(r))}
                    rows.append(row)
                    log(json.dumps(row))
                    del C, ws
                    torch.cuda.empty_cache()
            del Ad, Bd
            torch.cuda.empty_cache()
    return rows


def markdown(rows):
    out = ["| n | phi | format | Q (GEMMs) | channels | bits | bit-exact | max err [u·(|A||B|)] | median err | "
           "ms | TFLOP/s | GEMM ms | GEMM TFLOP/s (low precision) | DGEMM TFLOP/s |",
           "|---|---|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        out.append(f"| {r['n']} | {r['phi']} | {r['format']} | {r['q']} | {r['channels']} | {r['bits']} | "
                   f"{'yes' if r['bit_exact_vs_oracle'] else 'NO'} | {r['max_err_u']:.3g} | {r['median_err_u']:.3g} | "
                   f"{r['ms']:.2f} | {r['tflops']:.1f} | {r['gemm_ms']:.2f} | {r['gemm_lp_tflops']:.0f} | "
                   f"{r['dgemm_tflops']:.2f} |")
    return "\n".join(out) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[8192])
    ap.add_argument("--phi", type=float, nargs="+", default=[0.5, 2.0])
    ap.add_argument("--formats", nargs="+", default=FORMATS)
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=None)
    ap.add_argument("--md", default=None)
    a = ap.parse_args()
    t0 = time.time()
    rows = sweep(a.n, a.phi, a.formats, a.samples, a.reps)
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
