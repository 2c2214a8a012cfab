"""Forward + backward time of the emulated matmul (EmuMatmul: C = A B, then
dA = dC B^T and dB = A^T dC through the same emulated kernels) against torch
float64 autograd, at m = n = k = 4096 and m = 65536, k = n = 256.

    python tests/autograd_timing.py

Operands and dC ~ N(0, 1) (torch generator seeded 0). Each figure is the best
of three timed fwd+bwd passes after one untimed pass; TFLOP/s counts the three
products, 3 * 2mnk.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import paper_2609_37693_gb300 as oz  # noqa: E402


def tm(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def main():
    for (m, k, n) in ((4096, 4096, 4096), (65536, 256, 256)):
        g = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn(m, k, dtype=torch.float64, device="cuda", generator=g).requires_grad_()
        B = torch.randn(k, n, dtype=torch.float64, device="cuda", generator=g).requires_grad_()
        dC = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)

        def emu():
            A.grad = None
            B.grad = None
            oz.EmuMatmul.apply(A, B).backward(dC)

        def nat():
            A.grad = None
            B.grad = None
            (A @ B).backward(dC)

        te, tn = tm(emu), tm(nat)
        fl = 3 * 2.0 * m * n * k
        print(f"autograd m={m} k={k} n={n}: emulated fwd+bwd {te:.2f} ms ({fl / te / 1e9:.1f} TFLOP/s), "
              f"float64 autograd {tn:.2f} ms ({fl / tn / 1e9:.2f} TFLOP/s)", flush=True)


if __name__ == "__main__":
    main()
