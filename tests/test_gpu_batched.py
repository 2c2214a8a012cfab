"""Batched uneven products (one oz_dgemm_batched call, optionally one CUDA
graph): every product equals the one oz_dgemm computes alone, bit for bit."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2609_37693_gb300 as oz  # noqa: E402

DEV = torch.device("cuda:0")


def _problems(count, lo, hi, seed):
    shapes = [tuple(int(x) for x in s) for s in synth.batch_shapes(count, lo, hi, seed)]
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.phi_pair(m, n, k, 1.0, seed=100 + i)
        As.append(torch.from_numpy(A).to(DEV))
        Bs.append(torch.from_numpy(B).to(DEV))
        Cs.append(torch.full((m, n), np.nan, dtype=torch.float64, device=DEV))
    return shapes, As, Bs, Cs


def _alone(shapes, As, Bs, plans):
    out = []
    for (m, n, k), A, B, p in zip(shapes, As, Bs, plans):
        out.append(oz.dgemm(A, B, p).cpu().numpy())
    return out


@pytest.mark.parametrize("nstreams", [1, 3])
def test_batched_equals_individual_products(nstreams):
    shapes, As, Bs, Cs = _problems(24, 1, 700, seed=3)
    bg = oz.BatchedGemm(shapes, nstreams=nstreams)
    # least Q at 53 bits: kappa_rec is 4 at Q = 14, 836 at Q = 15, 159 819 at Q = 16
    assert [p.q for p in bg.plans] == [14 if k <= 4 else 15 if k <= 836 else 16 for (_, _, k) in shapes]
    bg.run(As, Bs, Cs)
    torch.cuda.synchronize()
    ref = _alone(shapes, As, Bs, bg.plans)
    for C, R in zip(Cs, ref):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), R.view(np.uint64))


def test_graph_capture_replays_on_new_inputs():
    shapes, As, Bs, Cs = _problems(16, 64, 1500, seed=4)
    bg = oz.BatchedGemm(shapes, nstreams=4)
    bg.capture(As, Bs, Cs)
    for rnd in range(2):
        for i, (A, B) in enumerate(zip(As, Bs)):      # new values in the captured buffers
            m, k = A.shape
            n = B.shape[1]
            a, b = synth.phi_pair(m, n, k, 2.0, seed=1000 * (rnd + 1) + i)
            A.copy_(torch.from_numpy(a))
            B.copy_(torch.from_numpy(b))
        bg.replay()
        torch.cuda.synchronize()
        ref = _alone(shapes, As, Bs, bg.plans)
        for C, R in zip(Cs, ref):
            assert np.array_equal(C.cpu().numpy().view(np.uint64), R.view(np.uint64))


def test_autotuner_picks_a_stream_count():
    shapes, As, Bs, Cs = _problems(12, 64, 512, seed=5)
    bg, timings = oz.autotune_batched(shapes, As, Bs, Cs, candidates=(1, 2, 4))
    assert set(timings) == {1, 2, 4} and bg.nstreams == min(timings, key=timings.get)
    torch.cuda.synchronize()
    ref = _alone(shapes, As, Bs, bg.plans)
    for C, R in zip(Cs, ref):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), R.view(np.uint64))
