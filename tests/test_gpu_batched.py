"""Batched uneven products (one oz_dgemm_batched call, optionally one CUDA
graph) and grouped products (one launch per phase): every product equals the
oracle's, bit for bit (Sec. "Emulation Problem": C = fl(2^-(s+t) A'B') for
each problem at its plan's bit budget)."""
import numpy as np
import pytest

import synth
from tests.oracle_check import assert_oracle_bits

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


def _check_oracle(shapes, As, Bs, Cs, plans, what):
    """Every product against the oracle at its own plan's moduli and bits."""
    for i, ((m, n, k), A, B, C, p) in enumerate(zip(shapes, As, Bs, Cs, plans)):
        assert_oracle_bits(C, A, B, p.moduli, p.bits, what=f"{what}, problem {i}", seed=i)


@pytest.mark.parametrize("nstreams", [1, 3])
def test_batched_equals_individual_products(nstreams):
    shapes, As, Bs, Cs = _problems(24, 1, 700, seed=3)
    bg = oz.BatchedGemm(shapes, nstreams=nstreams)
    # least Q at 53 bits: kappa_rec is 4 at Q = 14, 836 at Q = 15, 159 819 at Q = 16
    assert [p.q for p in bg.plans] == [14 if k <= 4 else 15 if k <= 836 else 16 for (_, _, k) in shapes]
    bg.run(As, Bs, Cs)
    torch.cuda.synchronize()
    _check_oracle(shapes, As, Bs, Cs, bg.plans, f"batched, {nstreams} streams")


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
        _check_oracle(shapes, As, Bs, Cs, bg.plans, f"batched graph, replay {rnd}")


def test_autotuner_picks_a_stream_count():
    shapes, As, Bs, Cs = _problems(12, 64, 512, seed=5)
    bg, timings = oz.autotune_batched(shapes, As, Bs, Cs, candidates=(1, 2, 4))
    assert set(timings) == {1, 2, 4} and bg.nstreams == min(timings, key=timings.get)
    torch.cuda.synchronize()
    _check_oracle(shapes, As, Bs, Cs, bg.plans, "autotuned streams")


# ---- grouped products: one launch per phase (oz_group_create / oz_group_run) ----

def _edge_problems():
    """Uneven shapes with the edge cases of the grouped path: 1 x 1 x 1, one
    row, one column, k = 0, k at a slab boundary, k on either side of the
    split of A's switch from one warp per row to one block per row (4096),
    ragged tiles, Q = 14/15/16."""
    shapes = [(1, 1, 1), (1, 300, 77), (300, 1, 77), (5, 7, 0), (130, 257, 1024), (129, 255, 1025),
              (64, 64, 3), (700, 513, 900), (256, 256, 5000), (33, 1000, 837), (41, 70, 4096),
              (9, 33, 4097)]
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.phi_pair(m, n, k, 1.5, seed=300 + i)
        As.append(torch.from_numpy(A).to(DEV))
        Bs.append(torch.from_numpy(B).to(DEV))
        Cs.append(torch.full((m, n), np.nan, dtype=torch.float64, device=DEV))
    return shapes, As, Bs, Cs


@pytest.mark.parametrize("which", ["uneven", "edges"])
def test_grouped_equals_individual_products(which):
    shapes, As, Bs, Cs = _problems(40, 1, 1500, seed=6) if which == "uneven" else _edge_problems()
    gg = oz.GroupedGemm(As, Bs, Cs)
    assert sorted({p.q for p in gg.plans}) == sorted({14 if k <= 4 else 15 if k <= 836 else 16
                                                        for (_, _, k) in shapes})
    gg.run()
    torch.cuda.synchronize()
    assert oz.query_status(gg.ws) == oz.OZ_OK
    _check_oracle(shapes, As, Bs, Cs, gg.plans, f"grouped ({which})")


def test_grouped_graph_replays_on_new_inputs():
    shapes, As, Bs, Cs = _problems(20, 16, 2000, seed=7)
    gg = oz.GroupedGemm(As, Bs, Cs)
    gg.capture()
    for rnd in range(2):
        for i, (A, B) in enumerate(zip(As, Bs)):
            m, k = A.shape
            n = B.shape[1]
            a, b = synth.phi_pair(m, n, k, 2.0, seed=2000 * (rnd + 1) + i)
            A.copy_(torch.from_numpy(a))
            B.copy_(torch.from_numpy(b))
        gg.replay()
        torch.cuda.synchronize()
        _check_oracle(shapes, As, Bs, Cs, gg.plans, f"grouped graph, replay {rnd}")


def test_grouped_reports_nonfinite():
    shapes, As, Bs, Cs = _problems(6, 32, 300, seed=8)
    As[2][0, 0] = float("nan")
    Bs[4][-1, -1] = float("inf")
    gg = oz.GroupedGemm(As, Bs, Cs)
    gg.run()
    assert oz.query_status(gg.ws) == oz.OZ_ERR_NONFINITE


def test_autotuned_batch_structures_agree():
    """Every candidate of the batch autotuner (streams, grouped at the least Q,
    grouped with every product on Q = 16) keeps 53 bits, so each returns the
    oracle's products at 53 bits; the autotuner keeps the fastest."""
    shapes, As, Bs, Cs = _problems(20, 16, 1200, seed=9)
    least = [oz.plan_least_q(k, 53) for (_, _, k) in shapes]
    runner, label, times = oz.autotune_batch(shapes, As, Bs, Cs, streams=(1, 4), reps=1)
    assert set(times) == {"streams=1", "streams=4", "streams=1 pairs", "grouped", "grouped q=16"} and label in times
    for C in Cs:
        C.fill_(np.nan)
    runner.replay()
    torch.cuda.synchronize()
    _check_oracle(shapes, As, Bs, Cs, least, f"autotuned batch ({label})")
    q16 = oz.Plan(16, 53, 1200, oz.OZ_ENGINE_TC)
    gq = oz.GroupedGemm(As, Bs, Cs, plans=[q16] * len(shapes))
    for C in Cs:
        C.fill_(np.nan)
    gq.run()
    torch.cuda.synchronize()
    assert gq.launches() <= 7
    _check_oracle(shapes, As, Bs, Cs, least, "grouped, every product on Q = 16")
