"""The C-ABI library without a GPU: it builds, loads, exports every symbol the
header declares, and its host-side logic (plans, caps, workspace sizes,
argument checks) is right. No call here launches a kernel."""
import ctypes
import os
import re

import pytest

import oracle
import paper_2609_37693_gb300 as oz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "oz.h")).read()
    return sorted(set(re.findall(r"OZ_API\s+[\w\s\*]+?\b(oz_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = _declared_symbols()
    assert len(names) >= 10
    lib = ctypes.CDLL(oz.LIBRARY_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(oz.EXPORTED)


@pytest.mark.parametrize("q", range(9, 21))
def test_plan_moduli_caps_and_bits_match_the_oracle(q):
    for k_hint in (256, 4096, 8192):
        st, h = oz.oz_plan_create(q, 0, k_hint, oz.OZ_ENGINE_IMMA)
        mods = oracle.max_product_moduli(q, 239)
        bmax = min(oracle.beta_max(mods, k_hint), oz.OZ_MAX_BITS)
        if bmax < 1 or oracle.caps(mods, bmax)[2] < k_hint:
            assert st == oz.OZ_ERR_K_TOO_LARGE
            continue
        assert st == oz.OZ_OK
        _, info = oz.oz_plan_info(h)
        assert info["moduli"] == mods
        assert info["bits"] == bmax
        assert info["k_max"] == oracle.caps(mods, bmax)[2]
        oz.oz_plan_destroy(h)


def test_paper_int8_plan():
    st, h = oz.oz_plan_create(16, 53, 8192, oz.OZ_ENGINE_IMMA)
    assert st == oz.OZ_OK
    _, info = oz.oz_plan_info(h)
    assert info["k_max"] == 151647 and max(info["moduli"]) == 239
    oz.oz_plan_destroy(h)
    # least Q at beta = 53 (num_moduli = 0): 15 up to K = 836, then 16
    for k, q in ((800, 15), (836, 15), (837, 16), (151647, 16)):
        st, h = oz.oz_plan_create(0, 53, k, oz.OZ_ENGINE_IMMA)
        assert st == oz.OZ_OK
        assert oz.oz_plan_info(h)[1]["q"] == q
        oz.oz_plan_destroy(h)
    # above K_max: refused (eq. caps), as the paper's builder refuses K above kappa_rec
    assert oz.oz_plan_create(16, 53, 151648, oz.OZ_ENGINE_IMMA)[0] == oz.OZ_ERR_K_TOO_LARGE
    # Q = 14 at beta = 53 is infeasible at K = 256 (kappa_rec = 4), feasible at beta = 50
    assert oz.oz_plan_create(14, 53, 256, oz.OZ_ENGINE_IMMA)[0] == oz.OZ_ERR_K_TOO_LARGE
    assert oz.oz_plan_create(14, 50, 256, oz.OZ_ENGINE_IMMA)[0] == oz.OZ_OK


def test_bad_plans_are_refused():
    assert oz.oz_plan_create(8, 0, 100)[0] == oz.OZ_ERR_UNSUPPORTED
    assert oz.oz_plan_create(21, 0, 100)[0] == oz.OZ_ERR_UNSUPPORTED
    assert oz.oz_plan_create(16, oz.OZ_MAX_BITS + 1, 100)[0] == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_plan_create(16, 65, 100)[0] == oz.OZ_ERR_K_TOO_LARGE        # the window, not the budget
    st, h = oz.oz_plan_create(20, 70, 100)                                   # widened (beta > 64)
    assert st == oz.OZ_OK
    oz.oz_plan_destroy(h)
    assert oz.oz_plan_create_fp(oz.OZ_FMT_E4M3, 100, oz.OZ_MAX_BITS_FP + 1)[0] == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_plan_create(16, 0, 0)[0] == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_plan_create(16, 0, 100, 7)[0] == oz.OZ_ERR_INVALID_ARG


def test_workspace_bytes():
    p = oz.Plan(16, 0, 1000, oz.OZ_ENGINE_IMMA)
    m, n, k = 300, 200, 1000
    ws = p.workspace_bytes(m, n, k)
    planes = 16 * (512 + 256) * 1024
    bt = 8 * n * k                     # B transposed, so that its columns split as rows
    assert ws >= planes + 16 * m * n + bt
    assert ws < planes + 16 * m * n + bt + 64 * 1024
    assert p.workspace_bytes(-1, 2, 3) == 0


def test_argument_errors_are_caught_on_the_host():
    p = oz.Plan(16, 0, 1000, oz.OZ_ENGINE_IMMA)
    h = p.handle
    fake = 1 << 20  # never dereferenced: every case fails its checks before a launch
    ws = p.workspace_bytes(8, 8, 8)
    assert oz.oz_dgemm(h, 0, 0, -1, 8, 8, fake, 8, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_dgemm(h, 2, 0, 8, 8, 8, fake, 8, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 8, fake, 7, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 8, fake, 8, fake, 8, fake, 7, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 200000, fake, 200000, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_K_TOO_LARGE
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 8, fake, 8, fake, 8, fake, 8, fake, ws - 1, None) == oz.OZ_ERR_WORKSPACE
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 8, fake, 8, fake, 8, fake, 8, None, ws, None) == oz.OZ_ERR_WORKSPACE
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 8, None, 8, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_dgemm(h, 0, 0, 8, 8, 8, fake + 4, 8, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_dgemm(None, 0, 0, 8, 8, 8, fake, 8, fake, 8, fake, 8, fake, ws, None) == oz.OZ_ERR_INVALID_ARG
    # empty products succeed without touching memory
    assert oz.oz_dgemm(h, 0, 0, 0, 8, 8, None, 8, None, 8, None, 8, None, 0, None) == oz.OZ_OK
    assert oz.oz_split(h, 1, 4, 4, fake, 4, 100, 128, fake, fake, None, None, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_split(h, 0, 4, 4, fake, 4, 256, 128, fake, fake, None, None, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_residue_gemm(h, 4, 4, 256, 256, 100, fake, fake, fake, 0, None, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_reconstruct(h, 4, 4, fake, fake, fake, fake, 3, None) == oz.OZ_ERR_INVALID_ARG


def test_status_strings():
    for s in range(7):
        assert oz.oz_status_str(s) and oz.oz_status_str(s) != "unknown status"


def test_batched_workspace_and_argument_checks():
    plans = [oz.Plan(16, 0, 1000, oz.OZ_ENGINE_IMMA), oz.Plan(15, 53, 500, oz.OZ_ENGINE_IMMA)]
    shapes = [(300, 200, 1000), (64, 64, 500), (1000, 10, 100)]
    parr = (ctypes.c_void_p * 3)(plans[0].handle, plans[1].handle, plans[1].handle)
    mnk = (ctypes.c_int64 * 9)(*[x for s in shapes for x in s])
    one = oz.oz_batched_workspace_bytes(3, parr, mnk, 1)
    assert one >= max(p.workspace_bytes(*s) for p, s in zip([plans[0], plans[1], plans[1]], shapes))
    two = oz.oz_batched_workspace_bytes(3, parr, mnk, 2)
    assert two % 2 == 0 and two >= one
    assert oz.oz_batched_workspace_bytes(3, parr, mnk, 0) == 0
    fake = 1 << 20
    P = ctypes.c_void_p
    ptrs = (P * 3)(fake, fake, fake)
    lds = (ctypes.c_int64 * 3)(1000, 500, 100)
    ldb = (ctypes.c_int64 * 3)(200, 64, 10)
    ldc = (ctypes.c_int64 * 3)(200, 64, 10)
    streams = (P * 1)(None)
    # short workspace, bad leading dimension, K above a plan's K_max: refused before any launch
    assert oz.oz_dgemm_batched(3, parr, mnk, None, ptrs, lds, ptrs, ldb, ptrs, ldc, fake, one - 256, streams,
                               1) == oz.OZ_ERR_WORKSPACE
    bad = (ctypes.c_int64 * 3)(1000, 499, 100)
    assert oz.oz_dgemm_batched(3, parr, mnk, None, ptrs, bad, ptrs, ldb, ptrs, ldc, fake, one, streams,
                               1) == oz.OZ_ERR_INVALID_ARG
    mnk_big = (ctypes.c_int64 * 9)(300, 200, 1000, 64, 64, 5000, 1000, 10, 100)
    big = oz.oz_batched_workspace_bytes(3, parr, mnk_big, 1)
    lda_big = (ctypes.c_int64 * 3)(1000, 5000, 100)
    assert oz.oz_dgemm_batched(3, parr, mnk_big, None, ptrs, lda_big, ptrs, ldb, ptrs, ldc, fake, big, streams,
                               1) == oz.OZ_ERR_K_TOO_LARGE
    assert oz.oz_dgemm_batched(0, parr, mnk, None, ptrs, lds, ptrs, ldb, ptrs, ldc, None, 0, streams, 1) == oz.OZ_OK


def test_grouped_refuses_unsupported_plans_before_any_work():
    """oz_group_create takes INT8 plans of a BF16 engine only; a float-format or
    IMMA plan is refused on the host, before any pointer is used."""
    import ctypes
    fp = oz.PlanFP("E4M3", 1000)
    imma = oz.Plan(16, 0, 1000, oz.OZ_ENGINE_IMMA)
    tc = oz.Plan(16, 0, 1000, oz.OZ_ENGINE_TC)
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    mnk = (I64 * 3)(64, 64, 64)
    for plan, want in ((fp, oz.OZ_ERR_UNSUPPORTED), (imma, oz.OZ_ERR_UNSUPPORTED)):
        arr = (P * 1)(plan.handle)
        assert oz._lib.oz_grouped_workspace_bytes(1, arr, mnk) == 0
        h = P()
        st = oz._lib.oz_group_create(ctypes.byref(h), 1, arr, mnk, None, None, None, None, None, None, None, 0)
        assert st == oz.OZ_ERR_INVALID_ARG           # null operand arrays are checked first
        one = (P * 1)(None)
        ld = (I64 * 1)(64)
        st = oz._lib.oz_group_create(ctypes.byref(h), 1, arr, mnk, one, ld, one, ld, one, ld, None, 0)
        assert st == want and not h.value
    arr = (P * 1)(tc.handle)
    assert oz._lib.oz_grouped_workspace_bytes(1, arr, mnk) > 0


@pytest.mark.parametrize("q", range(14, 21))
def test_plan_caps_match_the_oracle(q):
    """oz_plan_caps reports the two caps of eq. caps separately: on the IMMA
    engine k_acc is the INT32 accumulation cap and k_rec the window of eq.
    ov-crtgen, as the oracle computes them; the TC engine drains its FP32 slabs
    and has no accumulation cap below 2^31."""
    mods = oracle.max_product_moduli(q, 239)
    k_rec, k_acc, _ = oracle.caps(mods, 53)
    p = oz.Plan(q, 53, 1, oz.OZ_ENGINE_IMMA)
    assert (p.k_acc, p.k_rec) == (k_acc, k_rec)
    t = oz.Plan(q, 53, 1, oz.OZ_ENGINE_TC)
    assert (t.k_acc, t.k_rec) == (2**31 - 1, k_rec)


def test_paper_int8_caps():
    """Sec. "INT4 and INT8": K_max = 151 647 at Q = 16 comes from the INT32
    accumulator; the window alone admits 159 819 at beta = 53."""
    p = oz.Plan(16, 53, 8192, oz.OZ_ENGINE_IMMA)
    assert (p.k_acc, p.k_rec, p.k_max) == (151647, 159819, 151647)


def test_blocked_argument_errors_are_caught_on_the_host():
    p = oz.Plan(16, 53, 100000, oz.OZ_ENGINE_IMMA)
    h = p.handle
    fake = 1 << 20  # never dereferenced: every case fails its checks before a launch
    ws = oz.oz_blocked_workspace_bytes(h, 8, 8, 64)
    assert ws == p.workspace_bytes(8, 8, 64)
    assert oz.oz_blocked_workspace_bytes(h, 8, 8, 0) == 0

    def call(k, k_slab, lda=None, wsb=ws, A=fake):
        return oz.oz_dgemm_blocked(h, 0, 0, 8, 8, k, k_slab, A, lda or k, fake, 8, fake, 8, fake, wsb, None)

    assert call(159820, 64) == oz.OZ_ERR_K_TOO_LARGE        # above the window at beta = 53
    assert call(152000, 151648) == oz.OZ_ERR_K_TOO_LARGE    # a slab above the INT32 cap
    assert call(152000, 0) == oz.OZ_ERR_INVALID_ARG
    assert call(1000, 64, lda=999) == oz.OZ_ERR_INVALID_ARG
    assert call(1000, 64, wsb=ws - 1) == oz.OZ_ERR_WORKSPACE
    assert call(1000, 64, A=fake + 4) == oz.OZ_ERR_INVALID_ARG
    assert call(1000, 256) == oz.OZ_ERR_WORKSPACE            # workspace sized for slabs of k_pad 128
    assert oz.oz_dgemm_blocked(h, 0, 0, 0, 8, 8, 8, None, 8, None, 8, None, 8, None, 0, None) == oz.OZ_OK


def test_transpose_argument_checks():
    fake = 1 << 20
    assert oz.oz_transpose(4, 8, fake, 7, fake, None) == oz.OZ_ERR_INVALID_ARG     # ld < cols
    assert oz.oz_transpose(4, 8, None, 8, fake, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_transpose(4, 8, fake + 4, 8, fake, None) == oz.OZ_ERR_INVALID_ARG
    assert oz.oz_transpose(0, 8, None, 8, None, None) == oz.OZ_OK
    assert oz.oz_transpose(-1, 8, fake, 8, fake, None) == oz.OZ_ERR_INVALID_ARG


def _layout_plans():
    yield "tc q16", oz.Plan(16, 0, 8192, oz.OZ_ENGINE_TC), 2
    yield "tc1 q14", oz.Plan(14, 50, 256, oz.OZ_ENGINE_TC1), 2
    yield "imma q16", oz.Plan(16, 0, 8192, oz.OZ_ENGINE_IMMA), 1
    yield "tc q20 widened", oz.Plan(20, 0, 4096, oz.OZ_ENGINE_TC), 2
    for fmt in ("E4M3", "E5M2", "E2M3", "E3M2", "E2M1"):
        yield fmt, oz.PlanFP(fmt, 8192), None


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (0, 5, 7), (300, 200, 1000), (129, 257, 4097), (8192, 8192, 8192),
                                   (65536, 256, 256), (256, 65536, 300)])
def test_workspace_layout_regions_are_disjoint_aligned_and_fit(m, n, k):
    """Every region of the workspace the kernels address (shifts, column
    maxima, the residue planes of both operands, the product's residues, and
    B^T for int8 planes)
    has the size the header documents, starts on a 256-byte boundary (16 bytes
    is what TMA needs), overlaps no other region and ends inside
    oz_workspace_bytes; the padded sizes are multiples of the tile and k
    alignments. Host logic only."""
    for name, p, elem in _layout_plans():
        st, L = oz.oz_workspace_layout(p.handle, m, n, k)
        assert st == oz.OZ_OK, name
        ws = p.workspace_bytes(m, n, k)
        _, k_align, _ = oz.oz_plane_geometry(p.handle, 0)
        m_pad, n_pad, k_pad = L["m_pad"], L["n_pad"], L["k_pad"]
        assert m_pad >= max(m, 1) and m_pad % 256 == 0, name
        assert n_pad >= max(n, 1) and n_pad % 256 == 0, name
        assert k_pad >= max(k, 1) and k_pad % k_align == 0, name
        _, _, row = oz.oz_plane_geometry(p.handle, k_pad)
        assert row % 16 == 0, name          # a TMA row stride is a multiple of 16 bytes
        fp = elem is None
        if fp:
            nplanes, digits, digit_bytes = p.planes, len(p.moduli), 2
            assert row == (k_pad // 2 if p.format == oz.FORMATS["E2M1"] else k_pad), name
        else:
            nplanes, digits, digit_bytes = p.q, p.q, 1
            assert row == elem * k_pad, name
        pitch = -(-max(n, 1) // (16 // digit_bytes)) * (16 // digit_bytes)
        regions = [("flag", 16), ("s", 4 * m), ("t", 4 * n), ("colmax", 8 * max(m, n)),
                   ("u", nplanes * m_pad * row), ("v", nplanes * n_pad * row),
                   ("y", digits * m * pitch * digit_bytes), ("bt", 0 if fp or elem == 2 else 8 * n * k)]
        end = 0
        for key, size in regions:
            off = L[key]
            assert off % 256 == 0, (name, key)
            assert off >= end, (name, key, off, end)
            end = off + size
        assert end <= ws < end + 256, (name, end, ws)


def test_header_compiles_as_c_and_links(tmp_path):
    """The boundary is plain C: a C11 program that includes oz.h, takes the
    address of every declared entry point, links against liboz.so and runs
    the host-only calls (plan, info, caps, workspace size and layout, an
    argument error) gets what the Python binding gets."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    syms = _declared_symbols()
    table = ",\n  ".join(f"(anyfn){s}" for s in syms)
    src = tmp_path / "abi_client.c"
    src.write_text(f"""
#include <stdio.h>
#include "oz.h"
typedef void (*anyfn)(void);
static const anyfn syms[] = {{
  {table}
}};
int main(void) {{
  for (size_t i = 0; i < sizeof syms / sizeof syms[0]; ++i)
    if (!syms[i]) return 2;
  for (int s = OZ_OK; s <= OZ_ERR_CUDA; ++s) {{
    const char* t = oz_status_str((oz_status)s);
    if (!t || !t[0]) return 3;
  }}
  oz_plan plan = NULL;
  if (oz_plan_create(&plan, 16, 0, 8192, OZ_ENGINE_TC) != OZ_OK) return 4;
  int q = 0, bits = 0, engine = -1;
  int64_t kmax = 0, kacc = 0, krec = 0, lay[11];
  uint32_t mods[32] = {{0}};
  if (oz_plan_info(plan, &q, &bits, &kmax, &engine, mods) != OZ_OK) return 5;
  if (oz_plan_caps(plan, &kacc, &krec) != OZ_OK) return 6;
  if (oz_workspace_layout(plan, 1000, 300, 777, lay) != OZ_OK) return 7;
  const size_t ws = oz_workspace_bytes(plan, 1000, 300, 777);
  const oz_status bad = oz_dgemm(plan, 0, 0, 8, 8, 8, NULL, 8, NULL, 8, NULL, 8, NULL, 0, NULL);
  printf("%d %d %lld %d %u %u %lld %lld %zu %lld %lld %d\\n", q, bits, (long long)kmax, engine, mods[0],
         mods[q - 1], (long long)kacc, (long long)krec, ws, (long long)lay[4], (long long)lay[10], (int)bad);
  oz_plan_destroy(plan);
  if (oz_plan_create(&plan, 16, 0, 0, OZ_ENGINE_TC) != OZ_ERR_INVALID_ARG) return 8;
  return 0;
}}
""")
    libdir = os.path.dirname(oz._build.LIB)
    exe = tmp_path / "abi_client"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-loz", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    got = r.stdout.split()
    p = oz.Plan(16, 0, 8192, oz.OZ_ENGINE_TC)
    _, lay = oz.oz_workspace_layout(p.handle, 1000, 300, 777)
    want = [p.q, p.bits, p.k_max, p.engine, p.moduli[0], p.moduli[-1], p.k_acc, p.k_rec,
            p.workspace_bytes(1000, 300, 777), lay["u"], lay["bt"]]
    assert [int(x) for x in got[:-1]] == want
    assert int(got[-1]) != oz.OZ_OK


def test_split_k_workspace_holds_the_extra_residue_sets():
    """A TC product with too few output tiles for the GPU splits its inner
    dimension (whole 1024-term slabs per range) and keeps one residue set per
    range: 256 x 256 x 65536 on CTA pairs has 16 tiles (one per modulus) and
    64 slabs, split four ways, so its workspace holds three more sets of
    Q m ldy bytes than the unsplit layout of a blocked call; a product with
    enough tiles (8192^3) does not split."""
    plan = oz.Plan(16, 53, 65536, oz.OZ_ENGINE_TC)
    m = n = 256
    k = 65536
    split = oz.oz_workspace_bytes(plan.handle, m, n, k)
    unsplit = oz.oz_blocked_workspace_bytes(plan.handle, m, n, k)
    assert split - unsplit == 3 * 16 * m * 256
    big = oz.Plan(16, 0, 8192, oz.OZ_ENGINE_TC)
    assert oz.oz_workspace_bytes(big.handle, 8192, 8192, 8192) == oz.oz_blocked_workspace_bytes(big.handle, 8192, 8192, 8192)
    imma = oz.Plan(16, 53, 65536, oz.OZ_ENGINE_IMMA)
    assert oz.oz_workspace_bytes(imma.handle, m, n, 100000) == oz.oz_blocked_workspace_bytes(imma.handle, m, n, 100000)
