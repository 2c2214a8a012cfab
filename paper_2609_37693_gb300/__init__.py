"""Python binding of liboz, the GB300 Ozaki-II emulated FP64 GEMM library.

The functions named ``oz_*`` mirror the C ABI of ``include/oz.h`` one to one:
they marshal arguments (device pointers as integers, the stream as a handle)
and return the ``oz_status`` code. Every step of the computation runs in the
library's CUDA kernels; nothing here computes. The library is built in-tree by
``paper_2609_37693_gb300.build``; importing this package fails loudly if it is
missing or cannot be loaded, and there is no fallback path.

On top of the ABI sit small conveniences for torch tensors: ``Plan`` (owns an
``oz_plan``), ``dgemm`` (allocates the workspace with torch and calls
``oz_dgemm`` on the current stream) and ``EmuMatmul`` (autograd).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OZ_OK = 0
OZ_ERR_INVALID_ARG = 1
OZ_ERR_K_TOO_LARGE = 2
OZ_ERR_WORKSPACE = 3
OZ_ERR_NONFINITE = 4
OZ_ERR_UNSUPPORTED = 5
OZ_ERR_CUDA = 6

OZ_ENGINE_AUTO = 0
OZ_ENGINE_IMMA = 1
OZ_ENGINE_TC = 2
OZ_ENGINE_FP = 3
OZ_ENGINE_TC1 = 4

OZ_FMT_E4M3 = 1
OZ_FMT_E2M3 = 2
OZ_FMT_E3M2 = 3
OZ_FMT_E2M1 = 4
OZ_FMT_E5M2 = 5
FORMATS = {"E4M3": OZ_FMT_E4M3, "E2M3": OZ_FMT_E2M3, "E3M2": OZ_FMT_E3M2, "E2M1": OZ_FMT_E2M1,
           "E5M2": OZ_FMT_E5M2}

OZ_MAX_MODULI = 20
OZ_MIN_MODULI = 9
OZ_MAX_BITS = 80
OZ_MAX_BITS_FP = 72
OZ_MAX_CHANNELS = 32
OZ_STATIC_SCRATCH_BYTES = 32 << 20

EXPORTED = ("oz_plan_create", "oz_plan_info", "oz_plan_destroy", "oz_workspace_bytes", "oz_workspace_layout",
            "oz_dgemm",
            "oz_query_status", "oz_split", "oz_residue_gemm", "oz_reconstruct", "oz_status_str",
            "oz_dgemm_static", "oz_batched_workspace_bytes", "oz_dgemm_batched", "oz_host_workspace_bytes",
            "oz_dgemm_host", "oz_plan_create_fp", "oz_plan_info_fp", "oz_plane_geometry",
            "oz_grouped_workspace_bytes", "oz_group_create", "oz_group_run", "oz_group_destroy",
            "oz_plan_caps", "oz_blocked_workspace_bytes", "oz_dgemm_blocked", "oz_selftest_bounded_wait",
            "oz_transpose", "oz_static_query_status")


class OzError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {oz_status_str(status)} (status {status})")


def _load_library():
    path = _build.LIB
    try:
        path = _build.build()          # no-op unless a source is newer than the library
    except RuntimeError:
        if not os.path.exists(path):
            raise
    lib = ctypes.CDLL(path)
    P, I64, I32, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    sig = {
        "oz_plan_create": (I32, [ctypes.POINTER(P), I32, I32, I64, I32]),
        "oz_plan_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I64),
                               ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_uint32)]),
        "oz_plan_destroy": (None, [P]),
        "oz_workspace_bytes": (SZ, [P, I64, I64, I64]),
        "oz_workspace_layout": (I32, [P, I64, I64, I64, ctypes.POINTER(I64)]),
        "oz_plane_geometry": (I32, [P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "oz_dgemm": (I32, [P, I32, I32, I64, I64, I64, P, I64, P, I64, P, I64, P, SZ, P]),
        "oz_query_status": (I32, [P, P]),
        "oz_split": (I32, [P, I32, I64, I64, P, I64, I64, I64, P, P, P, P, P]),
        "oz_residue_gemm": (I32, [P, I64, I64, I64, I64, I64, P, P, P, I32, P, P]),
        "oz_reconstruct": (I32, [P, I64, I64, P, P, P, P, I64, P]),
        "oz_status_str": (ctypes.c_char_p, [I32]),
        "oz_dgemm_static": (I32, [P, I32, I32, I64, I64, I64, P, I64, P, I64, P, I64, P]),
        "oz_static_query_status": (I32, [P]),
        "oz_batched_workspace_bytes": (SZ, [I32, P, P, I32]),
        "oz_host_workspace_bytes": (SZ, [P, I64, I64, I64, I64, I64]),
        "oz_plan_create_fp": (I32, [ctypes.POINTER(P), I32, I64, I32]),
        "oz_plan_info_fp": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I64), P, P, P,
                                  ctypes.POINTER(I32), P, SZ]),
        "oz_dgemm_host": (I32, [P, I64, I64, I64, P, I64, P, I64, P, I64, I64, I64, P, SZ, P, P, P]),
        "oz_dgemm_batched": (I32, [I32, P, P, P, P, P, P, P, P, P, P, SZ, P, I32]),
        "oz_grouped_workspace_bytes": (SZ, [I32, P, P]),
        "oz_group_create": (I32, [ctypes.POINTER(P), I32, P, P, P, P, P, P, P, P, P, SZ]),
        "oz_group_run": (I32, [P, P]),
        "oz_group_destroy": (None, [P]),
        "oz_plan_caps": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "oz_blocked_workspace_bytes": (SZ, [P, I64, I64, I64]),
        "oz_dgemm_blocked": (I32, [P, I32, I32, I64, I64, I64, I64, P, I64, P, I64, P, I64, P, SZ, P]),
        "oz_selftest_bounded_wait": (I32, [I32, P, P]),
        "oz_transpose": (I32, [I64, I64, P, I64, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load_library()
LIBRARY_PATH = _lib._name


# ---------------------------------------------------------------------------
# The C ABI, name for name
# ---------------------------------------------------------------------------

def oz_status_str(status: int) -> str:
    return _lib.oz_status_str(int(status)).decode()


def oz_plan_create(num_moduli: int = 16, bits: int = 0, k_hint: int = 8192, engine: int = OZ_ENGINE_AUTO):
    """Returns (status, plan handle or None)."""
    h = ctypes.c_void_p()
    st = _lib.oz_plan_create(ctypes.byref(h), int(num_moduli), int(bits), int(k_hint), int(engine))
    return st, (h.value if st == OZ_OK else None)


def oz_plan_create_fp(fmt: int, k_hint: int = 8192, bits: int = 0):
    """Returns (status, plan handle or None) for a float-format configuration."""
    h = ctypes.c_void_p()
    st = _lib.oz_plan_create_fp(ctypes.byref(h), int(fmt), int(k_hint), int(bits))
    return st, (h.value if st == OZ_OK else None)


def oz_plan_info_fp(plan, want_values: bool = False):
    """Returns (status, dict(channels, gemms, k_cfg, moduli, forms, bases, planes[, values]))."""
    ch, gm, npl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    kc = ctypes.c_int64()
    mods = (ctypes.c_uint32 * OZ_MAX_CHANNELS)()
    forms = (ctypes.c_int * OZ_MAX_CHANNELS)()
    bases = (ctypes.c_int * OZ_MAX_CHANNELS)()
    st = _lib.oz_plan_info_fp(plan, ctypes.byref(ch), ctypes.byref(gm), ctypes.byref(kc), mods, forms, bases,
                              ctypes.byref(npl), None, 0)
    if st != OZ_OK:
        return st, None
    info = {"channels": ch.value, "gemms": gm.value, "k_cfg": kc.value, "moduli": list(mods[: ch.value]),
            "forms": list(forms[: ch.value]), "bases": list(bases[: ch.value]), "planes": npl.value}
    if want_values:
        total = 0
        for m, f in zip(info["moduli"], info["forms"]):
            total += m * (1 if f == 1 else 3 if f == 3 else 2)
        vals = (ctypes.c_int16 * total)()
        st = _lib.oz_plan_info_fp(plan, None, None, None, None, None, None, None, vals, total)
        if st != OZ_OK:
            return st, None
        info["values"] = list(vals)
    return st, info


def oz_plan_info(plan):
    """Returns (status, dict(q, bits, k_max, engine, moduli))."""
    q, b, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    km = ctypes.c_int64()
    mods = (ctypes.c_uint32 * OZ_MAX_MODULI)()
    st = _lib.oz_plan_info(plan, ctypes.byref(q), ctypes.byref(b), ctypes.byref(km), ctypes.byref(e), mods)
    if st != OZ_OK:
        return st, None
    return st, {"q": q.value, "bits": b.value, "k_max": km.value, "engine": e.value,
                "moduli": [int(x) for x in mods[: q.value]]}


def oz_plan_caps(plan):
    """Returns (status, k_acc, k_rec)."""
    a, r = ctypes.c_int64(0), ctypes.c_int64(0)
    st = _lib.oz_plan_caps(plan, ctypes.byref(a), ctypes.byref(r))
    return st, a.value, r.value


def oz_plan_destroy(plan) -> None:
    _lib.oz_plan_destroy(plan)


def oz_workspace_bytes(plan, m: int, n: int, k: int) -> int:
    return int(_lib.oz_workspace_bytes(plan, int(m), int(n), int(k)))


def oz_workspace_layout(plan, m: int, n: int, k: int):
    """Returns (status, dict of byte offsets flag/s/t/colmax/u/v/y, m_pad/n_pad/k_pad, and bt)."""
    out = (ctypes.c_int64 * 11)()
    st = _lib.oz_workspace_layout(plan, int(m), int(n), int(k), out)
    if st != OZ_OK:
        return st, None
    keys = ("flag", "s", "t", "colmax", "u", "v", "y", "m_pad", "n_pad", "k_pad", "bt")
    return st, {key: int(v) for key, v in zip(keys, out)}


def oz_plane_geometry(plan, k_pad: int):
    """Returns (status, k_align, row_bytes)."""
    a, r = ctypes.c_int64(0), ctypes.c_int64(0)
    st = _lib.oz_plane_geometry(plan, int(k_pad), ctypes.byref(a), ctypes.byref(r))
    return st, a.value, r.value


def oz_dgemm(plan, trans_a, trans_b, m, n, k, A, lda, B, ldb, C, ldc, workspace, workspace_bytes, stream) -> int:
    return _lib.oz_dgemm(plan, int(trans_a), int(trans_b), int(m), int(n), int(k), A, int(lda), B, int(ldb), C,
                         int(ldc), workspace, int(workspace_bytes), stream)


def oz_blocked_workspace_bytes(plan, m: int, n: int, k_slab: int) -> int:
    return int(_lib.oz_blocked_workspace_bytes(plan, int(m), int(n), int(k_slab)))


def oz_dgemm_blocked(plan, trans_a, trans_b, m, n, k, k_slab, A, lda, B, ldb, C, ldc, workspace, workspace_bytes,
                     stream) -> int:
    return _lib.oz_dgemm_blocked(plan, int(trans_a), int(trans_b), int(m), int(n), int(k), int(k_slab), A, int(lda),
                                 B, int(ldb), C, int(ldc), workspace, int(workspace_bytes), stream)


def oz_dgemm_static(plan, trans_a, trans_b, m, n, k, A, lda, B, ldb, C, ldc, stream) -> int:
    """oz_dgemm without a workspace argument: the library's built-in device
    scratch array (OZ_STATIC_SCRATCH_BYTES per GPU) serves as the workspace, for
    callers that cannot allocate device memory. Calls overlapping on the GPU race."""
    return _lib.oz_dgemm_static(plan, int(trans_a), int(trans_b), int(m), int(n), int(k), A, int(lda), B, int(ldb),
                                C, int(ldc), stream)


def oz_static_query_status(stream) -> int:
    """Status of the last oz_dgemm_static call on the current device (waits for the stream)."""
    return _lib.oz_static_query_status(stream)


def oz_batched_workspace_bytes(count, plans, mnk, nstreams) -> int:
    """plans: ctypes array of plan handles; mnk: ctypes int64 array of 3*count."""
    return int(_lib.oz_batched_workspace_bytes(int(count), plans, mnk, int(nstreams)))


def oz_dgemm_batched(count, plans, mnk, trans, A, lda, B, ldb, C, ldc, workspace, workspace_bytes, streams,
                     nstreams) -> int:
    """Array arguments are ctypes arrays (or None for trans); see include/oz.h."""
    return _lib.oz_dgemm_batched(int(count), plans, mnk, trans, A, lda, B, ldb, C, ldc, workspace,
                                 int(workspace_bytes), streams, int(nstreams))


def oz_host_workspace_bytes(plan, m, n, k, rows_per_chunk=0, cols_per_chunk=0) -> int:
    return int(_lib.oz_host_workspace_bytes(plan, int(m), int(n), int(k), int(rows_per_chunk), int(cols_per_chunk)))


def oz_dgemm_host(plan, m, n, k, A, lda, B, ldb, C, ldc, rows_per_chunk, cols_per_chunk, workspace, workspace_bytes,
                  stream, stream_h2d, stream_d2h) -> int:
    """A, B, C are HOST pointers (pinned memory overlaps the copies)."""
    return _lib.oz_dgemm_host(plan, int(m), int(n), int(k), A, int(lda), B, int(ldb), C, int(ldc),
                              int(rows_per_chunk), int(cols_per_chunk), workspace, int(workspace_bytes), stream,
                              stream_h2d, stream_d2h)


def oz_selftest_bounded_wait(arrive, status, stream) -> int:
    """status: device pointer to an int32 (OR-ed with 4 if the wait completed,
    2 if it ran out)."""
    return _lib.oz_selftest_bounded_wait(int(arrive), status, stream)


def oz_transpose(rows, cols, X, ld, Y, stream) -> int:
    return _lib.oz_transpose(int(rows), int(cols), X, int(ld), Y, stream)


def oz_query_status(workspace, stream) -> int:
    return _lib.oz_query_status(workspace, stream)


def oz_split(plan, contiguous, nvec, length, X, ld, nvec_pad, k_pad, shifts, planes, flag, colmax, stream) -> int:
    return _lib.oz_split(plan, int(contiguous), int(nvec), int(length), X, int(ld), int(nvec_pad), int(k_pad),
                         shifts, planes, flag, colmax, stream)


def oz_residue_gemm(plan, m, n, m_pad, n_pad, k_pad, U, V, Y, raw, flag, stream) -> int:
    return _lib.oz_residue_gemm(plan, int(m), int(n), int(m_pad), int(n_pad), int(k_pad), U, V, Y, int(raw),
                                flag, stream)


def oz_reconstruct(plan, m, n, Y, s, t, C, ldc, stream) -> int:
    return _lib.oz_reconstruct(plan, int(m), int(n), Y, s, t, C, int(ldc), stream)


# ---------------------------------------------------------------------------
# torch conveniences
# ---------------------------------------------------------------------------

def _check(st: int, what: str):
    if st != OZ_OK:
        raise OzError(st, what)


def _ld(t) -> int:
    """Leading dimension of a row-major 2-D tensor; for an empty tensor, its
    column count (the strides of empty tensors carry no layout)."""
    return max(t.stride(0), 1) if t.numel() else max(t.shape[1], 1)


def round_up(x: int, r: int) -> int:
    return (x + r - 1) // r * r


class Plan:
    """An oz_plan owned by Python. ``Plan(q=16, bits=0, k_hint=8192, engine=OZ_ENGINE_AUTO)``."""

    def __init__(self, q: int = 16, bits: int = 0, k_hint: int = 8192, engine: int = OZ_ENGINE_AUTO):
        st, h = oz_plan_create(q, bits, k_hint, engine)
        _check(st, "oz_plan_create")
        self.handle = h
        _, info = oz_plan_info(h)
        self.q, self.bits, self.k_max = info["q"], info["bits"], info["k_max"]
        self.engine, self.moduli = info["engine"], info["moduli"]
        _, self.k_acc, self.k_rec = oz_plan_caps(h)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            oz_plan_destroy(h)
            self.handle = None

    def workspace_bytes(self, m: int, n: int, k: int) -> int:
        return oz_workspace_bytes(self.handle, m, n, k)

    def plane_geometry(self, k: int):
        """(k_pad, row_bytes) of the planes for inner dimension k."""
        _, align, _ = oz_plane_geometry(self.handle, 0)
        k_pad = round_up(max(int(k), 1), align)
        _, _, row = oz_plane_geometry(self.handle, k_pad)
        return k_pad, row

    def __repr__(self):
        return f"Plan(q={self.q}, bits={self.bits}, k_max={self.k_max}, engine={self.engine})"


class PlanFP(Plan):
    """A float-format configuration (oz_plan_create_fp): ``PlanFP("E4M3", k_hint=8192)``.
    q is the number of low-precision GEMMs; moduli, forms and bases describe
    the channels."""

    def __init__(self, fmt, k_hint: int = 8192, bits: int = 0):
        code = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
        st, h = oz_plan_create_fp(code, k_hint, bits)
        _check(st, "oz_plan_create_fp")
        self.handle = h
        _, info = oz_plan_info(h)
        _, fi = oz_plan_info_fp(h)
        self.format = code
        self.bits, self.k_max, self.engine = info["bits"], info["k_max"], info["engine"]
        _, self.k_acc, self.k_rec = oz_plan_caps(h)
        self.channels, self.q, self.k_cfg = fi["channels"], fi["gemms"], fi["k_cfg"]
        self.moduli, self.forms, self.bases, self.planes = fi["moduli"], fi["forms"], fi["bases"], fi["planes"]

    def plane_values(self):
        """[plane][class] scaled alphabet values of every plane's table."""
        _, fi = oz_plan_info_fp(self.handle, want_values=True)
        out, off = [], 0
        for m, f in zip(self.moduli, self.forms):
            for _ in range(1 if f == 1 else 3 if f == 3 else 2):
                out.append(fi["values"][off: off + m])
                off += m
        return out

    def __repr__(self):
        return f"PlanFP(format={self.format}, q={self.q}, channels={self.channels}, bits={self.bits})"


def _stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def workspace(plan: Plan, m: int, n: int, k: int, device=None):
    import torch
    nbytes = plan.workspace_bytes(m, n, k)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")


def dgemm(A, B, plan: Plan | None = None, trans_a: bool = False, trans_b: bool = False, out=None, ws=None,
          stream=None):
    """C = op(A) op(B) for float64 CUDA tensors (row-major, unit inner stride)."""
    import torch
    if A.dtype != torch.float64 or B.dtype != torch.float64 or not A.is_cuda or not B.is_cuda:
        raise TypeError("dgemm takes float64 CUDA tensors")
    if A.dim() != 2 or B.dim() != 2 or (A.numel() and A.stride(1) != 1) or (B.numel() and B.stride(1) != 1):
        raise ValueError("dgemm takes 2-D tensors with unit inner stride")
    m, k = (A.shape[1], A.shape[0]) if trans_a else (A.shape[0], A.shape[1])
    k2, n = (B.shape[1], B.shape[0]) if trans_b else (B.shape[0], B.shape[1])
    if k != k2:
        raise ValueError(f"inner dimensions differ: {k} vs {k2}")
    if plan is None:
        plan = Plan(16, 0, max(k, 1))
    C = out if out is not None else torch.empty((m, n), dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace(plan, m, n, k, A.device)
    st = oz_dgemm(plan.handle, int(trans_a), int(trans_b), m, n, k, A.data_ptr(), _ld(A),
                  B.data_ptr(), _ld(B), C.data_ptr(), _ld(C), ws.data_ptr(),
                  ws.numel(), _stream_handle(stream))
    _check(st, "oz_dgemm")
    return C


def _operands(A, B, trans_a, trans_b, what):
    import torch
    if A.dtype != torch.float64 or B.dtype != torch.float64 or not A.is_cuda or not B.is_cuda:
        raise TypeError(f"{what} takes float64 CUDA tensors")
    if A.dim() != 2 or B.dim() != 2 or (A.numel() and A.stride(1) != 1) or (B.numel() and B.stride(1) != 1):
        raise ValueError(f"{what} takes 2-D tensors with unit inner stride")
    m, k = (A.shape[1], A.shape[0]) if trans_a else (A.shape[0], A.shape[1])
    k2, n = (B.shape[1], B.shape[0]) if trans_b else (B.shape[0], B.shape[1])
    if k != k2:
        raise ValueError(f"inner dimensions differ: {k} vs {k2}")
    return m, n, k


def dgemm_blocked(A, B, plan: Plan, k_slab: int, trans_a: bool = False, trans_b: bool = False, out=None, ws=None,
                  stream=None):
    """C = op(A) op(B) through oz_dgemm_blocked: the inner dimension in slabs
    of k_slab terms, each slab's digits added into a running residue (the same
    bits as ``dgemm`` wherever both apply; K up to ``plan.k_rec``, slabs up to
    ``plan.k_acc``). The workspace holds one slab's planes."""
    import torch
    m, n, k = _operands(A, B, trans_a, trans_b, "dgemm_blocked")
    C = out if out is not None else torch.empty((m, n), dtype=torch.float64, device=A.device)
    if ws is None:
        nbytes = oz_blocked_workspace_bytes(plan.handle, m, n, max(min(int(k_slab), k), 1))
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=A.device)
    st = oz_dgemm_blocked(plan.handle, int(trans_a), int(trans_b), m, n, k, int(k_slab), A.data_ptr(), _ld(A),
                          B.data_ptr(), _ld(B), C.data_ptr(), _ld(C), ws.data_ptr(), ws.numel(),
                          _stream_handle(stream))
    _check(st, "oz_dgemm_blocked")
    return C


def launches_per_dgemm(trans_a: bool = False, trans_b: bool = False, engine: int = OZ_ENGINE_TC) -> int:
    """Kernels one INT8 oz_dgemm launches without a split of K: A's rows split
    in one kernel (its columns, for trans_a, in three: column maxima, shifts,
    split); B's columns in three (bf16 planes) or transposed and split as rows
    (two, int8 planes of the IMMA engine); one when trans_b; then the GEMM and
    the reconstruct."""
    a = 3 if trans_a else 1
    b = 1 if trans_b else (2 if engine == OZ_ENGINE_IMMA else 3)
    return a + b + 2


def query_status(ws, stream=None) -> int:
    return oz_query_status(ws.data_ptr(), _stream_handle(stream))


# ---------------------------------------------------------------------------
# Differentiable emulated FP64 matmul
# ---------------------------------------------------------------------------

_plan_cache: dict = {}


def plan_for(k: int, q: int = 16, engine: int = OZ_ENGINE_AUTO) -> Plan:
    """A cached plan for inner dimension k (bits chosen as the largest the
    window allows at that k)."""
    key = (int(q), int(max(k, 1)), int(engine))
    p = _plan_cache.get(key)
    if p is None:
        p = Plan(q, 0, max(k, 1), engine)
        _plan_cache[key] = p
    return p


def _matmul_op(A, B, trans_a: bool, trans_b: bool, q: int, engine: int):
    k = A.shape[0] if trans_a else A.shape[1]
    return dgemm(A, B, plan_for(k, q, engine), trans_a=trans_a, trans_b=trans_b)


def _import_torch():
    import torch
    return torch


class EmuMatmul:
    """C = A @ B for float64 CUDA matrices through the emulated product, with
    dA = dC B^T and dB = A^T dC computed by the same kernels (the transposed
    operand modes of oz_dgemm). Use ``EmuMatmul.apply(A, B, q=16)``."""

    _fn = None

    @classmethod
    def _function(cls):
        if cls._fn is None:
            torch = _import_torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, A, B, q=16, engine=OZ_ENGINE_AUTO):
                    A_ = A.contiguous()
                    B_ = B.contiguous()
                    ctx.save_for_backward(A_, B_)
                    ctx.q, ctx.engine = q, engine
                    return _matmul_op(A_, B_, False, False, q, engine)

                @staticmethod
                def backward(ctx, dC):
                    A, B = ctx.saved_tensors
                    dC = dC.contiguous()
                    dA = dB = None
                    if ctx.needs_input_grad[0]:
                        dA = _matmul_op(dC, B, False, True, ctx.q, ctx.engine)      # dC (m x n) B^T (n x k)
                    if ctx.needs_input_grad[1]:
                        dB = _matmul_op(A, dC, True, False, ctx.q, ctx.engine)      # A^T (k x m) dC (m x n)
                    return dA, dB, None, None

            cls._fn = _F
        return cls._fn

    @classmethod
    def apply(cls, A, B, q: int = 16, engine: int = OZ_ENGINE_AUTO):
        return cls._function().apply(A, B, q, engine)


def emu_matmul(A, B, q: int = 16, engine: int = OZ_ENGINE_AUTO):
    return EmuMatmul.apply(A, B, q, engine)


# ---------------------------------------------------------------------------
# Batched uneven products, CUDA-graph capture and the autotuner
# ---------------------------------------------------------------------------

def plan_least_q(k: int, bits: int = 53, engine: int = OZ_ENGINE_AUTO) -> Plan:
    """The paper's configuration rule for one product: the least Q whose
    window holds at inner dimension k with `bits` kept (Q = 15 up to k = 836
    and 16 above at 53 bits). Cached."""
    key = ("least", int(bits), int(max(k, 1)), int(engine))
    p = _plan_cache.get(key)
    if p is None:
        p = Plan(0, bits, max(k, 1), engine)
        _plan_cache[key] = p
    return p


class BatchedGemm:
    """count products C_i = A_i B_i of uneven shapes through one
    oz_dgemm_batched call (optionally captured into one CUDA graph).

    shapes: list of (m, n, k). plans: one Plan per problem, or None for the
    least-Q rule at `bits` (TC engine with one CTA per tile: over several
    streams oz_dgemm_batched runs TC GEMMs that way in any case).
    nstreams: streams the problems spread over."""

    def __init__(self, shapes, plans=None, nstreams: int = 4, bits: int = 53, engine: int = OZ_ENGINE_TC1,
                 device=None):
        torch = _import_torch()
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        self.count = len(self.shapes)
        self.plans = list(plans) if plans is not None else [plan_least_q(k, bits, engine) for (_, _, k) in self.shapes]
        self.nstreams = int(nstreams)
        self.device = torch.device(device or "cuda")
        self._plan_arr = (ctypes.c_void_p * max(self.count, 1))(*[p.handle for p in self.plans])
        flat = [x for s in self.shapes for x in s]
        self._mnk = (ctypes.c_int64 * max(len(flat), 1))(*flat)
        nbytes = oz_batched_workspace_bytes(self.count, self._plan_arr, self._mnk, self.nstreams)
        if self.count and nbytes == 0:
            raise OzError(OZ_ERR_INVALID_ARG, "oz_batched_workspace_bytes")
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        # streams[0] is the batch's origin stream (a side stream, so that the
        # batch can be captured); run() orders it after the caller's stream
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.nstreams)]
        self._graph = None

    def _ptrs(self, As, Bs, Cs):
        n = max(self.count, 1)
        P = ctypes.c_void_p
        self._A = (P * n)(*[a.data_ptr() for a in As])
        self._B = (P * n)(*[b.data_ptr() for b in Bs])
        self._C = (P * n)(*[c.data_ptr() for c in Cs])
        self._lda = (ctypes.c_int64 * n)(*[_ld(a) for a in As])
        self._ldb = (ctypes.c_int64 * n)(*[_ld(b) for b in Bs])
        self._ldc = (ctypes.c_int64 * n)(*[_ld(c) for c in Cs])
        self._str = (P * self.nstreams)(*[s.cuda_stream for s in self.streams])

    def run(self, As, Bs, Cs):
        """Launch the batch after the work queued on the current stream; the
        current stream then waits for the batch."""
        torch = _import_torch()
        self._ptrs(As, Bs, Cs)
        cur = torch.cuda.current_stream(self.device)
        self.streams[0].wait_stream(cur)
        st = oz_dgemm_batched(self.count, self._plan_arr, self._mnk, None, self._A, self._lda, self._B, self._ldb,
                              self._C, self._ldc, self.ws.data_ptr(), self.ws.numel(), self._str, self.nstreams)
        cur.wait_stream(self.streams[0])
        _check(st, "oz_dgemm_batched")

    def capture(self, As, Bs, Cs):
        """Record the batch into one CUDA graph over these exact tensors;
        replay() reruns it on whatever they hold then."""
        torch = _import_torch()
        self._ptrs(As, Bs, Cs)
        # the first call on each shape sets kernel attributes outside the capture
        self.run(As, Bs, Cs)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.streams[0], capture_error_mode="relaxed"):
            st = oz_dgemm_batched(self.count, self._plan_arr, self._mnk, None, self._A, self._lda, self._B,
                                  self._ldb, self._C, self._ldc, self.ws.data_ptr(), self.ws.numel(), self._str,
                                  self.nstreams)
        _check(st, "oz_dgemm_batched (capture)")
        self._graph = g
        return g

    def replay(self):
        """Replay the captured batch after the work queued on the current stream."""
        torch = _import_torch()
        cur = torch.cuda.current_stream(self.device)
        self.streams[0].wait_stream(cur)
        with torch.cuda.stream(self.streams[0]):
            self._graph.replay()
        cur.wait_stream(self.streams[0])


_autotune_cache: dict = {}


def autotune_batched(shapes, As, Bs, Cs, candidates=(1, 2, 4, 8, 16), bits: int = 53, reps: int = 3):
    """Pick the stream count for a batch of shapes by timing captured-graph
    replays of each candidate; returns (best BatchedGemm with its graph
    captured over As/Bs/Cs, {nstreams: ms}). Results are cached per shape list."""
    torch = _import_torch()
    key = (tuple(tuple(int(x) for x in s) for s in shapes), int(bits))
    timings = {}
    best = None
    choices = [_autotune_cache[key]] if key in _autotune_cache else list(candidates)
    for ns in choices:
        bg = BatchedGemm(shapes, nstreams=ns, bits=bits)
        bg.capture(As, Bs, Cs)
        bg.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(bg.streams[0])
            bg.replay()
            e1.record(bg.streams[0])
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        timings[ns] = min(ts)
        if best is None or timings[ns] < timings[best[0]]:
            best = (ns, bg)
        else:
            del bg
    _autotune_cache[key] = best[0]
    return best[1], timings


def blocked_candidates(k: int, bits: int = 53, formats=("E4M3", "E2M1"), slabs=(8192, 16384, 32768)):
    """Configurations that can run a product with inner dimension k through
    the blocked call at `bits` kept bits, as (label, plan, k_slab): the INT8
    plan of the least Q on the TC engine (whole K, and the given slab lengths
    below K), and each float format's plan for its largest frozen K_cfg whose
    window admits k, in slabs of its accumulation cap. Every candidate keeps
    the same bits, so every one returns the same C."""
    out = []
    try:
        p = Plan(0, bits, max(k, 1), OZ_ENGINE_TC)
    except OzError:
        p = None
    if p is not None:
        out.append(("int8 q=%d" % p.q, p, max(k, 1)))
        for s in slabs:
            if s < k:
                out.append(("int8 q=%d slab=%d" % (p.q, s), p, s))
    for f in formats:
        for kcfg in (16384, 8192):
            try:
                q = PlanFP(f, kcfg, bits)
            except OzError:
                continue
            if k <= q.k_rec:
                out.append(("%s (%d GEMMs) slab=%d" % (f, q.q, min(q.k_acc, max(k, 1))), q, min(q.k_acc, max(k, 1))))
                break
    return out


def autotune_blocked(A, B, candidates=None, bits: int = 53, reps: int = 2, stream=None):
    """The configuration trade-off of a blocked product (plane format, the
    GEMM count it implies, slab length): time C = A B through
    oz_dgemm_blocked for each candidate (label, plan, k_slab) -- by default
    blocked_candidates(K, bits) -- and return (label, plan, k_slab) of the
    fastest with {label: ms}."""
    torch = _import_torch()
    m, n, k = _operands(A, B, False, False, "autotune_blocked")
    cands = candidates if candidates is not None else blocked_candidates(k, bits)
    if not cands:
        raise OzError(OZ_ERR_K_TOO_LARGE, "autotune_blocked")
    C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    s = torch.cuda.current_stream(A.device) if stream is None else stream
    timings, best = {}, None
    for label, plan, k_slab in cands:
        nbytes = oz_blocked_workspace_bytes(plan.handle, m, n, max(min(int(k_slab), k), 1))
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=A.device)
        dgemm_blocked(A, B, plan, k_slab, out=C, ws=ws, stream=s)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            dgemm_blocked(A, B, plan, k_slab, out=C, ws=ws, stream=s)
            e1.record(s)
            torch.cuda.synchronize(A.device)
            ts.append(e0.elapsed_time(e1))
        timings[label] = min(ts)
        if best is None or timings[label] < timings[best[0]]:
            best = (label, plan, k_slab)
        del ws
    return best, timings


def autotune_batch(shapes, As, Bs, Cs, streams=(1, 2, 4, 8, 16), bits: int = 53, reps: int = 3):
    """Launch structure and modulus counts of a batch of uneven products,
    chosen by timing captured-graph replays of each candidate:
      "streams=S": oz_dgemm_batched over S streams, each product at its least Q;
      "grouped":   oz_group_run, each product at its least Q (one set of
                   launches per distinct Q);
      "grouped q=16": oz_group_run with every product on the Q = 16 plan (one
                   set of launches for the whole batch; at 53 bits Q = 16 holds
                   the window for every k up to 159 819, so the bits are the
                   same as at the least Q).
      "streams=1 pairs": one stream, the products' GEMMs on CTA pairs (256 x
                   256 tiles instead of 128 x 256).
    Candidates are built, timed and freed one at a time. Returns (the fastest
    runner, captured over As/Bs/Cs and with a replay() method, its label,
    {label: ms})."""
    torch = _import_torch()
    shapes = [tuple(int(x) for x in sh) for sh in shapes]

    def time_replays(runner):
        runner.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            runner.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    builders = [("streams=%d" % ns, lambda ns=ns: BatchedGemm(shapes, nstreams=ns, bits=bits)) for ns in streams]
    # one stream: the products may take the CTA-pair GEMM (256 x 256 tiles)
    builders.append(("streams=1 pairs", lambda: BatchedGemm(shapes, nstreams=1, bits=bits, engine=OZ_ENGINE_TC)))
    builders.append(("grouped", lambda: GroupedGemm(As, Bs, Cs, bits=bits)))
    if all(k <= 159819 for (_, _, k) in shapes):
        q16 = Plan(16, bits, max([k for (_, _, k) in shapes] + [1]), OZ_ENGINE_TC)
        builders.append(("grouped q=16", lambda: GroupedGemm(As, Bs, Cs, plans=[q16] * len(shapes))))
    timings, best = {}, None
    for label, build in builders:
        runner = build()
        if isinstance(runner, BatchedGemm):
            runner.capture(As, Bs, Cs)
        else:
            runner.capture()
        timings[label] = time_replays(runner)
        if best is None or timings[label] < timings[best[0]]:
            best = (label, runner)
        else:
            del runner
        torch.cuda.empty_cache()
    return best[1], best[0], timings


class GroupedGemm:
    """count products C_i = A_i B_i (float64 CUDA tensors, row-major) through
    oz_group_create / oz_group_run: one launch per phase over all products of
    a plan. The tensors are fixed at construction; new values written into
    them are picked up by the next run or replay. Plans: the least-Q rule at
    `bits` per product (TC engine) unless given."""

    def __init__(self, As, Bs, Cs, plans=None, bits: int = 53, engine: int = OZ_ENGINE_AUTO, device=None):
        torch = _import_torch()
        self.count = len(As)
        self.shapes = [(int(A.shape[0]), int(B.shape[1]), int(A.shape[1])) for A, B in zip(As, Bs)]
        self.plans = list(plans) if plans is not None else [plan_least_q(k, bits, engine) for (_, _, k) in self.shapes]
        self.device = torch.device(device or "cuda")
        P, I64 = ctypes.c_void_p, ctypes.c_int64
        n = max(self.count, 1)
        self._plan_arr = (P * n)(*[p.handle for p in self.plans])
        self._mnk = (I64 * (3 * n))(*[x for s in self.shapes for x in s])
        nbytes = _lib.oz_grouped_workspace_bytes(self.count, self._plan_arr, self._mnk)
        if self.count and not nbytes:
            raise OzError(OZ_ERR_UNSUPPORTED, "oz_grouped_workspace_bytes")
        self.ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        self._keep = (As, Bs, Cs)
        self._A = (P * n)(*[A.data_ptr() for A in As])
        self._B = (P * n)(*[B.data_ptr() for B in Bs])
        self._C = (P * n)(*[C.data_ptr() for C in Cs])
        self._lda = (I64 * n)(*[_ld(A) for A in As])
        self._ldb = (I64 * n)(*[_ld(B) for B in Bs])
        self._ldc = (I64 * n)(*[_ld(C) for C in Cs])
        h = P()
        st = _lib.oz_group_create(ctypes.byref(h), self.count, self._plan_arr, self._mnk, self._A, self._lda,
                                  self._B, self._ldb, self._C, self._ldc, self.ws.data_ptr(), self.ws.numel())
        _check(st, "oz_group_create")
        self.handle = h
        self.graph = None

    def run(self, stream=None):
        _check(_lib.oz_group_run(self.handle, _stream_handle(stream)), "oz_group_run")

    def launches(self) -> int:
        """Kernels one run launches: per group of alike plans, the split of A
        (one kernel for long rows, one for short rows of at most 4096 padded
        entries), column maxima, shifts and split of B, the GEMMs and the
        Reconstruct."""
        groups = {}
        for p, (m, n, k) in zip(self.plans, self.shapes):
            g = groups.setdefault((p.q, p.bits, tuple(p.moduli)), set())
            if m and n and k:
                g.add(round_up(k, 128) > 4096)
        return sum(5 + len(kinds) for kinds in groups.values() if kinds)

    def capture(self, stream=None):
        """Record one run into a CUDA graph (replay() runs it)."""
        torch = _import_torch()
        s = stream or torch.cuda.Stream(self.device)
        self.run(s)                       # warm-up outside the capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(s)
        self.graph = g

    def replay(self):
        self.graph.replay()

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.oz_group_destroy(h)
            self.handle = None


class HostGemm:
    """C = A B for host (CPU) float64 tensors through oz_dgemm_host: C in blocks
    of rows_per_chunk x cols_per_chunk, the copies to and from the device
    overlapping the phases of neighbouring blocks. Pin the host tensors
    (tensor.pin_memory()) for the overlap to happen."""

    def __init__(self, plan: Plan, m: int, n: int, k: int, rows_per_chunk: int = 0, device=None,
                 cols_per_chunk: int = 0):
        torch = _import_torch()
        self.plan, self.m, self.n, self.k = plan, m, n, k
        self.rows, self.cols = rows_per_chunk, cols_per_chunk
        # the block edges the library uses (0 picks about a quarter of m or n, a
        # multiple of 256)
        edge = lambda x: round_up(max((x + 3) // 4, 1), 256)
        r = rows_per_chunk or edge(m)
        c = cols_per_chunk or edge(n)
        self.block = (min(r, m) if m else r, min(c, n) if n else c)
        self.device = torch.device(device or "cuda")
        nbytes = oz_host_workspace_bytes(plan.handle, m, n, k, rows_per_chunk, cols_per_chunk)
        if nbytes == 0:
            raise OzError(OZ_ERR_INVALID_ARG, "oz_host_workspace_bytes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.h2d = torch.cuda.Stream(self.device)
        self.d2h = torch.cuda.Stream(self.device)

    def __call__(self, A, B, C, stream=None):
        torch = _import_torch()
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        st = oz_dgemm_host(self.plan.handle, self.m, self.n, self.k, A.data_ptr(), _ld(A), B.data_ptr(),
                           _ld(B), C.data_ptr(), _ld(C), self.rows, self.cols, self.ws.data_ptr(),
                           self.ws.numel(), ctypes.c_void_p(s.cuda_stream), ctypes.c_void_p(self.h2d.cuda_stream),
                           ctypes.c_void_p(self.d2h.cuda_stream))
        _check(st, "oz_dgemm_host")
        return C
