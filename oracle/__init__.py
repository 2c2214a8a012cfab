"""CPU oracle for Ozaki-II emulated FP64 GEMM (INT8 residue path).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package. It
shares no code with the CUDA library: the arithmetic lives in ``oz_oracle.c``
(plain C, compiled with gcc) and in the plain Python below, and neither side
imports the other.

What is here:

* ``max_product_moduli(Q, m_max)`` -- the modulus set. The paper fixes the INT8
  configuration as sixteen pairwise-coprime moduli up to 239, radius 119,
  K_max = 151 647 (Sec. "INT4 and INT8"). It does not print the set. Our
  reading: the set of Q pairwise-coprime integers <= m_max with the largest
  product (ties: the smaller largest modulus). The search is an exact dynamic
  program over the primes up to sqrt(m_max), as in step 3 of the search of
  Sec. "Solving the Program"; every integer <= m_max has at most one prime
  factor above sqrt(m_max), so each such prime is a group of which at most one
  member is taken.
* ``caps(moduli, K, beta)`` -- kappa_rec, kappa_acc, K_max (eq. caps) and
  r_max(1) (eq. rmax) for INT32 accumulation (Lambda = 2^31 - 1).
* ``least_q(K)`` -- the least INT8 Q at inner dimension K (Table tab:moduli).
* ``beta_max(moduli, K)`` -- the largest beta with 2K(2^beta - 1)^2 < P
  (eq. ov-crtgen with B_A = B_B = 2^beta - 1).
* ``dgemm``, ``dgemm_entries``, ``planes``, ``scale``, ``crt``, ``round_scaled``,
  ``exact_error`` -- ctypes wrappers of ``oz_oracle.c``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oz_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboz_oracle.so")
_lock = threading.Lock()
_lib = None

INT32_LAMBDA = 2**31 - 1          # Sec. "Exactness Constraints": INT32 accumulator bound
FP32_LAMBDA = 2**24               # the FP32 accumulator bound of the same section


def build(force: bool = False) -> str:
    """Compile oz_oracle.c into oracle/_build/liboz_oracle.so with gcc + OpenMP."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            i32 = ctypes.c_int
            lib.ozo_scale.argtypes = [P, i64, i64, i64, i64, i32, P]
            lib.ozo_residue_planes.argtypes = [P, i64, i64, i64, i64, P, P, i32, P]
            lib.ozo_dgemm.argtypes = [i64, i64, i64, P, i64, P, i64, P, i32, i32, P, i64, P, P, P]
            lib.ozo_dgemm_entries.argtypes = [i64, i64, i64, P, i64, P, i64, P, i32, i32, i64, P, P, P, P]
            lib.ozo_crt.argtypes = [i64, P, P, i32, P]
            lib.ozo_round.argtypes = [i64, P, P, P]
            lib.ozo_exact_error.argtypes = [i64, i64, i64, P, i64, P, i64, P, i64, i64, P, P, P, P]
            for f in ("ozo_scale", "ozo_residue_planes", "ozo_dgemm", "ozo_dgemm_entries", "ozo_crt",
                      "ozo_round", "ozo_exact_error"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


# --------------------------------------------------------------------------
# Configuration: moduli, caps, bits
# --------------------------------------------------------------------------

def _primes_upto(n: int):
    return [p for p in range(2, n + 1) if all(p % d for d in range(2, int(math.isqrt(p)) + 1))]


def max_product_moduli(Q: int, m_max: int = 239, m_min: int = 2):
    """Q pairwise-coprime integers in [m_min, m_max] with the largest product,
    in decreasing order (ties broken towards the smaller largest modulus)."""
    small = _primes_upto(math.isqrt(m_max))
    bit = {p: 1 << i for i, p in enumerate(small)}

    def split(n):
        mask, rest = 0, n
        for p in small:
            if rest % p == 0:
                mask |= bit[p]
                while rest % p == 0:
                    rest //= p
        return mask, (rest if rest > 1 else None)

    singles, groups = [], {}
    for n in range(max(2, m_min), m_max + 1):
        mask, big = split(n)
        if big is None:
            singles.append([(n, mask)])
        else:
            groups.setdefault(big, []).append((n, mask))
    # state (mask of small primes used, count) -> (product, -largest, members)
    dp = {(0, 0): (1, 0, ())}
    for grp in singles + list(groups.values()):
        new = dict(dp)
        for (mask, c), (prod, negmax, mem) in dp.items():
            if c >= Q:
                continue
            for n, nm in grp:
                if nm & mask:
                    continue
                key = (mask | nm, c + 1)
                cand = (prod * n, min(negmax, -n), mem + (n,))
                old = new.get(key)
                if old is None or cand[:2] > old[:2]:
                    new[key] = cand
        dp = new
    best = None
    for (mask, c), val in dp.items():
        if c == Q and (best is None or val[:2] > best[:2]):
            best = val
    if best is None:
        raise ValueError(f"no {Q} pairwise-coprime integers up to {m_max}")
    return sorted(best[2], reverse=True)


def modulus_product(moduli) -> int:
    return math.prod(int(m) for m in moduli)


def radius(m: int) -> int:
    """Largest magnitude of the representative nearest zero modulo m."""
    return m // 2


def r_max(ell: int, K: int, lam: int = INT32_LAMBDA) -> int:
    """eq. rmax: floor(sqrt(Lambda / (ell K)))."""
    return math.isqrt(lam // (ell * K)) if lam // (ell * K) > 0 else 0


def caps(moduli, beta: int = 53, lam: int = INT32_LAMBDA):
    """eq. caps for a one-limb configuration: (kappa_rec, kappa_acc, K_max).

    kappa_rec = (P - 1) / (2 B_A B_B), B = 2^beta - 1 (eq. ov-crtgen);
    kappa_acc = Lambda / r^2 with r the largest representative magnitude
    (eq. ov-accgen with one GEMM per accumulator)."""
    P = modulus_product(moduli)
    B = 2**beta - 1
    k_rec = (P - 1) // (2 * B * B)
    r = max(radius(int(m)) for m in moduli)
    k_acc = lam // (r * r)
    return k_rec, k_acc, min(k_rec, k_acc)


def beta_max(moduli, K: int) -> int:
    """Largest beta with 2 K (2^beta - 1)^2 < P."""
    P = modulus_product(moduli)
    b = 1
    while 2 * K * (2**(b + 1) - 1) ** 2 < P:
        b += 1
    return b if 2 * K * (2**b - 1) ** 2 < P else 0


def counting_bound(K: int, alphabet_size: int = 256, beta: int = 53) -> int:
    """Sec. "Certifying the Least GEMM Count": Q >= log2(2 K B_A B_B + 1) / log2 |S|."""
    B = 2**beta - 1
    n = 2 * K * B * B + 1
    # least Q with |S|^Q >= n, in exact integers
    Q = 0
    while alphabet_size**Q < n:
        Q += 1
    return Q


def least_q(K: int, m_max: int = 256, beta: int = 53, lam: int = INT32_LAMBDA) -> int:
    """Least number of one-limb INT8 channels that satisfies eq. ov-crt at K:
    moduli whose representatives fit INT8 ({-128..127}, so m <= 256) and whose
    radius meets eq. ov-acc (radius <= r_max(1))."""
    rm = r_max(1, K, lam)
    top = min(m_max, 2 * rm + 1)
    while top > 2 and radius(top) > rm:
        top -= 1
    need = K * 2**107
    for Q in range(1, 40):
        try:
            mods = max_product_moduli(Q, top)
        except ValueError:
            return -1
        if modulus_product(mods) > need:
            return Q
    return -1


# --------------------------------------------------------------------------
# Wrappers of the C oracle
# --------------------------------------------------------------------------

def _mods(moduli):
    return np.ascontiguousarray(np.asarray(moduli, dtype=np.int32))


def scale(X: np.ndarray, beta: int, axis: int) -> np.ndarray:
    """Shifts s (axis=1: one per row, the A side) or t (axis=0: one per column, the B side)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    R, Ccols = X.shape
    if axis == 1:
        nvec, length, s_vec, s_elem = R, Ccols, Ccols, 1
    else:
        nvec, length, s_vec, s_elem = Ccols, R, 1, Ccols
    out = np.zeros(nvec, dtype=np.int32)
    _check(_load().ozo_scale(_ptr(X), nvec, length, s_vec, s_elem, beta, _ptr(out)), "scale")
    return out


def planes(X: np.ndarray, shifts: np.ndarray, moduli, axis: int) -> np.ndarray:
    """Balanced residue planes [Q][vec][len] (axis=1: rows of A; axis=0: columns of B,
    giving the transposed [Q][N][K] planes)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    R, Ccols = X.shape
    if axis == 1:
        nvec, length, s_vec, s_elem = R, Ccols, Ccols, 1
    else:
        nvec, length, s_vec, s_elem = Ccols, R, 1, Ccols
    mods = _mods(moduli)
    out = np.zeros((len(mods), nvec, length), dtype=np.int16)
    sh = np.ascontiguousarray(shifts, dtype=np.int32)
    _check(_load().ozo_residue_planes(_ptr(X), nvec, length, s_vec, s_elem, _ptr(sh), _ptr(mods), len(mods),
                                      _ptr(out)), "planes")
    return out


def dgemm(A: np.ndarray, B: np.ndarray, moduli, beta: int, want_residues: bool = False):
    """Every entry of the emulated product. Returns C, or (C, W, s, t) with
    W[k][i][j] = (A'B')_ij mod m_k in [0, m_k)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    mods = _mods(moduli)
    C = np.zeros((M, N), dtype=np.float64)
    W = np.zeros((len(mods), M, N), dtype=np.uint16) if want_residues else None
    s = np.zeros(M, dtype=np.int32)
    t = np.zeros(N, dtype=np.int32)
    _check(_load().ozo_dgemm(M, N, K, _ptr(A), K, _ptr(B), N, _ptr(mods), len(mods), beta, _ptr(C), N,
                             _ptr(W), _ptr(s), _ptr(t)), "dgemm")
    return (C, W, s, t) if want_residues else C


def dgemm_entries(A: np.ndarray, B: np.ndarray, moduli, beta: int, rows, cols, want_x: bool = False):
    """Selected entries C[rows[e], cols[e]], each from one row of A and one column of B.
    With want_x, also X (the CRT integer) as Python ints."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    _, N = B.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    mods = _mods(moduli)
    out = np.zeros(len(r), dtype=np.float64)
    xw = np.zeros((len(r), 4), dtype=np.uint64) if want_x else None
    _check(_load().ozo_dgemm_entries(M, N, K, _ptr(A), K, _ptr(B), N, _ptr(mods), len(mods), beta, len(r),
                                     _ptr(r), _ptr(c), _ptr(out), _ptr(xw)), "dgemm_entries")
    if not want_x:
        return out
    return out, [_words_to_int(w) for w in xw]


def _words_to_int(w) -> int:
    v = sum(int(x) << (64 * q) for q, x in enumerate(w))
    return v - (1 << 256) if v >> 255 else v


def _int_to_words(v: int):
    v %= 1 << 256
    return [(v >> (64 * q)) & (2**64 - 1) for q in range(4)]


def crt(residues, moduli):
    """CRT alone: residues [n][Q] in [0, m_k) -> list of X in [-P/2, P/2)."""
    w = np.ascontiguousarray(residues, dtype=np.int32)
    mods = _mods(moduli)
    n = w.shape[0]
    out = np.zeros((n, 4), dtype=np.uint64)
    _check(_load().ozo_crt(n, _ptr(w), _ptr(mods), len(mods), _ptr(out)), "crt")
    return [_words_to_int(x) for x in out]


def round_scaled(xs, exps) -> np.ndarray:
    """fl(X * 2^e) for integers |X| < 2^255, one rounding to nearest even."""
    words = np.ascontiguousarray(np.array([_int_to_words(int(x)) for x in xs], dtype=np.uint64).reshape(-1, 4))
    e = np.ascontiguousarray(exps, dtype=np.int64)
    out = np.zeros(len(e), dtype=np.float64)
    _check(_load().ozo_round(len(e), _ptr(words), _ptr(e), _ptr(out)), "round")
    return out


def exact_error(A: np.ndarray, B: np.ndarray, C, rows, cols):
    """|C_ij - (AB)_ij| formed exactly and rounded once, and (|A||B|)_ij in binary64,
    at the selected entries. C may be None (then the first output is |(AB)_ij|)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    _, N = B.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    Cc = None if C is None else np.ascontiguousarray(C, dtype=np.float64)
    err = np.zeros(len(r), dtype=np.float64)
    ab = np.zeros(len(r), dtype=np.float64)
    _check(_load().ozo_exact_error(M, N, K, _ptr(A), K, _ptr(B), N, _ptr(Cc), N if Cc is not None else 0,
                                   len(r), _ptr(r), _ptr(c), _ptr(err), _ptr(ab)), "exact_error")
    return err, ab


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS or the CPU count)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)
