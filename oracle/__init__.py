"""Oracle for GF(p^k) matrix multiplication through the q-adic transform.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the library path never does.  It
shares no code with the CUDA path (own field construction, own tables, own
bounds) and never imports it.

The heavy routines are plain C (``oracle.c``, schoolbook integer arithmetic on
coefficient vectors) loaded through ctypes; the small definitional helpers
below are plain Python/numpy.  Each helper cites the passage of the paper it
restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into a shared library with gcc (-O2, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _c():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            f64p = ctypes.POINTER(ctypes.c_double)
            u32, u64, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            sig = {
                "or_num_threads": (ctypes.c_int, []),
                "or_set_threads": (None, [ctypes.c_int]),
                "or_is_prime": (ctypes.c_int, [u32]),
                "or_irreducible": (ctypes.c_int, [u32, u32, u32p]),
                "or_smallest_irreducible": (ctypes.c_int, [u32, u32, u32p]),
                "or_field_mul": (None, [u32, u32, u32p, u32p, u32p, u32p]),
                "or_order": (u64, [u32, u32, u32p, u32p]),
                "or_generator": (ctypes.c_int, [u32, u32, u32p, u32p]),
                "or_antilog": (None, [u32, u32, u32p, u32p, u32p]),
                "or_gemm": (None, [u32, u32, u32p, i64, i64, i64, i32p, i32p, u32p]),
                "or_dot_batch": (None, [u32, u32, u32p, i64, i64, i32p, i32p, u32p]),
                "or_polymul": (None, [u32, u32, i64, i32p, i32p, u32p]),
                "or_polymul_long": (None, [u32, i64, i64, i32p, i32p, u32p]),
                "or_redq": (None, [u32, u64, u32, i64, f64p, f64p]),
                "or_redq_digits_u128": (None, [u32, u64, u32, u64, u64, u32p]),
                "or_redq_alg2_u128": (None, [u32, u64, u32, u64, u64, u64p, i64p, u32p]),
                "or_lemma1_floor": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def num_threads() -> int:
    return int(_c().or_num_threads())


def set_threads(n: int) -> None:
    """Threads used by the OpenMP loops from now on (CPU timing runs)."""
    _c().or_set_threads(int(n))


# ---------------------------------------------------------------- field ----

def is_prime(p: int) -> bool:
    return bool(_c().or_is_prime(p))


def irreducible(p: int, poly) -> bool:
    """poly: k+1 coefficients low->high, monic.  Exhaustive factor search."""
    P = _u32(poly)
    return bool(_c().or_irreducible(p, len(P) - 1, _ptr(P, ctypes.c_uint32)))


def smallest_irreducible(p: int, k: int) -> list[int]:
    """Monic irreducible of degree k with the smallest value sum a_i p^i."""
    P = np.zeros(k + 1, dtype=np.uint32)
    if _c().or_smallest_irreducible(p, k, _ptr(P, ctypes.c_uint32)) != 0:
        raise ValueError(f"no irreducible polynomial for p={p}, k={k}")
    return [int(x) for x in P]


def field_mul(p: int, poly, a, b) -> list[int]:
    """a*b in Z_p[X]/(P): schoolbook product, mod p, long division (Sec. 7)."""
    P = _u32(poly)
    k = len(P) - 1
    A, B = _u32(a), _u32(b)
    C = np.zeros(k, dtype=np.uint32)
    _c().or_field_mul(p, k, _ptr(P, ctypes.c_uint32), _ptr(A, ctypes.c_uint32),
                      _ptr(B, ctypes.c_uint32), _ptr(C, ctypes.c_uint32))
    return [int(x) for x in C]


def order(p: int, poly, a) -> int:
    P = _u32(poly)
    A = _u32(a)
    return int(_c().or_order(p, len(P) - 1, _ptr(P, ctypes.c_uint32), _ptr(A, ctypes.c_uint32)))


def generator(p: int, poly) -> list[int]:
    """Primitive element with the smallest value sum c_i p^i."""
    P = _u32(poly)
    k = len(P) - 1
    g = np.zeros(k, dtype=np.uint32)
    if _c().or_generator(p, k, _ptr(P, ctypes.c_uint32), _ptr(g, ctypes.c_uint32)) != 0:
        raise ValueError("no generator")
    return [int(x) for x in g]


def antilog(p: int, poly, g=None) -> np.ndarray:
    """(p^k, k) table: row e = coefficients of g^e, row p^k-1 = zero.

    Field elements stored as discrete logarithms of a generator (Sec. 7,
    Alg. 4's input requirement)."""
    P = _u32(poly)
    k = len(P) - 1
    if g is None:
        g = generator(p, poly)
    G = _u32(g)
    T = np.zeros((p ** k, k), dtype=np.uint32)
    _c().or_antilog(p, k, _ptr(P, ctypes.c_uint32), _ptr(G, ctypes.c_uint32),
                    _ptr(T, ctypes.c_uint32))
    return T


# ----------------------------------------------------------------- GEMM ----

def gemm(p: int, poly, A, B) -> np.ndarray:
    """C = A*B over GF(p^k).  A: (m, K, k), B: (K, n, k) integer coefficients
    (any integers, taken mod p).  Returns (m, n, k) uint32 in [0, p-1].

    Each entry is sum_l A_il B_lj with the schoolbook products accumulated in
    int64, then mod p, then mod P (Alg. 4 ENSURE: R = v1^T v2)."""
    P = _u32(poly)
    k = len(P) - 1
    A, B = _i32(A), _i32(B)
    m, K, ka = A.shape
    K2, n, kb = B.shape
    assert ka == k and kb == k and K2 == K
    C = np.zeros((m, n, k), dtype=np.uint32)
    _c().or_gemm(p, k, _ptr(P, ctypes.c_uint32), m, n, K, _ptr(A, ctypes.c_int32),
                 _ptr(B, ctypes.c_int32), _ptr(C, ctypes.c_uint32))
    return C


def dot_batch(p: int, poly, rows, cols) -> np.ndarray:
    """rows, cols: (count, K, k).  Entry s = sum_l rows[s,l] * cols[s,l]."""
    P = _u32(poly)
    k = len(P) - 1
    R, C = _i32(rows), _i32(cols)
    count, K, kk = R.shape
    assert C.shape == R.shape and kk == k
    out = np.zeros((count, k), dtype=np.uint32)
    _c().or_dot_batch(p, k, _ptr(P, ctypes.c_uint32), K, count, _ptr(R, ctypes.c_int32),
                      _ptr(C, ctypes.c_int32), _ptr(out, ctypes.c_uint32))
    return out


def gemm_entries(p: int, poly, A, B, ii, jj) -> np.ndarray:
    """Entries C[ii[s], jj[s]] of A*B, one by one.  A: (m, K, k), B: (K, n, k)."""
    A = np.asarray(A)
    B = np.asarray(B)
    ii = np.asarray(ii)
    jj = np.asarray(jj)
    rows = A[ii]                          # (count, K, k)
    cols = np.transpose(B[:, jj], (1, 0, 2))  # (count, K, k)
    return dot_batch(p, poly, rows, cols)


# -------------------------------------------------------------- polymul ----

def polymul(p: int, a, b) -> np.ndarray:
    """Products in Z_p[X] (Alg. 1 ENSURE, R = v1.v2, no defining polynomial).
    a, b: (count, k).  Returns (count, 2k-1) in [0, p-1]."""
    A, B = _i32(a), _i32(b)
    count, k = A.shape
    out = np.zeros((count, 2 * k - 1), dtype=np.uint32)
    _c().or_polymul(p, k, count, _ptr(A, ctypes.c_int32), _ptr(B, ctypes.c_int32),
                    _ptr(out, ctypes.c_uint32))
    return out


def polymul_long(p: int, a, b) -> np.ndarray:
    """Products of degree-N polynomials in Z_p[X] (Sec. 6's workload): a, b
    (count, N+1), lowest coefficient first.  Returns (count, 2N+1) in
    [0, p-1]: the schoolbook convolution, accumulated in int64, mod p."""
    A, B = _i32(a), _i32(b)
    count, n1 = A.shape
    assert B.shape == A.shape and n1 >= 1
    out = np.zeros((count, 2 * n1 - 1), dtype=np.uint32)
    _c().or_polymul_long(p, n1 - 1, count, _ptr(A, ctypes.c_int32), _ptr(B, ctypes.c_int32),
                         _ptr(out, ctypes.c_uint32))
    return out


# ----------------------------------------------------------------- REDQ ----

def redq(p: int, q: int, d: int, words) -> np.ndarray:
    """Alg. 2 ENSURE for each word: rho = sum_{i<=d} (mu~_i mod p) q^i, where
    mu~_i are the base-q digits of the word (the top one unbounded)."""
    W = np.ascontiguousarray(np.asarray(words, dtype=np.float64))
    out = np.zeros_like(W)
    _c().or_redq(p, q, d, W.size, _ptr(W, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def redq_digits_u128(p: int, q: int, d: int, r: int) -> list[int]:
    mu = np.zeros(d + 1, dtype=np.uint32)
    _c().or_redq_digits_u128(p, q, d, r & (2 ** 64 - 1), r >> 64, _ptr(mu, ctypes.c_uint32))
    return [int(x) for x in mu]


def redq_alg2_u128(p: int, q: int, d: int, r: int):
    """Alg. 2's intermediate values: (rop, [u_0..u_d], [mu_0..mu_d])."""
    rop = np.zeros(2, dtype=np.uint64)
    u = np.zeros(d + 1, dtype=np.int64)
    mu = np.zeros(d + 1, dtype=np.uint32)
    _c().or_redq_alg2_u128(p, q, d, r & (2 ** 64 - 1), r >> 64, _ptr(rop, ctypes.c_uint64),
                           _ptr(u, ctypes.c_int64), _ptr(mu, ctypes.c_uint32))
    return int(rop[0]) + (int(rop[1]) << 64), [int(x) for x in u], [int(x) for x in mu]


def lemma1_floor(r: float, p: float) -> float:
    """floor((r * (1/p)_up)_up), both operations rounded toward +infinity
    (Lemma 1)."""
    return float(_c().or_lemma1_floor(float(r), float(p)))


# ------------------------------------------------------- representations ----

def qadic_value(coeffs, q: int) -> np.ndarray:
    """The q-adic substitution a~ = sum_i alpha_i q^i (Eq. 1), exact in int64.
    coeffs: (..., k)."""
    c = np.asarray(coeffs, dtype=np.int64)
    k = c.shape[-1]
    powers = np.array([q ** i for i in range(k)], dtype=np.int64)
    return (c * powers).sum(axis=-1)


def centred(coeffs, p: int) -> np.ndarray:
    """Centred representative in [-(p-1)/2, (p-1)/2] (Sec. 6, Eq. 3's centred
    representation); p = 2 keeps {0, 1}."""
    c = np.asarray(coeffs, dtype=np.int64) % p
    if p == 2:
        return c
    h = (p - 1) // 2
    return np.where(c > h, c - p, c)


# --------------------------------------------------------------- bounds ----

def qadic_bounds(p: int, k: int, mantissa_bits: int = 53):
    """(q, n_q) under Eq. 2 with q a power of two: the largest power of two
    with (2k-1) log2 q < m, then the largest n_q with q > n_q k (p-1)^2.
    Returns (q, n_q); n_q = 0 means Eq. 2 cannot hold."""
    s = (mantissa_bits - 1) // (2 * k - 1)
    while (2 * k - 1) * s >= mantissa_bits:
        s -= 1
    q = 2 ** s
    step = k * (p - 1) ** 2
    n_q = (q - 1) // step if step else 0
    return q, n_q


def smallest_power_of_two_above(x: int) -> int:
    """Smallest power of two strictly greater than x (the q of Alg. 1 for a
    single product, n_q = 1)."""
    q = 1
    while q <= x:
        q *= 2
    return q


def delayed_k_bound(p: int, k: int, acc_bits: int = 31) -> int:
    """Largest K such that every plane-sum coefficient of K products of
    centred elements stays in a signed accumulator of acc_bits magnitude
    bits: each output coefficient collects at most k*K products of size
    h^2 with h = (p-1)/2 (Eq. 3 with the centred representation)."""
    h = 1 if p == 2 else (p - 1) // 2
    return (2 ** acc_bits - 1) // (k * h * h)
