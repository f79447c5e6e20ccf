"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers (numpy ``default_rng``); it holds none
of the method's arithmetic.  Both the CUDA path and the oracle are fed from
it.  Seeds: 7100510 + workload index.
"""
from __future__ import annotations

import numpy as np

SEED = 7100510


def rng(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED + index + 1000003 * salt)


def polymul_pairs(count: int, p: int, k: int, index: int = 0, salt: int = 0):
    """count x k coefficients uniform in [0, p-1] for a and for b (uint8)."""
    g = rng(index, salt)
    a = g.integers(0, p, (count, k), dtype=np.uint8)
    b = g.integers(0, p, (count, k), dtype=np.uint8)
    return a, b


def polylong_pairs(count: int, N: int, p: int, index: int = 5, salt: int = 0):
    """count pairs of degree-N polynomials over Z_p (Sec. 6's workload; the
    paper's example is p = 3, N = 500): coefficients uniform in [0, p-1],
    uint8 arrays of shape (count, N+1)."""
    g = rng(index, salt)
    a = g.integers(0, p, (count, N + 1), dtype=np.uint8)
    b = g.integers(0, p, (count, N + 1), dtype=np.uint8)
    return a, b


def log_matrix(rows: int, cols: int, order: int, index: int = 1, salt: int = 0):
    """Discrete-log codes uniform over all `order` field elements (code
    order-1 is zero): uint8 when order <= 256, else uint16."""
    g = rng(index, salt)
    dt = np.uint8 if order <= 256 else np.uint16
    return g.integers(0, order, (rows, cols), dtype=dt)


def centred_planes(k: int, rows: int, cols: int, h: int, index: int = 2, salt: int = 0):
    """k planes of int8 coefficients uniform in [-h, h]."""
    g = rng(index, salt)
    return g.integers(-h, h + 1, (k, rows, cols), dtype=np.int8)


def coeff_planes(k: int, rows: int, cols: int, p: int, index: int = 3, salt: int = 0):
    """k planes of uint8 coefficients uniform in [0, p-1]."""
    g = rng(index, salt)
    return g.integers(0, p, (k, rows, cols), dtype=np.uint8)


def redq_words(count: int, ndigits: int, log2_q: int, index: int = 4, salt: int = 0):
    """Packed words with `ndigits` base-2^log2_q digits, each uniform in
    [0, 2^log2_q - 1]: a uniform integer below 2^(ndigits*log2_q), as float64."""
    g = rng(index, salt)
    return g.integers(0, 1 << (ndigits * log2_q), count, dtype=np.int64).astype(np.float64)


def redq_words_q(count: int, ndigits: int, q: int, index: int = 4, salt: int = 0):
    """Packed words sum_j mu~_j q^j with the digits independent and uniform
    in [0, q-1] -- the same law as a uniform integer below q^ndigits (the
    base-q digits are a bijection) -- for any q with q^ndigits <= 2^53, as
    float64."""
    g = rng(index, salt)
    return g.integers(0, q ** ndigits, count, dtype=np.int64).astype(np.float64)


def batched_shapes(count: int, lo: int = 16, hi: int = 256, index: int = 3, salt: int = 0):
    """(m, n, K) per product: round(exp(U[ln lo, ln hi])) independently, and a
    field index uniform in {0, 1, 2}."""
    g = rng(index, salt)
    dims = np.rint(np.exp(g.uniform(np.log(lo), np.log(hi), (count, 3)))).astype(np.int64)
    fields = g.integers(0, 3, count)
    return dims, fields
