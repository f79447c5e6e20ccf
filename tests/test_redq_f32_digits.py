"""The FP32 digit arithmetic of QADIC_REDQ_F32_DIGITS, checked on the CPU.

The kernel takes floor(X / m) for integer-valued floats X < 2^21 as the
nearest integer of fma(X, RN(1/m), RN(1/(2m) - 1/2)) (rounded by adding and
subtracting 1.5 * 2^23), then the remainder X - m floor(X / m) by one more
fma.  Here that sequence is replayed with IEEE binary32 rounding (each fma
evaluated exactly in extended precision, then rounded once to binary32) for
every X below q^2 of several (p, q) pairs, including the largest q the flag
admits, and compared with integer floor division; then whole words are
reduced the kernel's way and compared with the definition of REDQ for q a
multiple of p (each base-q digit replaced by its residue mod p, Alg. 2
with the corrections gone since p | q)."""
import numpy as np
import pytest

LD = np.longdouble
if np.finfo(LD).nmant < 60:
    pytest.skip("needs an extended-precision long double to evaluate fma exactly",
                allow_module_level=True)

ROUND = np.float32(12582912.0)   # 1.5 * 2^23


def fma32(a, b, c):
    """fma in binary32: the exact a*b + c (at most 64 significant bits for
    these operands), rounded once."""
    return (a.astype(LD) * LD(b) + LD(c)).astype(np.float32)


def floor_div_f32(X, m):
    inv = np.float32(1.0) / np.float32(m)
    c = np.float32(0.5 / m - 0.5)
    y = fma32(X, inv, c)
    return (y + ROUND) - ROUND


def rem_f32(X, m, t):
    return fma32(t, -np.float32(m), X)   # -m * t + X, exact here


@pytest.mark.parametrize("p,q", [(7, 1176), (2, 1448), (181, 1448), (251, 1255), (3, 1401),
                                 (2, 2), (3, 3), (5, 10), (7, 7)])
def test_floor_by_q_and_p_exact_for_every_chunk(p, q):
    Q = q * q
    assert Q < 2 ** 21
    X = np.arange(Q, dtype=np.float32)
    hi = floor_div_f32(X, q)
    lo = rem_f32(X, q, hi)
    xi = np.arange(Q, dtype=np.int64)
    assert np.array_equal(hi.astype(np.int64), xi // q)
    assert np.array_equal(lo.astype(np.int64), xi % q)
    d = np.arange(q, dtype=np.float32)
    fp = floor_div_f32(d, p)
    assert np.array_equal(fp.astype(np.int64), np.arange(q) // p)
    assert np.array_equal(rem_f32(d, p, fp).astype(np.int64), np.arange(q) % p)


def test_floor_margin_at_the_chunk_limit():
    """X up to 2^21 - 1 for the largest admitted divisor sizes (the error
    bound (2X/m + 3/4) 2^-24 < 1/(2m) holds for every X < 2^21)."""
    X = np.arange(2 ** 21 - 2 ** 16, 2 ** 21, dtype=np.float32)
    xi = X.astype(np.int64)
    for m in (2, 3, 7, 1176, 1447, 1448, 2 ** 20 + 7):
        assert np.array_equal(floor_div_f32(X, m).astype(np.int64), xi // m), m


def reduce_words_f32(words, p, q, nd):
    """The kernel's word: chunks of two digits by integer floors by q^2,
    FP32 floors inside each chunk, Horner in q^2."""
    Q = q * q
    out = []
    for w in words:
        t = int(w)
        nc = (nd + 1) // 2
        c = []
        for _ in range(nc - 1):
            c.append(t % Q)
            t //= Q
        c.append(t)
        rho = 0
        for i in range(nc - 1, -1, -1):
            X = np.array([c[i]], dtype=np.float32)
            if 2 * i + 1 < nd:
                hi = floor_div_f32(X, q)
                lo = rem_f32(X, q, hi)
                uhi = rem_f32(hi, p, floor_div_f32(hi, p))
                ulo = rem_f32(lo, p, floor_div_f32(lo, p))
                r = fma32(uhi, np.float32(q), ulo)
            else:
                r = rem_f32(X, p, floor_div_f32(X, p))
            rho = rho * Q + int(r[0])
        out.append(rho)
    return out


def reduce_words_definition(words, p, q, nd):
    out = []
    for w in words:
        t, rho, qj = int(w), 0, 1
        for _ in range(nd):
            rho += (t % q % p) * qj
            t //= q
            qj *= q
        out.append(rho)
    return out


@pytest.mark.parametrize("p,q,nd", [(7, 1176, 5), (7, 1176, 4), (2, 1448, 5), (181, 1448, 3),
                                    (5, 10, 8), (3, 3, 7), (251, 1255, 1)])
def test_words_match_the_definition(p, q, nd):
    rng = np.random.default_rng(1000 * p + nd)
    top = q ** nd
    words = [0, top - 1, q - 1, q, q * q - 1, q * q] + \
            [int(x) for x in rng.integers(0, top, size=400, dtype=np.int64)]
    words = [w for w in words if w < top]
    assert reduce_words_f32(words, p, q, nd) == reduce_words_definition(words, p, q, nd)
