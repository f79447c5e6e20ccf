"""Pins for the oracle's long polynomial product in Z_p[X] (the workload of
Sec. 6: degree-N polynomials, Table 2's comparison of the classical method
with the d-FQT).  CPU only."""
import numpy as np
import pytest


def binom_mod_p(n, r, p):
    """C(n, r) mod p by Lucas's theorem (base-p digits), small digits by
    Pascal's rule: independent of any convolution."""
    pascal = [[1]]
    for i in range(1, p):
        row = [1] * (i + 1)
        for j in range(1, i):
            row[j] = pascal[i - 1][j - 1] + pascal[i - 1][j]
        pascal.append(row)
    out = 1
    while n or r:
        ni, ri = n % p, r % p
        if ri > ni:
            return 0
        out = out * pascal[ni][ri] % p
        n //= p
        r //= p
    return out


@pytest.mark.parametrize("p,N", [(3, 500), (7, 130), (2, 255), (251, 40)])
def test_binomial_square_by_lucas(orc, p, N):
    """(1+X)^N * (1+X)^N = (1+X)^(2N); the coefficients of (1+X)^N and of
    the product both come from Lucas's theorem."""
    a = np.array([[binom_mod_p(N, i, p) for i in range(N + 1)]])
    out = orc.polymul_long(p, a, a)[0]
    assert out.tolist() == [binom_mod_p(2 * N, c, p) for c in range(2 * N + 1)]


@pytest.mark.parametrize("p,N,count", [(3, 500, 6), (5, 17, 40), (101, 63, 10), (2, 0, 5)])
def test_against_numpy_convolve(orc, p, N, count):
    rng = np.random.default_rng(p + N)
    a = rng.integers(0, p, (count, N + 1))
    b = rng.integers(0, p, (count, N + 1))
    out = orc.polymul_long(p, a, b)
    for s in range(count):
        assert np.array_equal(out[s], np.convolve(a[s], b[s]) % p)


def test_evaluation_homomorphism(orc):
    """(a b)(x) = a(x) b(x) in Z_p for every x in Z_p."""
    p, N = 7, 300
    rng = np.random.default_rng(3)
    a = rng.integers(0, p, (4, N + 1))
    b = rng.integers(0, p, (4, N + 1))
    out = orc.polymul_long(p, a, b)

    def ev(c, x):
        v = 0
        for coef in reversed([int(t) for t in c]):
            v = (v * x + coef) % p
        return v

    for s in range(4):
        for x in range(p):
            assert ev(out[s], x) == ev(a[s], x) * ev(b[s], x) % p


def test_shift_and_unit(orc):
    p, N = 3, 50
    rng = np.random.default_rng(4)
    a = rng.integers(0, p, (1, N + 1))
    for j in (0, 1, 17, N):
        xj = np.zeros((1, N + 1), dtype=np.int64)
        xj[0, j] = 1
        out = orc.polymul_long(p, a, xj)[0]
        want = np.zeros(2 * N + 1, dtype=np.int64)
        want[j:j + N + 1] = a[0]
        assert np.array_equal(out, want)


def test_matches_short_products(orc):
    """Degree k-1 products agree with the separately pinned short product
    routine (Alg. 1's ENSURE)."""
    rng = np.random.default_rng(5)
    for p, k in [(7, 4), (3, 8), (31, 2)]:
        a = rng.integers(0, p, (200, k))
        b = rng.integers(0, p, (200, k))
        assert np.array_equal(orc.polymul_long(p, a, b), orc.polymul(p, a, b))


def test_reduces_inputs_mod_p(orc):
    a = np.array([[10, -4, 7]])
    b = np.array([[3, 3, -1]])
    assert np.array_equal(orc.polymul_long(5, a, b), orc.polymul_long(5, a % 5, b % 5))
