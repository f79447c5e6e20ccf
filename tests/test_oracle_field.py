"""Pins for the oracle's field construction and arithmetic (CPU only).

Every check compares the oracle with something that is not the oracle:
published values, counting formulas, a companion-matrix field model, or a
library routine (numpy convolution / matmul)."""
import itertools
import json
import os

import numpy as np
import pytest

from tests import _pins

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# Defining polynomials and generators used by the workloads (smallest by the
# value sum a_i p^i of the low coefficients, smallest primitive element).
FIELDS = {
    (3, 3): ([1, 2, 0, 1], [0, 1, 0]),
    (101, 2): ([2, 0, 1], [1, 1]),
    (251, 2): ([1, 0, 1], None),
    (2, 8): ([1, 1, 0, 1, 1, 0, 0, 0, 1], [1, 1, 0, 0, 0, 0, 0, 0]),
    (7, 4): ([1, 1, 0, 0, 1], [5, 1, 0, 0]),
    (31, 2): ([1, 0, 1], [4, 1]),
}


def test_is_prime(orc):
    primes = [p for p in range(2, 300) if all(p % d for d in range(2, int(p ** 0.5) + 1))]
    assert [p for p in range(300) if orc.is_prime(p)] == primes


@pytest.mark.parametrize("p,k,count", json.load(open(os.path.join(GOLD, "external_pins.json")))
                         ["irreducible_counts"]["cases"])
def test_irreducible_count_matches_gauss(orc, p, k, count):
    n = 0
    for v in range(p ** k):
        poly = _pins.digits(v, p, k) + [1]
        n += orc.irreducible(p, poly)
    assert n == count


@pytest.mark.parametrize("p,k", [(3, 2), (3, 3), (5, 2), (5, 3), (7, 2), (2, 3)])
def test_irreducible_low_degree_is_rootless(orc, p, k):
    # degree 2 and 3: irreducible <=> no root in Z_p
    for v in range(p ** k):
        poly = _pins.digits(v, p, k) + [1]
        has_root = any(sum(c * x ** i for i, c in enumerate(poly)) % p == 0 for x in range(p))
        assert orc.irreducible(p, poly) == (not has_root), poly


@pytest.mark.parametrize("pk", list(FIELDS))
def test_smallest_irreducible(orc, pk):
    p, k = pk
    poly = orc.smallest_irreducible(p, k)
    assert poly == FIELDS[pk][0]
    if p ** k <= 3000:
        assert _pins.is_field(p, poly)
    # every polynomial of smaller value is reducible: has a root (k <= 3) or
    # leaves zero divisors (k >= 4, small fields only)
    v = _pins.value(poly[:-1], p)
    for w in range(v):
        cand = _pins.digits(w, p, k) + [1]
        if k <= 3:
            assert any(sum(c * x ** i for i, c in enumerate(cand)) % p == 0 for x in range(p))
        elif p ** k <= 300:
            assert not _pins.is_field(p, cand)


def test_aes_field_product(orc):
    pin = json.load(open(os.path.join(GOLD, "external_pins.json")))["aes_gf256"]
    a = _pins.digits(pin["a"], 2, 8)
    b = _pins.digits(pin["b"], 2, 8)
    assert _pins.value(orc.field_mul(2, pin["poly"], a, b), 2) == pin["product"]


@pytest.mark.parametrize("p,k", [(3, 2), (2, 4), (3, 3)])
def test_field_mul_all_pairs_vs_companion(orc, p, k):
    poly = orc.smallest_irreducible(p, k)
    elems = [_pins.digits(v, p, k) for v in range(p ** k)]
    for a, b in itertools.product(elems, elems):
        assert orc.field_mul(p, poly, a, b) == _pins.mul(p, poly, a, b)


@pytest.mark.parametrize("pk", [(101, 2), (7, 4), (2, 8), (31, 2), (251, 2)])
def test_field_mul_sampled_vs_companion(orc, pk):
    p, k = pk
    poly = FIELDS[pk][0]
    rng = np.random.default_rng(11)
    for _ in range(300):
        a = rng.integers(0, p, k).tolist()
        b = rng.integers(0, p, k).tolist()
        assert orc.field_mul(p, poly, a, b) == _pins.mul(p, poly, a, b)


@pytest.mark.parametrize("pk", [(3, 3), (7, 4), (31, 2), (101, 2)])
def test_field_invariants(orc, pk):
    p, k = pk
    poly = FIELDS[pk][0]
    rng = np.random.default_rng(5)
    q = p ** k
    for _ in range(40):
        a, b, c = (rng.integers(0, p, k).tolist() for _ in range(3))
        # distributivity a(b+c) = ab + ac
        bc = [(x + y) % p for x, y in zip(b, c)]
        lhs = orc.field_mul(p, poly, a, bc)
        rhs = [(x + y) % p for x, y in zip(orc.field_mul(p, poly, a, b), orc.field_mul(p, poly, a, c))]
        assert lhs == rhs
        # Frobenius fixes everything: a^(p^k) = a
        x = [1] + [0] * (k - 1)
        e, base = q, list(a)
        while e:
            if e & 1:
                x = orc.field_mul(p, poly, x, base)
            base = orc.field_mul(p, poly, base, base)
            e >>= 1
        assert x == list(a)
        # inverse round trip a * a^(q-2) = 1
        if any(a):
            inv = [1] + [0] * (k - 1)
            e, base = q - 2, list(a)
            while e:
                if e & 1:
                    inv = orc.field_mul(p, poly, inv, base)
                base = orc.field_mul(p, poly, base, base)
                e >>= 1
            assert orc.field_mul(p, poly, a, inv) == [1] + [0] * (k - 1)


@pytest.mark.parametrize("pk", [pk for pk in FIELDS if FIELDS[pk][1] is not None])
def test_generator_is_smallest_primitive(orc, pk):
    p, k = pk
    poly, g_expected = FIELDS[pk]
    g = orc.generator(p, poly)
    assert g == g_expected
    assert _pins.is_primitive(p, poly, g)
    assert orc.order(p, poly, g) == p ** k - 1
    for w in range(1, _pins.value(g, p)):
        assert not _pins.is_primitive(p, poly, _pins.digits(w, p, k))


def test_generator_gf251_2_is_primitive(orc):
    poly = FIELDS[(251, 2)][0]
    g = orc.generator(251, poly)
    assert _pins.is_primitive(251, poly, g)


@pytest.mark.parametrize("pk", [(3, 3), (7, 4), (31, 2), (2, 8)])
def test_antilog_table(orc, pk):
    p, k = pk
    poly = FIELDS[pk][0]
    T = orc.antilog(p, poly)
    q = p ** k
    assert T.shape == (q, k)
    assert not T[q - 1].any()                          # code q-1 is zero
    vals = {_pins.value(row, p) for row in T[: q - 1]}
    assert vals == set(range(1, q))                    # bijection onto F*
    g = T[1].tolist()
    M = _pins.mult_matrix(p, poly, g)
    nxt = (T[: q - 2].astype(np.int64) @ M.T) % p      # g^(e+1) = g * g^e
    assert np.array_equal(nxt, T[1: q - 1])


@pytest.mark.parametrize("pk,shape", [((3, 3), (5, 7, 6)), ((101, 2), (4, 9, 3)),
                                      ((2, 8), (3, 5, 4)), ((7, 4), (6, 4, 5)),
                                      ((31, 2), (7, 3, 8))])
def test_gemm_vs_companion_blocks(orc, pk, shape):
    p, k = pk
    poly = FIELDS[pk][0]
    m, K, n = shape
    rng = np.random.default_rng(3)
    h = max(1, (p - 1) // 2)
    A = rng.integers(-h, h + 1, (m, K, k))            # centred inputs are allowed
    B = rng.integers(0, p, (K, n, k))
    assert np.array_equal(orc.gemm(p, poly, A, B), _pins.gemm(p, poly, A, B))


def test_gemm_prime_field_is_numpy_matmul(orc):
    p = 97
    rng = np.random.default_rng(4)
    A = rng.integers(0, p, (13, 21))
    B = rng.integers(0, p, (21, 17))
    C = orc.gemm(p, [0, 1], A[..., None], B[..., None])[..., 0]
    assert np.array_equal(C, (A @ B) % p)


def test_gemm_associative(orc):
    p, k = 7, 4
    poly = FIELDS[(7, 4)][0]
    rng = np.random.default_rng(8)
    A, B, C = (rng.integers(0, p, s + (k,)) for s in [(3, 4), (4, 5), (5, 2)])
    left = orc.gemm(p, poly, orc.gemm(p, poly, A, B), C)
    right = orc.gemm(p, poly, A, orc.gemm(p, poly, B, C))
    assert np.array_equal(left, right)


def test_gemm_entries_match_full(orc):
    p, k = 101, 2
    poly = FIELDS[(101, 2)][0]
    rng = np.random.default_rng(9)
    A = rng.integers(-50, 51, (9, 33, k))
    B = rng.integers(-50, 51, (33, 11, k))
    C = orc.gemm(p, poly, A, B)
    ii = rng.integers(0, 9, 20)
    jj = rng.integers(0, 11, 20)
    assert np.array_equal(orc.gemm_entries(p, poly, A, B, ii, jj), C[ii, jj])


@pytest.mark.parametrize("p,k", [(7, 4), (3, 3), (251, 2), (2, 8)])
def test_polymul_is_convolution(orc, p, k):
    rng = np.random.default_rng(2)
    a = rng.integers(0, p, (200, k))
    b = rng.integers(0, p, (200, k))
    out = orc.polymul(p, a, b)
    ref = np.stack([np.convolve(x, y) % p for x, y in zip(a, b)])
    assert np.array_equal(out, ref)


def test_example1_polymul(orc):
    ex = json.load(open(os.path.join(GOLD, "paper_examples.json")))["example1"]
    assert orc.polymul(ex["p"], [ex["a"]], [ex["b"]])[0].tolist() == ex["result"]
    assert int(orc.qadic_value(ex["a"], ex["q"])) == ex["a_tilde"]
    assert int(orc.qadic_value(ex["b"], ex["q"])) == ex["b_tilde"]


def test_centred_representation(orc):
    for p in [2, 3, 7, 101, 251]:
        c = np.arange(p)
        r = orc.centred(c, p)
        assert np.array_equal(r % p, c)
        h = 1 if p == 2 else (p - 1) // 2
        assert r.min() >= (0 if p == 2 else -h) and r.max() <= h
