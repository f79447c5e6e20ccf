"""Pins for the oracle's REDQ (Alg. 2), the tabulated corrections (Sec. 5)
and the floating-point floor (Lemma 1).  CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EX = json.load(open(os.path.join(GOLD, "paper_examples.json")))


def test_example2_p_divides_q(orc):
    ex = EX["example2"]
    p, q = ex["p"], ex["q"]
    r = int(orc.qadic_value(ex["a"], q)) * int(orc.qadic_value(ex["b"], q))
    assert r == ex["product"]
    rop, u, mu = orc.redq_alg2_u128(p, q, 4, r)
    assert rop == ex["rop"]
    assert mu == ex["result"]
    assert orc.redq_digits_u128(p, q, 4, r) == ex["result"]
    assert sum(m * q ** i for i, m in enumerate(mu)) == ex["rho"]
    # the p | q shortcut of the example: rho = r - p * (quotient digits)
    quot = sum(((r // q ** i) % q // p) * q ** i for i in range(5))
    assert r - p * quot == ex["rho"]


def test_example3_full_redq(orc):
    ex = EX["example3"]
    p, q, r = ex["p"], ex["q"], ex["r"]
    assert int(sum(c * q ** i for i, c in enumerate(ex["coefficients"]))) == r
    rop, u, mu = orc.redq_alg2_u128(p, q, 3, r)
    assert rop == ex["rop"]
    assert rop * p == ex["rop_times_p"]
    assert u == ex["u"]
    assert (-q) % p == ex["minus_q_mod_p"]
    assert mu == ex["mu"]
    assert orc.redq_digits_u128(p, q, 3, r) == ex["mu"]


def test_example1_radix(orc):
    ex = EX["example1"]
    r = ex["product"]
    assert orc.redq_digits_u128(ex["p"], ex["q"], 2, r) == ex["result"]
    assert [(r // ex["q"] ** i) % ex["q"] for i in range(3)] == ex["radix_digits"]


@pytest.mark.parametrize("p,q,d", [(7, 1024, 4), (23, 10 ** 6, 3), (5, 10000, 4), (3, 8, 6),
                                   (101, 2 ** 17, 2), (2, 3, 9), (251, 2 ** 20, 2)])
def test_alg2_agrees_with_plain_digits_and_thm2(orc, p, q, d):
    """Alg. 2's route (one division, shifts, corrections) against the digit
    definition, with Thm. 2's invariants on u_i."""
    rng = np.random.default_rng(p * 1000 + d)
    for _ in range(300):
        dig = [int(x) for x in rng.integers(0, q, d + 1)]
        r = sum(x * q ** i for i, x in enumerate(dig))
        if r >= 2 ** 127:
            continue
        rop, u, mu = orc.redq_alg2_u128(p, q, d, r)
        assert mu == [x % p for x in dig]
        assert orc.redq_digits_u128(p, q, d, r) == mu
        for i in range(d + 1):
            assert 0 <= u[i] < p
            assert u[i] % p == sum(mu[j] * q ** (j - i) for j in range(i, d + 1)) % p


def test_redq_words_all_tuples_small(orc):
    """Every word with 3 base-8 digits, p = 3: the output's digits are the
    inputs' digits mod p (checked through the 128-bit digit routine)."""
    p, q, d = 3, 8, 2
    words = np.arange(q ** (d + 1), dtype=np.float64)
    out = orc.redq(p, q, d, words)
    for w, o in zip(words.astype(int), out.astype(int)):
        mu = orc.redq_digits_u128(p, q, d, int(w))
        assert o == sum(m * q ** i for i, m in enumerate(mu))
        assert all(((o >> (3 * i)) & 7) < p for i in range(d + 1))


def test_redq_of_packed_product_is_polymul(orc):
    """REDQ of a~ b~ = the packed product polynomial mod p (Alg. 1 with
    Alg. 2 as its last steps), against the convolution oracle."""
    p, k = 7, 3
    q = 2 ** 10
    rng = np.random.default_rng(1)
    a = rng.integers(0, p, (500, k))
    b = rng.integers(0, p, (500, k))
    r = orc.qadic_value(a, q) * orc.qadic_value(b, q)
    assert r.max() < 2 ** 53
    rho = orc.redq(p, q, 2 * k - 2, r.astype(np.float64)).astype(np.int64)
    assert np.array_equal(rho, orc.qadic_value(orc.polymul(p, a, b), q))


def test_redq_large_words_vs_u128(orc):
    p, q, d = 7, 2 ** 10, 4
    rng = np.random.default_rng(2)
    w = rng.integers(0, 2 ** 50, 2000)
    out = orc.redq(p, q, d, w.astype(np.float64)).astype(np.int64)
    for x, o in zip(w[:300], out[:300]):
        mu = orc.redq_digits_u128(p, q, d, int(x))
        assert int(o) == sum(m * q ** i for i, m in enumerate(mu))


# ------------------------------------------ q a multiple of p (Sec. 4) ----

def test_example2_result_at_a_smaller_multiple_of_p(orc):
    """Ex. 2's product, packed with q = 100 (also a multiple of p = 5, and
    large enough for its coefficients) so that the word is an exact double:
    the oracle's word-level REDQ returns the example's residues."""
    ex = EX["example2"]
    p, q = ex["p"], 100
    r = int(orc.qadic_value(ex["a"], q)) * int(orc.qadic_value(ex["b"], q))
    assert r < 2 ** 53
    rho = int(orc.redq(p, q, 4, np.array([float(r)]))[0])
    assert [(rho // q ** i) % q for i in range(5)] == ex["result"]


@pytest.mark.parametrize("p,q,d", [(3, 6, 2), (5, 10, 3), (2, 4, 4), (7, 7, 2)])
def test_redq_p_divides_q_shortcut(orc, p, q, d):
    """With p | q the whole reduction is one subtraction (Ex. 2):
    rho = r - p * sum_i floor(mu~_i / p) q^i, over every word with d+1
    base-q digits."""
    words = np.arange(q ** (d + 1), dtype=np.int64)
    out = orc.redq(p, q, d, words.astype(np.float64)).astype(np.int64)
    for w, o in zip(words.tolist(), out.tolist()):
        quot = sum((((w // q ** i) % q) // p) * q ** i for i in range(d + 1))
        assert o == w - p * quot


def test_redq_p_divides_q_sweep_vs_u128(orc):
    p, q, d = 7, 1176, 4
    assert q % p == 0 and q ** (d + 1) <= 2 ** 51
    rng = np.random.default_rng(3)
    digits = rng.integers(0, q, (3000, d + 1))
    words = (digits * np.array([q ** i for i in range(d + 1)])).sum(axis=1)
    out = orc.redq(p, q, d, words.astype(np.float64)).astype(np.int64)
    assert np.array_equal(out, ((digits % p) * np.array([q ** i for i in range(d + 1)])).sum(axis=1))
    for x, o in zip(words[:200].tolist(), out[:200].tolist()):
        mu = orc.redq_digits_u128(p, q, d, int(x))
        assert o == sum(m * q ** i for i, m in enumerate(mu))


@pytest.mark.parametrize("D", [1176, 1176 ** 2, 7 * 1176 ** 3, 1176 ** 4, 7 * 1176 ** 4,
                               10 ** 4, 5 * 10 ** 12])
def test_lemma1_composite_divisors(orc, D):
    """Lemma 1 holds for any positive integer divisor, not only primes: the
    floors by q^j and p q^j near the 2^51 limit."""
    limit = 2 ** 51
    rng = np.random.default_rng(D % 1000003)
    us = [int(x) for x in rng.integers(0, limit // D, 300)] + [limit // D - 1, 0, 1]
    for u in us:
        for i in (0, 1, D - 1):
            r = u * D + i
            if r < limit:
                assert orc.lemma1_floor(float(r), float(D)) == r // D


def test_nested_floor_identity():
    """floor(floor(r/p)/q^j) = floor(r/(p q^j)) (Lemma 2, used in the proof of Thm. 2),
    the identity that lets each digit's second floor divide r directly."""
    rng = np.random.default_rng(5)
    for p, q in [(7, 1176), (5, 10), (3, 8), (251, 251)]:
        for _ in range(2000):
            r = int(rng.integers(0, 2 ** 51))
            for j in range(4):
                assert (r // p) // q ** j == r // (p * q ** j)


# ------------------------------------------------ Sec. 5: Q_d matrices ----

def qd_matrix(d, q, p):
    """Q_d: 1 on the diagonal, -q on the superdiagonal (Sec. 5.1)."""
    Q = np.eye(d + 1, dtype=np.int64)
    for i in range(d):
        Q[i, i + 1] = (-q) % p
    return Q % p


def test_qd_is_inverse_of_power_matrix():
    for p, q, d in [(23, 10 ** 6, 3), (7, 1024, 4), (3, 8, 6)]:
        T = np.zeros((d + 1, d + 1), dtype=object)
        for i in range(d + 1):
            for j in range(i, d + 1):
                T[i, j] = pow(q, j - i, p)
        prod = (qd_matrix(d, q, p).astype(object) @ T) % p
        assert (prod == np.eye(d + 1, dtype=object)).all()


def test_example3_matrix_form(orc):
    ex = EX["example3"]
    mu = (qd_matrix(3, ex["q"], ex["p"]) @ np.array(ex["u"])) % ex["p"]
    assert mu.tolist() == ex["mu"]


@pytest.mark.parametrize("p", [3, 5])
def test_alg3_q6_from_three_q2(p):
    """Alg. 3: Q_6 u = [a0, a1, b0, b1, c0, c1, c2] with a = Q_2 u[0:3],
    b = Q_2 u[2:5], c = Q_2 u[4:7], over every u in Z_p^7."""
    q = 10 if p == 3 else 12
    Q6 = qd_matrix(6, q, p)
    table = {}
    for t in itertools.product(range(p), repeat=3):
        table[t] = tuple(int(x) for x in (qd_matrix(2, q, p) @ np.array(t)) % p)
    for u in itertools.product(range(p), repeat=7):
        a = table[u[0:3]]
        b = table[u[2:5]]
        c = table[u[4:7]]
        assert [a[0], a[1], b[0], b[1], c[0], c[1], c[2]] == ((Q6 @ np.array(u)) % p).tolist()


@pytest.mark.parametrize("d,kk,lookups", EX["table2"]["cases"])
def test_table2_lookup_count(d, kk, lookups):
    """With a table for Q_{kk-1} (p^kk entries) the correction of degree d
    takes ceil(d/(kk-1)) overlapping lookups, and they reproduce Q_d u."""
    assert math.ceil(d / (kk - 1)) == lookups
    p, q = 3, 7
    rng = np.random.default_rng(d * 10 + kk)
    Qs = qd_matrix(kk - 1, q, p)
    starts = [s * (kk - 1) for s in range(lookups)]
    starts[-1] = d + 1 - kk
    for _ in range(50):
        u = rng.integers(0, p, d + 1)
        mu = [None] * (d + 1)
        for idx, s in enumerate(starts):
            part = (Qs @ u[s:s + kk]) % p
            take = kk if idx == len(starts) - 1 else kk - 1
            for j in range(take):
                mu[s + j] = int(part[j])
        assert mu == ((qd_matrix(d, q, p) @ u) % p).tolist()


# ----------------------------------------------------------- Lemma 1 ----

@pytest.mark.parametrize("p", [2, 3, 7, 23, 101, 251])
def test_lemma1_bruteforce_small(orc, p):
    for r in list(range(0, 1 << 14)) + list(range((1 << 24) - 2000, 1 << 24)):
        assert orc.lemma1_floor(r, p) == r // p


@pytest.mark.parametrize("p", [3, 7, 23, 101, 251, 65521])
def test_lemma1_near_limit(orc, p):
    """eps = 2^-52 (round-upward binary64); the lemma's limit
    1/(2 eps + eps^2) is just under 2^51.  Random and worst-case residues
    (i = p - 1) below 2^51."""
    limit = 2 ** 51
    rng = np.random.default_rng(p)
    us = [int(x) for x in rng.integers(0, limit // p, 500)] + [limit // p - 1]
    for u in us:
        for i in (0, 1, p - 1):
            r = u * p + i
            if r < limit:
                assert orc.lemma1_floor(float(r), p) == r // p
