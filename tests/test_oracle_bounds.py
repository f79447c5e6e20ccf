"""Pins for the bounds the method relies on (Thm. 1 / Eq. 2, Eq. 3) and for
the reading that the single-rounded FP64 product of the 65,536-pair
polynomial workload (p = 7, k = 4, q = 2^8) breaks Eq. 2.  CPU only."""
import numpy as np
import pytest


@pytest.mark.parametrize("p,k,q,nq", [(3, 3, 1024, 85), (101, 2, 2 ** 17, 6), (7, 3, 1024, 9)])
def test_eq2_block_sizes(orc, p, k, q, nq):
    assert orc.qadic_bounds(p, k, 53) == (q, nq)


@pytest.mark.parametrize("p,k", [(3, 3), (101, 2), (31, 2), (7, 3)])
def test_eq2_all_max_exact_at_nq_and_carries_beyond(orc, p, k):
    """n_q products of all-(p-1) elements: every base-q digit of the packed
    sum stays below q and the sum below 2^53 (exact in FP64); one more
    product makes the middle digit carry, so REDQ would return a wrong
    coefficient: the block size must be rejected, not run."""
    q, nq = orc.qadic_bounds(p, k, 53)
    amax = sum((p - 1) * q ** i for i in range(k))
    for n, ok in [(nq, True), (nq + 1, False)]:
        r = n * amax * amax
        digits = [(r // q ** t) % q for t in range(2 * k - 1)]
        true = [n * (p - 1) ** 2 * min(t + 1, 2 * k - 1 - t) for t in range(2 * k - 1)]
        assert (digits == true) == ok
        if ok:
            assert r < 2 ** 53
            # FP64 accumulation of the n products is exact
            acc = 0.0
            for _ in range(n):
                acc += float(amax) * float(amax)
            assert int(acc) == r


def test_single_product_q_config1(orc):
    # Alg. 1 with one product: q the smallest power of two above k (p-1)^2
    assert orc.smallest_power_of_two_above(4 * 6 ** 2) == 256
    # (2k-1) log2 q = 56 >= 53: Eq. 2 fails for binary64, holds for 64-bit words
    assert (2 * 4 - 1) * 8 >= 53
    assert (2 * 4 - 1) * 8 < 64


def test_config1_single_rounded_product_is_inexact():
    """Exhaustive over the 7^8 operand pairs: 21,609 single-rounded FP64
    products differ from the exact product, which is why the plain
    product is rejected for this workload."""
    vals = np.array([sum(((v // 7 ** i) % 7) * 256 ** i for i in range(4))
                     for v in range(7 ** 4)], dtype=np.int64)
    vf = vals.astype(np.float64)
    bad = 0
    for a in vals:
        bad += int(np.count_nonzero((float(a) * vf).astype(np.int64) != a * vals))
    assert bad == 21609
    # ...while the two-term FMA split hi + lo is exact for every pair
    hi = np.multiply.outer(vf[:50], vf)
    lo_exact = np.multiply.outer(vals[:50], vals) - hi.astype(np.int64)
    assert np.abs(lo_exact).max() <= 2 ** 3   # < ulp(2^54)/2: representable


@pytest.mark.parametrize("p,k,K", [(251, 2, 68719), (101, 2, 429496), (2, 8, 268435455 // 1)])
def test_eq4_int32_plane_bound(orc, p, k, K):
    """Centred planes: each product coefficient collects at most k*K
    products of size h^2; K is the largest with k K h^2 < 2^31."""
    h = 1 if p == 2 else (p - 1) // 2
    assert orc.delayed_k_bound(p, k, 31) == K
    assert k * K * h * h <= 2 ** 31 - 1 < k * (K + 1) * h * h
    # Eq. 3 form: n_d (p-1)^2 < 2^(m+1) with m = 31 bits of magnitude
    if p > 2:
        nd = k * K
        assert nd * (p - 1) ** 2 < 2 ** 33
