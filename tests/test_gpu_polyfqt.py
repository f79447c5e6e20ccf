"""GPU parity of the d-FQT long polynomial product (Sec. 6) against the
oracle's schoolbook product, element by element, bit-exact."""
import numpy as np
import pytest

import paper_0710_0510_gb300 as q
from paper_0710_0510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def valid_ds(p, int_words, top=8):
    out = []
    for d in range(top):
        try:
            q.polymul_fqt_info(p, 10, d, int_words)
            out.append(d)
        except q.QadicError:
            pass
    return out


@pytest.mark.parametrize("int_words", [False, True])
@pytest.mark.parametrize("p,N,count", [(3, 500, 37), (7, 130, 64), (2, 255, 33), (31, 64, 50),
                                       (251, 40, 21), (101, 1000, 5), (3, 0, 9), (5, 1, 17),
                                       (3, 2, 8)])
def test_fqt_against_oracle(torch, orc, int_words, p, N, count):
    a, b = W.polylong_pairs(count, N, p, salt=p + N)
    want = orc.polymul_long(p, a, b)
    da, db = dev(torch, a), dev(torch, b)
    for d in valid_ds(p, int_words):
        out = q.polymul_fqt(p, d, da, db, int_words=int_words)
        assert np.array_equal(out.cpu().numpy(), want), d


@pytest.mark.parametrize("int_words", [False, True])
@pytest.mark.parametrize("p,N", [(3, 500), (251, 300), (2, 1000), (7, 2047)])
def test_fqt_all_max_inputs(torch, orc, int_words, p, N):
    """Every coefficient p-1: each chunk of products drives every digit of
    the accumulator to its bound n_q (d+1)(p-1)^2 + (p-1)."""
    a = np.full((3, N + 1), p - 1, np.uint8)
    want = orc.polymul_long(p, a, a)
    da = dev(torch, a)
    for d in valid_ds(p, int_words):
        out = q.polymul_fqt(p, d, da, da, int_words=int_words)
        assert np.array_equal(out.cpu().numpy(), want), d


def test_fqt_bytes_above_p_are_reduced(torch, orc):
    rng = np.random.default_rng(9)
    a = rng.integers(0, 256, (20, 301), dtype=np.uint8)
    b = rng.integers(0, 256, (20, 301), dtype=np.uint8)
    want = orc.polymul_long(7, a % 7, b % 7)
    for int_words in (False, True):
        for d in (0, 2):
            out = q.polymul_fqt(7, d, dev(torch, a), dev(torch, b), int_words=int_words)
            assert np.array_equal(out.cpu().numpy(), want)


def test_fqt_largest_degree_and_grid_stride(torch, orc):
    """N = 4095 (the largest degree whose words fit one CTA for d = 0) and
    more pairs than resident CTAs (grid-stride loop), checked on a sample."""
    p, N = 3, 4095
    a, b = W.polylong_pairs(6, N, p, salt=1)
    want = orc.polymul_long(p, a, b)
    for int_words in (False, True):
        for d in (0, 3):
            out = q.polymul_fqt(p, d, dev(torch, a), dev(torch, b), int_words=int_words)
            assert np.array_equal(out.cpu().numpy(), want), (int_words, d)
    count = 20000
    a, b = W.polylong_pairs(count, 40, p, salt=2)
    out = q.polymul_fqt(p, 2, dev(torch, a), dev(torch, b), int_words=True).cpu().numpy()
    idx = np.random.default_rng(3).choice(count, 300, replace=False)
    assert np.array_equal(out[idx], orc.polymul_long(p, a[idx], b[idx]))
    assert np.array_equal(out[-5:], orc.polymul_long(p, a[-5:], b[-5:]))


def test_fqt_paper_workload_all_pairs(torch, orc):
    """The benchmark's workload (p = 3, N = 500, 16384 pairs) in its timed
    configurations, every pair compared."""
    a, b = W.polylong_pairs(16384, 500, 3)
    want = orc.polymul_long(3, a, b)
    da, db = dev(torch, a), dev(torch, b)
    for int_words in (False, True):
        for d in valid_ds(3, int_words):
            out = q.polymul_fqt(3, d, da, db, int_words=int_words)
            assert np.array_equal(out.cpu().numpy(), want), (int_words, d)
