"""GPU parity: each CUDA kernel, called through the C ABI, against the oracle,
element by element, bit-exact (all results are integers)."""
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


def host(t):
    return t.cpu().numpy()


# ------------------------------------------------------------ polymul ----

@pytest.mark.parametrize("int_words", [False, True])
@pytest.mark.parametrize("count", [1, 255, 257, 4099, 65536, 1 << 20])
def test_polymul_config1(torch, orc, count, int_words):
    a, b = W.polymul_pairs(count, 7, 4, salt=count)
    out = q.polymul_batched(7, 4, dev(torch, a), dev(torch, b), int_words=int_words)
    torch.cuda.synchronize()
    assert np.array_equal(host(out), orc.polymul(7, a, b))


def test_polymul_unaligned_inputs(torch, orc):
    """Operands one byte off a 4-byte boundary take the byte-load path."""
    a, b = W.polymul_pairs(5001, 7, 4, salt=3)
    da = torch.zeros(a.size + 1, dtype=torch.uint8, device="cuda")
    db = torch.zeros(b.size + 1, dtype=torch.uint8, device="cuda")
    da[1:] = dev(torch, a.ravel())
    db[1:] = dev(torch, b.ravel())
    for int_words in (False, True):
        out = q.polymul_batched(7, 4, da[1:].view(5001, 4), db[1:].view(5001, 4),
                                int_words=int_words)
        assert np.array_equal(host(out), orc.polymul(7, a, b))


def test_polymul_example1(torch):
    out = q.polymul_batched(3, 2, dev(torch, np.array([[1, 1]], np.uint8)),
                            dev(torch, np.array([[2, 1]], np.uint8)))
    assert host(out).tolist() == [[2, 0, 1]]


@pytest.mark.parametrize("p,k", [(3, 3), (2, 8), (31, 2), (251, 2), (5, 5), (101, 2)])
def test_polymul_other_rings(torch, orc, p, k):
    a, b = W.polymul_pairs(3000, p, k, salt=p * 10 + k)
    for plain, ints in ((False, False), (True, False), (False, True)):
        try:
            out = q.polymul_batched(p, k, dev(torch, a), dev(torch, b), plain_f64=plain,
                                    int_words=ints)
        except q.QadicError as e:
            assert plain and e.status == q.E_OVERFLOW
            continue
        assert np.array_equal(host(out), orc.polymul(p, a, b))


@pytest.mark.parametrize("p,k", [(7, 4), (3, 3), (2, 8), (251, 2), (5, 5)])
def test_polymul_unreduced_bytes(torch, orc, p, k):
    """Coefficient bytes at or above p are taken mod p; pairs with such bytes
    sit between canonical ones in the same warps (every third pair canonical),
    so both packing paths run side by side."""
    rng = np.random.default_rng(p * 7 + k)
    a = rng.integers(0, 256, (4099, k), dtype=np.uint8)
    b = rng.integers(0, 256, (4099, k), dtype=np.uint8)
    a[::3] %= p
    b[::3] %= p
    b[1::3] %= p                      # some pairs with one canonical operand only
    for int_words in (False, True):
        out = q.polymul_batched(p, k, dev(torch, a), dev(torch, b), int_words=int_words)
        assert np.array_equal(host(out), orc.polymul(p, a, b)), int_words


def test_polymul_all_max(torch, orc):
    a = np.full((1000, 4), 6, np.uint8)
    for int_words in (False, True):
        out = q.polymul_batched(7, 4, dev(torch, a), dev(torch, a), int_words=int_words)
        assert np.array_equal(host(out), orc.polymul(7, a, a))


# --------------------------------------------------------------- REDQ ----

def redq_cases():
    for mode in (0, 1, 2, 3):
        for int_floor in (False, True):
            yield mode, int_floor


@pytest.mark.parametrize("mode,int_floor", list(redq_cases()))
def test_redq_sweep_words(torch, orc, mode, int_floor):
    w = W.redq_words(100001, 5, 10, salt=mode)   # odd count: ragged tail
    out = q.redq(7, 10, 5, dev(torch, w), table_mode=mode, int_floor=int_floor)
    assert np.array_equal(host(out), orc.redq(7, 1024, 4, w))


@pytest.mark.parametrize("p,s,nd", [(5, 8, 6), (23, 12, 4), (101, 17, 3), (251, 16, 3),
                                    (2, 3, 17), (3, 25, 2)])
def test_redq_other_parameters(torch, orc, p, s, nd):
    w = W.redq_words(20000, nd, s, salt=p)
    for mode in (0, 1, 2, 3):
        for int_floor in (False, True):
            out = q.redq(p, s, nd, dev(torch, w), table_mode=mode, int_floor=int_floor)
            assert np.array_equal(host(out), orc.redq(p, 2 ** s, nd - 1, w)), (mode, int_floor)


def test_redq_adversarial_words(torch, orc):
    p, s, nd = 7, 10, 5
    q_ = 1 << s
    digs = [[q_ - 1] * nd, [0] * nd, [p - 1] * nd, [2 * p - 1] * nd, [q_ - 2] * nd,
            [p * (q_ // p) - 1] * nd, [q_ - 1, 0, q_ - 1, 0, q_ - 1]]
    words = np.array([sum(d * q_ ** i for i, d in enumerate(x)) for x in digs] * 3,
                     dtype=np.float64)
    top = float(2 ** 50 - 1)
    words = np.concatenate([words, [top, top - 1, 1.0]])
    for mode in (0, 1, 2, 3):
        for int_floor in (False, True):
            out = q.redq(p, s, nd, dev(torch, words), table_mode=mode, int_floor=int_floor)
            assert np.array_equal(host(out), orc.redq(p, q_, nd - 1, words))


# ------------------------------------------------- REDQ, p divides q ----

@pytest.mark.parametrize("p,q_,nd", [(7, 1176, 5), (5, 10 ** 4, 3), (5, 10, 15), (2, 6, 19),
                                     (251, 251, 6), (2, 1024, 5), (3, 3 * 2 ** 14, 3),
                                     (101, 101 * 64, 3), (13, 13, 1), (7, 7 * 2 ** 20, 2),
                                     (3, 3 * 2 ** 9, 4), (2, 128, 7), (5, 80, 8),
                                     (251, 251 * 2 ** 17, 2), (13, 13 * 2 ** 30, 1),
                                     (2, 2 ** 16, 3), (3, 3 * 2 ** 15, 3)])
def test_redq_pq_parameters(torch, orc, p, q_, nd):
    w = W.redq_words_q(30001, nd, q_, salt=p)   # odd count: ragged tail
    want = orc.redq(p, q_, nd - 1, w)
    for int_floor in (False, True):
        out = q.redq_pq(p, q_, nd, dev(torch, w), int_floor=int_floor)
        assert np.array_equal(host(out), want), int_floor
    if q_ <= 1448 and nd <= 8:      # q^2 < 2^21: the FP32-digit form applies
        out = q.redq_pq(p, q_, nd, dev(torch, w), f32_digits=True)
        assert np.array_equal(host(out), want), "f32 digits"
    else:
        with pytest.raises(q.QadicError):
            q.redq_pq(p, q_, nd, dev(torch, w), f32_digits=True)


@pytest.mark.parametrize("p,q_,nd", [(2, 1448, 4), (181, 1448, 4), (3, 1401, 4), (2, 2, 8),
                                     (5, 5, 1), (7, 1176, 1), (7, 1176, 2), (7, 1176, 3),
                                     (251, 1255, 4), (5, 1445, 4)])
def test_redq_pq_f32_digits_limits(torch, orc, p, q_, nd):
    """The FP32-digit form at its largest q (1448^2 < 2^21), one to eight
    digits, chunks with and without a lone top digit."""
    w = W.redq_words_q(20001, nd, q_, salt=p + nd)
    top = float(q_ ** nd - 1)
    w = np.concatenate([w, [top, 0.0, float(q_ - 1), float(q_)]])
    out = q.redq_pq(p, q_, nd, dev(torch, w), f32_digits=True)
    assert np.array_equal(host(out), orc.redq(p, q_, nd - 1, w))


def test_redq_pq_adversarial_words(torch, orc):
    p, q_, nd = 7, 1176, 5
    digs = [[q_ - 1] * nd, [0] * nd, [p - 1] * nd, [p] * nd, [2 * p - 1] * nd,
            [q_ - p] * nd, [q_ - p - 1] * nd, [q_ - 1, 0, q_ - 1, 0, q_ - 1],
            [0, 0, 0, 0, q_ - 1], [q_ - 1, 0, 0, 0, 0]]
    words = np.array([sum(d * q_ ** i for i, d in enumerate(x)) for x in digs] * 3 + [1.0],
                     dtype=np.float64)
    assert words.max() == q_ ** nd - 1
    for kw in (dict(int_floor=False), dict(int_floor=True), dict(f32_digits=True)):
        out = q.redq_pq(p, q_, nd, dev(torch, words), **kw)
        assert np.array_equal(host(out), orc.redq(p, q_, nd - 1, words))
        one = q.redq_pq(p, q_, nd, dev(torch, words[:1]), **kw)
        assert np.array_equal(host(one), orc.redq(p, q_, nd - 1, words[:1]))


def test_redq_pq_in_place(torch, orc):
    w = W.redq_words_q(4096, 5, 1176, salt=9)
    x = dev(torch, w)
    q.redq_pq(7, 1176, 5, x, out=x)
    assert np.array_equal(host(x), orc.redq(7, 1176, 4, w))
    x = dev(torch, w)
    q.redq_pq(7, 1176, 5, x, out=x, f32_digits=True)
    assert np.array_equal(host(x), orc.redq(7, 1176, 4, w))


def test_redq_pq_agrees_with_power_of_two_path(torch):
    """q = 2^10 is a multiple of p = 2: both REDQ entry points apply."""
    w = dev(torch, W.redq_words(10000, 5, 10, salt=2))
    a = q.redq_pq(2, 1024, 5, w)
    for mode in (0, 3):
        assert torch.equal(a, q.redq(2, 10, 5, w, table_mode=mode))


# --------------------------------------------------------------- pack ----

@pytest.mark.parametrize("pk", [(3, 3), (101, 2), (7, 4), (2, 8), (251, 2)])
def test_pack_log_formats(torch, orc, pk):
    p, k = pk
    f = q.Field(p, k)
    T = orc.antilog(p, f.poly)                       # oracle's own generator
    rows, cols = 37, 70
    L = W.log_matrix(rows, cols, f.order, salt=p)
    x = dev(torch, L)
    coeff = T[L.astype(np.int64)]                    # (rows, cols, k)
    got = host(f.pack(q.FMT_LOG, x, rows, cols, q.FMT_COEFF_U8))
    assert np.array_equal(got, np.transpose(coeff, (2, 0, 1)))
    cen = orc.centred(coeff, p)
    got = host(f.pack(q.FMT_LOG, x, rows, cols, q.FMT_OPERAND_A, ld_out=72,
                      out=torch.empty((k, rows, 72), dtype=torch.bfloat16, device="cuda")).float())
    assert np.array_equal(got[:, :, :cols], np.transpose(cen, (2, 0, 1)))
    got = host(f.pack(q.FMT_LOG, x, rows, cols, q.FMT_OPERAND_B, ld_out=40,
                      out=torch.empty((k, cols, 40), dtype=torch.bfloat16, device="cuda")).float())
    assert np.array_equal(got[:, :, :rows], np.transpose(cen, (2, 1, 0)))
    if f.n_q > 0:
        got = host(f.pack(q.FMT_LOG, x, rows, cols, q.FMT_QADIC_F64))
        assert np.array_equal(got.astype(np.int64), orc.qadic_value(coeff, 2 ** f.log2_q))


@pytest.mark.parametrize("pk", [(101, 2), (251, 2), (3, 3)])
def test_pack_plane_formats(torch, orc, pk):
    p, k = pk
    f = q.Field(p, k)
    rows, cols = 45, 66
    I8 = np.random.default_rng(p).integers(-128, 128, (k, rows, cols), dtype=np.int8)
    U8 = W.coeff_planes(k, rows, cols, p, salt=p)
    for fmt, X in ((q.FMT_INT8_PLANES, I8), (q.FMT_COEFF_U8, U8)):
        canon = np.transpose(X.astype(np.int64) % p, (1, 2, 0))   # (rows, cols, k)
        x = dev(torch, X)
        got = host(f.pack(fmt, x, rows, cols, q.FMT_QADIC_F64))
        assert np.array_equal(got.astype(np.int64), orc.qadic_value(canon, 2 ** f.log2_q))
        cen = orc.centred(canon, p)
        got = host(f.pack(fmt, x, rows, cols, q.FMT_OPERAND_A, ld_out=72,
                          out=torch.empty((k, rows, 72), dtype=torch.bfloat16, device="cuda")).float())
        assert np.array_equal(got[:, :, :cols], np.transpose(cen, (2, 0, 1)))
        got = host(f.pack(fmt, x, rows, cols, q.FMT_OPERAND_B, ld_out=48,
                          out=torch.empty((k, cols, 48), dtype=torch.bfloat16, device="cuda")).float())
        assert np.array_equal(got[:, :, :rows], np.transpose(cen, (2, 1, 0)))


# ----------------------------------------------------- GEMM helpers ----

def oracle_gemm_from_planes(orc, p, poly, Ap, Bp):
    """Ap: (k, m, K), Bp: (k, K, n) integer planes -> (k, m, n)."""
    C = orc.gemm(p, poly, np.transpose(Ap, (1, 2, 0)), np.transpose(Bp, (1, 2, 0)))
    return np.transpose(C, (2, 0, 1))


def run_fp64(torch, f, fmt, A, B, m, n, K):
    a = f.pack(fmt, dev(torch, A), m, K, q.FMT_QADIC_F64)
    b = f.pack(fmt, dev(torch, B), K, n, q.FMT_QADIC_F64)
    return host(f.gemm(q.PATH_FP64_QADIC, a, b, m, n, K))


def run_planes(torch, f, fmt, A, B, m, n, K):
    Kp = (K + 7) // 8 * 8
    a = torch.zeros((f.k, m, Kp), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros((f.k, n, Kp), dtype=torch.bfloat16, device="cuda")
    f.pack(fmt, dev(torch, A), m, K, q.FMT_OPERAND_A, out=a, ld_out=Kp)
    f.pack(fmt, dev(torch, B), K, n, q.FMT_OPERAND_B, out=b, ld_out=Kp)
    return host(f.gemm(q.PATH_PLANES, a, b, m, n, K, lda=Kp, ldb=Kp))


# ----------------------------------------------------------- FP64 GEMM ----

@pytest.mark.parametrize("shape", [(70, 45, 200), (64, 64, 85), (1, 1, 1), (130, 3, 171),
                                   (5, 129, 86)])
def test_gemm_fp64_gf27_log(torch, orc, shape):
    m, n, K = shape
    f = q.Field(3, 3)
    assert (f.log2_q, f.n_q) == (10, 85)
    T = orc.antilog(3, f.poly)
    A = W.log_matrix(m, K, 27, salt=m)
    B = W.log_matrix(K, n, 27, salt=n + 1)
    got = run_fp64(torch, f, q.FMT_LOG, A, B, m, n, K)
    want = orc.gemm(3, f.poly, T[A.astype(np.int64)], T[B.astype(np.int64)])
    assert np.array_equal(got, np.transpose(want, (2, 0, 1)))


def test_gemm_fp64_rejects_field_without_block(torch):
    """GF(7^4): the largest q with 7 log2 q <= 51 is 2^7 = 128 < k (p-1)^2 =
    144, so Eq. 2 admits no block: the FP64 form is refused, not run."""
    f = q.Field(7, 4)
    assert f.n_q == 0
    x = torch.zeros((4, 8, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QadicError) as e:
        f.pack(q.FMT_COEFF_U8, x, 8, 8, q.FMT_QADIC_F64)
    assert e.value.status == q.E_OVERFLOW


@pytest.mark.parametrize("pk,shape", [((101, 2), (67, 70, 333)), ((5, 3), (40, 33, 50)),
                                      ((31, 2), (33, 65, 257)), ((251, 2), (20, 20, 40))])
def test_gemm_fp64_planes_input(torch, orc, pk, shape):
    p, k = pk
    m, n, K = shape
    f = q.Field(p, k)
    h = (p - 1) // 2
    A = W.centred_planes(k, m, K, h, salt=1)
    B = W.centred_planes(k, K, n, h, salt=2)
    got = run_fp64(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


def test_gemm_fp64_all_max(torch, orc):
    """All coefficients p-1: every block sum sits at the Eq. 2 limit."""
    p, k = 101, 2
    f = q.Field(p, k)
    m, n, K = 16, 16, 6 * 7 + 5
    A = np.full((k, m, K), p - 1, np.uint8)
    B = np.full((k, K, n), p - 1, np.uint8)
    got = run_fp64(torch, f, q.FMT_COEFF_U8, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


# ------------------------------------------------ tensor-core plane GEMM ----

@pytest.mark.parametrize("shape", [(128, 128, 64), (293, 261, 209), (1, 1, 1), (128, 256, 8),
                                   (200, 129, 1000), (384, 384, 4096 + 64 * 3 + 5)])
def test_gemm_planes_gf101_2(torch, orc, shape):
    m, n, K = shape
    p, k = 101, 2
    f = q.Field(p, k)
    A = W.centred_planes(k, m, K, 50, salt=m)
    B = W.centred_planes(k, K, n, 50, salt=n)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("shape", [(130, 140, 2000), (128, 128, 512), (64, 300, 1537)])
def test_gemm_planes_gf251_2_drains(torch, orc, shape):
    """p = 251: the exact FP32 chunk is 536 -> 8 K-blocks, so K = 2000 crosses
    three in-place reductions."""
    m, n, K = shape
    p, k = 251, 2
    f = q.Field(p, k)
    A = W.centred_planes(k, m, K, 125, salt=K)
    B = W.centred_planes(k, K, n, 125, salt=K + 1)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


def test_gemm_planes_gf101_2_two_split_chunks(torch, orc):
    """k = 2 keeps one product per accumulator per K step, so the exact chunk
    for p = 101 is 6656; K = 13412 crosses two in-place reductions."""
    p, k = 101, 2
    f = q.Field(p, k)
    m, n, K = 128, 130, 2 * 6656 + 100
    A = W.centred_planes(k, m, K, 50, salt=77)
    B = W.centred_planes(k, K, n, 50, salt=78)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("p,val", [(251, 125), (251, -125), (101, 50), (101, -50)])
def test_gemm_planes_sums_at_the_fp32_limit(torch, orc, p, val):
    """All coefficients at +-h with the same sign: every accumulator grows by
    the maximum k h^2 per K step, reaching the 2^24 bound at each chunk end."""
    k = 2
    f = q.Field(p, k)
    m, n = 128, 128
    K = 3 * f.k_chunk_f32 // 64 * 64 + 64
    A = np.full((k, m, K), val, np.int8)
    B = np.full((k, K, n), val, np.int8)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    full = oracle_gemm_from_planes(orc, p, f.poly, A[:, :2, :], B[:, :, :2])
    assert np.array_equal(got[:, :2, :2], full)
    assert (got == got[:, :1, :1]).all()


@pytest.mark.parametrize("p,val", [(251, 125), (251, -125), (101, 50), (101, -50)])
@pytest.mark.parametrize("extra", [0, 1])
def test_gemm_planes_pair_sums_at_the_fp32_limit(torch, orc, p, val, extra):
    """k = 2, m > 128.  extra = 0: K is the longest with no in-place
    reduction (a whole number of exact chunks' worth of K-blocks), which runs
    on CTA pairs (one M = 256 MMA per A plane, the peer's rows in the peer's
    tensor memory); all coefficients at +-h with one sign, so each split
    accumulator ends at the 2^24 bound.  extra = 1: one K element more, which
    takes the one-CTA kernel with one in-place reduction.  Rows of both CTAs
    of a pair (0, 127 | 128, 255) and of a second pair are checked."""
    k = 2
    f = q.Field(p, k)
    h2 = ((p - 1) // 2) ** 2
    K = (2 ** 24 - 2 * p) // h2 // 64 * 64 + extra
    m, n = 384, 256
    A = np.full((k, m, K), val, np.int8)
    B = np.full((k, K, n), val, np.int8)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    rows = [0, 127, 128, 255, 256, 383]
    full = oracle_gemm_from_planes(orc, p, f.poly, A[:, :2, :], B[:, :, :2])
    for r in rows:
        assert np.array_equal(got[:, r, :2], full[:, 0, :]), r
    assert (got == got[:, :1, :1]).all()


@pytest.mark.parametrize("pk,shape", [((101, 2), (257, 130, 777)), ((251, 2), (512, 200, 2179)),
                                      ((101, 2), (1000, 72, 136)), ((31, 2), (300, 520, 64))])
def test_gemm_planes_pair_shapes(torch, orc, pk, shape):
    """k = 2 with m > 128 on ragged shapes: odd tile-row counts (the last
    pair's peer rows wholly outside A), ragged n and K; GF(251^2) with
    K = 2179 crosses exact chunks and takes the one-CTA kernel."""
    p, k = pk
    m, n, K = shape
    f = q.Field(p, k)
    h = (p - 1) // 2
    A = W.centred_planes(k, m, K, h, salt=m + 3)
    B = W.centred_planes(k, K, n, h, salt=n + 4)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("pk,shape", [((3, 3), (200, 130, 300)), ((7, 4), (129, 64, 256)),
                                      ((13, 3), (128, 192, 1000)), ((5, 4), (77, 65, 90)),
                                      ((31, 3), (128, 64, 64 * 390 + 20))])
def test_gemm_planes_k3_k4(torch, orc, pk, shape):
    """k = 3, 4: one MMA of N = k*64 per A plane into 2k-1 accumulators;
    GF(31^3) with K = 24980 crosses the exact FP32 chunk (24855)."""
    p, k = pk
    m, n, K = shape
    f = q.Field(p, k)
    h = (p - 1) // 2
    A = W.centred_planes(k, m, K, h, salt=m + 1)
    B = W.centred_planes(k, K, n, h, salt=n + 2)
    got = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_gemm_from_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("rows,cols", [(64, 128), (45, 128), (128, 64), (7, 192)])
def test_pack_aligned_fast_paths(torch, orc, rows, cols):
    for p in (101, 251, 3):
        k = 2 if p > 3 else 3
        f = q.Field(p, k)
        I8 = np.random.default_rng(rows + p).integers(-128, 128, (k, rows, cols), dtype=np.int8)
        U8 = np.random.default_rng(cols + p).integers(0, 256, (k, rows, cols), dtype=np.uint8)
        for fmt, X in ((q.FMT_INT8_PLANES, I8), (q.FMT_COEFF_U8, U8)):
            cen = orc.centred(np.transpose(X.astype(np.int64) % p, (1, 2, 0)), p)
            x = dev(torch, X)
            ldb = (rows + 7) // 8 * 8
            a = host(f.pack(fmt, x, rows, cols, q.FMT_OPERAND_A).float())
            assert np.array_equal(a, np.transpose(cen, (2, 0, 1)))
            b = host(f.pack(fmt, x, rows, cols, q.FMT_OPERAND_B, ld_out=ldb,
                            out=torch.zeros((k, cols, ldb), dtype=torch.bfloat16,
                                            device="cuda")).float())
            assert np.array_equal(b[:, :, :rows], np.transpose(cen, (2, 1, 0)))
            assert not b[:, :, rows:].any()


def test_gemm_planes_k0_gives_zero(torch):
    f = q.Field(101, 2)
    a = torch.zeros((2, 4, 8), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros((2, 4, 8), dtype=torch.bfloat16, device="cuda")
    C = torch.full((2, 4, 4), 7, dtype=torch.uint8, device="cuda")
    f.gemm(q.PATH_PLANES, a, b, 4, 4, 0, C=C, lda=8, ldb=8)
    assert not host(C).any()


def test_fp64_and_planes_agree_config3_slice(torch, orc):
    """The two contraction forms on the same inputs (GF(101^2))."""
    p, k = 101, 2
    f = q.Field(p, k)
    m, n, K = 256, 192, 1024
    A = W.centred_planes(k, m, K, 50, salt=5)
    B = W.centred_planes(k, K, n, 50, salt=6)
    g1 = run_planes(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    g2 = run_fp64(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(g1, g2)
    ii = np.arange(0, m, 17)
    jj = np.arange(0, n, 13)[: len(ii)]
    ii = ii[: len(jj)]
    want = orc.gemm_entries(p, f.poly, np.transpose(A, (1, 2, 0)), np.transpose(B, (1, 2, 0)),
                            ii, jj)
    assert np.array_equal(g1[:, ii, jj].T, want)


@pytest.mark.parametrize("path,shape", [(q.PATH_PLANES, (640, 200, 136)),
                                        (q.PATH_PLANES, (300, 96, 64)),
                                        (q.PATH_FP64_QADIC, (130, 70, 45))])
def test_matmul_host_end_to_end(torch, orc, path, shape):
    """qadic_matmul_host from pinned host buffers (copies overlapped with the
    pack, the plane GEMM in two row blocks when m >= 512) against the oracle."""
    m, n, K = shape
    p, k = 101, 2
    f = q.Field(p, k)
    A = W.centred_planes(k, m, K, 50, salt=31)
    B = W.centred_planes(k, K, n, 50, salt=32)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.full((k, m, n), 255, dtype=torch.uint8).pin_memory()
    ws = torch.empty(f.matmul_workspace_size(path, q.FMT_INT8_PLANES, m, n, K), dtype=torch.uint8,
                     device="cuda")
    for _ in range(2):
        hC.fill_(255)
        f.matmul_host(path, q.FMT_INT8_PLANES, hA, hB, hC, m, n, K, ws)
        torch.cuda.synchronize()
        assert np.array_equal(hC.numpy(), oracle_gemm_from_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("pk,shape", [((101, 2), (1100, 130, 72)), ((3, 3), (768, 64, 40)),
                                      ((7, 4), (520, 33, 16))])
def test_matmul_host_log_codes_split(torch, orc, pk, shape):
    """Log-coded host inputs (2-byte codes for GF(101^2), 1-byte otherwise)
    through the two-block host pipeline: B first, A in two row blocks."""
    p, k = pk
    m, n, K = shape
    f = q.Field(p, k)
    LA = W.log_matrix(m, K, f.order, salt=41)
    LB = W.log_matrix(K, n, f.order, salt=42)
    hA = torch.from_numpy(LA).pin_memory()
    hB = torch.from_numpy(LB).pin_memory()
    hC = torch.full((k, m, n), 255, dtype=torch.uint8).pin_memory()
    ws = torch.empty(f.matmul_workspace_size(q.PATH_PLANES, q.FMT_LOG, m, n, K),
                     dtype=torch.uint8, device="cuda")
    f.matmul_host(q.PATH_PLANES, q.FMT_LOG, hA, hB, hC, m, n, K, ws)
    torch.cuda.synchronize()
    T = orc.antilog(p, f.poly)
    want = orc.gemm(p, f.poly, T[LA.astype(np.int64)], T[LB.astype(np.int64)])
    assert np.array_equal(np.transpose(hC.numpy(), (1, 2, 0)), want)


def test_matmul_host_blocks(torch, orc):
    """m = 2048, n = 4096: the host pipeline cuts B into four column blocks
    and A into row blocks (each block GEMM one round of 256 x 128 output
    units on the SM pairs), C going back block by block on its own stream;
    rows of every block against the oracle, and the whole result against the
    device path."""
    p, k, m, n, K = 101, 2, 2048, 4096, 64
    f = q.Field(p, k)
    A = W.centred_planes(k, m, K, 50, salt=71)
    B = W.centred_planes(k, K, n, 50, salt=72)
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    hC = torch.full((k, m, n), 255, dtype=torch.uint8).pin_memory()
    ws = torch.empty(f.matmul_workspace_size(q.PATH_PLANES, q.FMT_INT8_PLANES, m, n, K),
                     dtype=torch.uint8, device="cuda")
    f.matmul_host(q.PATH_PLANES, q.FMT_INT8_PLANES, hA, hB, hC, m, n, K, ws)
    torch.cuda.synchronize()
    a = f.pack(q.FMT_INT8_PLANES, dev(torch, A), m, K, q.FMT_OPERAND_A)
    b = f.pack(q.FMT_INT8_PLANES, dev(torch, B), K, n, q.FMT_OPERAND_B)
    C = f.gemm(q.PATH_PLANES, a, b, m, n, K).cpu().numpy()
    assert np.array_equal(hC.numpy(), C)
    rows = np.array([0, 511, 512, 1023, 1024, 1535, 1536, 2047])
    want = orc.gemm(p, f.poly, np.transpose(A[:, rows], (1, 2, 0)), np.transpose(B, (1, 2, 0)))
    assert np.array_equal(np.transpose(C[:, rows], (1, 2, 0)), want)


@pytest.mark.parametrize("fmt", [q.FMT_INT8_PLANES, q.FMT_COEFF_U8, q.FMT_LOG])
@pytest.mark.parametrize("shape", [(1100, 1024, 72), (520, 1536, 40), (2304, 2048, 16)])
def test_matmul_host_column_blocks(torch, orc, fmt, shape):
    """n a multiple of 512 (>= 1024) and m >= 512: B crosses the link in four
    column blocks and A in row blocks (ragged last block), one GEMM per
    block pair, C back in 2-D block copies, twice in a row on the same
    workspace; the whole result against the device path, sampled rows of
    every row block against the oracle."""
    m, n, K = shape
    p, k = 101, 2
    f = q.Field(p, k)
    if fmt == q.FMT_LOG:
        A, B = W.log_matrix(m, K, f.order, salt=81), W.log_matrix(K, n, f.order, salt=82)
    elif fmt == q.FMT_INT8_PLANES:
        A, B = W.centred_planes(k, m, K, 50, salt=81), W.centred_planes(k, K, n, 50, salt=82)
    else:
        A, B = W.coeff_planes(k, m, K, p, salt=81), W.coeff_planes(k, K, n, p, salt=82)
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    hC = torch.full((k, m, n), 255, dtype=torch.uint8).pin_memory()
    ws = torch.empty(f.matmul_workspace_size(q.PATH_PLANES, fmt, m, n, K), dtype=torch.uint8,
                     device="cuda")
    a = f.pack(fmt, dev(torch, A), m, K, q.FMT_OPERAND_A)
    b = f.pack(fmt, dev(torch, B), K, n, q.FMT_OPERAND_B)
    C = f.gemm(q.PATH_PLANES, a, b, m, n, K).cpu().numpy()
    for _ in range(2):
        hC.fill_(255)
        f.matmul_host(q.PATH_PLANES, fmt, hA, hB, hC, m, n, K, ws)
        torch.cuda.synchronize()
        q.sync_status()
        assert np.array_equal(hC.numpy(), C)
    rows = np.unique(np.clip(np.array([0, 255, 256, 511, 512, 1023, 1024, m // 2, m - 1]), 0, m - 1))
    if fmt == q.FMT_LOG:
        T = orc.antilog(p, f.poly)
        want = orc.gemm(p, f.poly, T[A[rows].astype(np.int64)], T[B.astype(np.int64)])
    else:
        want = orc.gemm(p, f.poly, np.transpose(A[:, rows].astype(np.int64) % p, (1, 2, 0)),
                        np.transpose(B.astype(np.int64) % p, (1, 2, 0)))
    assert np.array_equal(np.transpose(C[:, rows], (1, 2, 0)), want)


def test_bounded_wait_timeout_is_reported_and_context_survives(torch, orc):
    """A bounded wait that runs out (nothing arrives on its barrier) records
    QADIC_E_DEVICE_TIMEOUT; sync_status reports it once, clears it, and the
    context keeps computing correctly."""
    q.sync_status()
    q.selftest_bounded_wait(4096)
    with pytest.raises(q.QadicError) as e:
        q.sync_status()
    assert e.value.status == q.E_DEVICE_TIMEOUT
    assert b"site 9" in q.lib().qadic_last_error()
    q.sync_status()   # cleared
    a, b = W.polymul_pairs(1000, 7, 4, salt=5)
    out = q.polymul_batched(7, 4, dev(torch, a), dev(torch, b))
    assert np.array_equal(host(out), orc.polymul(7, a, b))
    q.sync_status()


def test_sync_status_clean(torch):
    q.sync_status()


# ------------------------------------------------------- fold-before form ----

def fold_operands(torch, f, A, B, m, n, K):
    """Coefficient planes (k, m, K) and (k, K, n) -> OPERAND_A, OPERAND_B_FOLD."""
    lda = (K + 7) // 8 * 8
    a = f.pack(q.FMT_COEFF_U8, dev(torch, A), m, K, q.FMT_OPERAND_A,
               out=torch.zeros((f.k, m, lda), dtype=torch.bfloat16, device="cuda"), ld_out=lda)
    b = f.pack(q.FMT_COEFF_U8, dev(torch, B), K, n, q.FMT_OPERAND_B_FOLD)
    return a, b, lda


@pytest.mark.parametrize("pk", [(101, 1), (31, 2), (101, 2), (3, 3), (7, 4), (5, 5), (2, 6), (3, 7),
                                (2, 8)])
@pytest.mark.parametrize("shape", [(130, 70, 45), (300, 257, 200), (128, 512, 64), (1, 1, 1)])
def test_fold_path_against_oracle(torch, orc, pk, shape):
    p, k = pk
    m, n, K = shape
    f = q.Field(p, k)
    rng = np.random.default_rng(p * 31 + k + m)
    A = rng.integers(0, p, (k, m, K), dtype=np.uint8)
    B = rng.integers(0, p, (k, K, n), dtype=np.uint8)
    a, b, lda = fold_operands(torch, f, A, B, m, n, K)
    C = f.gemm(q.PATH_FOLD, a, b, m, n, K, lda=lda).cpu().numpy()
    want = orc.gemm(p, f.poly, np.transpose(A, (1, 2, 0)), np.transpose(B, (1, 2, 0)))
    assert np.array_equal(np.transpose(C, (1, 2, 0)), want)


def test_fold_operand_is_the_multiplication_matrix(torch, orc):
    """Plane i, block j of OPERAND_B_FOLD = coefficient j of b X^i mod P
    (centred), checked element by element with the oracle's field product;
    padding rows are zero."""
    for p, k in [(7, 4), (3, 3), (2, 8)]:
        f = q.Field(p, k)
        K, n = 19, 37
        B = np.random.default_rng(p).integers(0, p, (k, K, n), dtype=np.uint8)
        out = f.pack(q.FMT_COEFF_U8, dev(torch, B), K, n, q.FMT_OPERAND_B_FOLD).float().cpu().numpy()
        n_pad = q.fold_n_pad(n)
        assert out.shape == (k, k * n_pad, 24)
        for i in range(k):
            xi = [0] * k
            if i < k:
                xi[i] = 1
            for r in range(0, K, 5):
                for c in range(0, n, 3):
                    prod = orc.field_mul(p, f.poly, [int(B[l, r, c]) for l in range(k)], xi)
                    for j in range(k):
                        assert int(out[i, j * n_pad + c, r]) % p == prod[j], (p, k, i, j, r, c)
                        assert abs(int(out[i, j * n_pad + c, r])) <= max(1, (p - 1) // 2)
            assert not out[i, :, :K].reshape(k, n_pad, K)[:, n:, :].any()


def test_fold_equals_plane_path(torch):
    for pk, (m, n, K) in [((101, 2), (640, 384, 512)), ((13, 3), (256, 200, 300)),
                          ((7, 4), (300, 128, 640))]:
        f = q.Field(*pk)
        rng = np.random.default_rng(pk[0])
        A = rng.integers(0, pk[0], (f.k, m, K), dtype=np.uint8)
        B = rng.integers(0, pk[0], (f.k, K, n), dtype=np.uint8)
        a, b, lda = fold_operands(torch, f, A, B, m, n, K)
        C1 = f.gemm(q.PATH_FOLD, a, b, m, n, K, lda=lda)
        bp = f.pack(q.FMT_COEFF_U8, dev(torch, B), K, n, q.FMT_OPERAND_B,
                    out=torch.zeros((f.k, n, lda), dtype=torch.bfloat16, device="cuda"), ld_out=lda)
        C2 = f.gemm(q.PATH_PLANES, a, bp, m, n, K, lda=lda, ldb=lda)
        assert torch.equal(C1, C2), pk


def test_fold_exact_chunks_p251(torch, orc):
    """GF(251^2), all coefficients -125, K = 2000: every accumulator crosses
    one in-place reduction (exact chunk 1073 -> 16 K-blocks)."""
    f = q.Field(251, 2)
    m, n, K = 256, 300, 2000
    A = np.full((2, m, K), 126, np.uint8)
    B = np.full((2, K, n), 126, np.uint8)
    B[1, ::3, ::5] = 7
    a, b, lda = fold_operands(torch, f, A, B, m, n, K)
    C = f.gemm(q.PATH_FOLD, a, b, m, n, K, lda=lda).cpu().numpy()
    rows = np.array([0, 1, 100, 255])
    want = orc.gemm(251, f.poly, np.transpose(A[:, rows], (1, 2, 0)), np.transpose(B, (1, 2, 0)))
    assert np.array_equal(np.transpose(C[:, rows], (1, 2, 0)), want)


# ------------------------------------------------------- Karatsuba (k = 2) ----

def kara_operands(torch, f, A, B, m, n, K):
    ld = (K + 7) // 8 * 8
    a = f.pack(q.FMT_COEFF_U8, dev(torch, A), m, K, q.FMT_OPERAND_A_KARA,
               out=torch.zeros((3, m, ld), dtype=torch.bfloat16, device="cuda"), ld_out=ld)
    b = f.pack(q.FMT_COEFF_U8, dev(torch, B), K, n, q.FMT_OPERAND_B_KARA,
               out=torch.zeros((3, n, ld), dtype=torch.bfloat16, device="cuda"), ld_out=ld)
    return a, b, ld


@pytest.mark.parametrize("p", [2, 3, 31, 101, 251])
@pytest.mark.parametrize("shape", [(130, 70, 45), (300, 257, 200), (128, 512, 64), (1, 1, 1),
                                   (256, 128, 3000)])
def test_karatsuba_against_oracle(torch, orc, p, shape):
    m, n, K = shape
    f = q.Field(p, 2)
    rng = np.random.default_rng(p + m + K)
    A = rng.integers(0, p, (2, m, K), dtype=np.uint8)
    B = rng.integers(0, p, (2, K, n), dtype=np.uint8)
    a, b, ld = kara_operands(torch, f, A, B, m, n, K)
    C = f.gemm(q.PATH_KARATSUBA, a, b, m, n, K, lda=ld, ldb=ld).cpu().numpy()
    if m * n * K > 4e7:
        rows = np.arange(0, m, 17)
        want = orc.gemm(p, f.poly, np.transpose(A[:, rows], (1, 2, 0)), np.transpose(B, (1, 2, 0)))
        assert np.array_equal(np.transpose(C[:, rows], (1, 2, 0)), want)
    else:
        want = orc.gemm(p, f.poly, np.transpose(A, (1, 2, 0)), np.transpose(B, (1, 2, 0)))
        assert np.array_equal(np.transpose(C, (1, 2, 0)), want)


def test_karatsuba_operand_planes(torch, orc):
    f = q.Field(101, 2)
    A = np.random.default_rng(1).integers(0, 101, (2, 37, 29), dtype=np.uint8)
    a = f.pack(q.FMT_COEFF_U8, dev(torch, A), 37, 29, q.FMT_OPERAND_A_KARA,
               out=torch.zeros((3, 37, 32), dtype=torch.bfloat16, device="cuda"), ld_out=32)
    b = f.pack(q.FMT_COEFF_U8, dev(torch, A), 37, 29, q.FMT_OPERAND_B_KARA,
               out=torch.zeros((3, 29, 40), dtype=torch.bfloat16, device="cuda"), ld_out=40)
    want = np.stack([orc.centred(A[0], 101), orc.centred(A[1], 101),
                     orc.centred(A[0].astype(int) + A[1], 101)])
    assert np.array_equal(a.float().cpu().numpy()[:, :, :29], want)
    assert np.array_equal(b.float().cpu().numpy()[:, :, :37], np.transpose(want, (0, 2, 1)))


def test_karatsuba_equals_plane_path_and_worst_case(torch, orc):
    f = q.Field(251, 2)
    m, n, K = 384, 256, 2048
    rng = np.random.default_rng(7)
    A = rng.choice(np.array([0, 126, 125], np.uint8), (2, m, K))   # centred 0, -125, 125
    B = rng.choice(np.array([0, 126, 125], np.uint8), (2, K, n))
    A[:, :64] = 126                      # rows with every D_0, D_2 product at the bound
    B[:, :, :64] = 126
    a, b, ld = kara_operands(torch, f, A, B, m, n, K)
    C1 = f.gemm(q.PATH_KARATSUBA, a, b, m, n, K, lda=ld, ldb=ld)
    ap = f.pack(q.FMT_COEFF_U8, dev(torch, A), m, K, q.FMT_OPERAND_A)
    bp = f.pack(q.FMT_COEFF_U8, dev(torch, B), K, n, q.FMT_OPERAND_B)
    C2 = f.gemm(q.PATH_PLANES, ap, bp, m, n, K)
    assert torch.equal(C1, C2)
    rows = np.array([0, 63, 64, 383])
    want = orc.gemm(251, f.poly, np.transpose(A[:, rows], (1, 2, 0)), np.transpose(B, (1, 2, 0)))
    assert np.array_equal(np.transpose(C1.cpu().numpy()[:, rows], (1, 2, 0)), want)


def test_karatsuba_rejects_other_k(torch):
    f = q.Field(7, 3)
    x = torch.zeros((3, 16, 16), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(q.QadicError) as e:
        f.gemm(q.PATH_KARATSUBA, x, x, 16, 16, 16)
    assert e.value.status == q.E_UNSUPPORTED


# ------------------------------------------- pack_operands / qadic_matmul ----

@pytest.mark.parametrize("fmt", [q.FMT_INT8_PLANES, q.FMT_COEFF_U8, q.FMT_LOG])
@pytest.mark.parametrize("shape", [(320, 256, 192), (130, 40, 70), (64, 4096, 128)])
def test_pack_operands_equals_two_packs(torch, fmt, shape):
    m, K, n = shape
    f = q.Field(101, 2)
    if fmt == q.FMT_LOG:
        A, B = W.log_matrix(m, K, f.order, salt=51), W.log_matrix(K, n, f.order, salt=52)
    elif fmt == q.FMT_INT8_PLANES:
        A, B = W.centred_planes(2, m, K, 50, salt=51), W.centred_planes(2, K, n, 50, salt=52)
    else:
        A, B = W.coeff_planes(2, m, K, 101, salt=51), W.coeff_planes(2, K, n, 101, salt=52)
    ld = (K + 7) // 8 * 8
    oa = torch.zeros((2, m, ld), dtype=torch.bfloat16, device="cuda")
    ob = torch.zeros((2, n, ld), dtype=torch.bfloat16, device="cuda")
    f.pack_operands(fmt, dev(torch, A), dev(torch, B), m, n, K, oa, ob)
    ra = f.pack(fmt, dev(torch, A), m, K, q.FMT_OPERAND_A,
                out=torch.zeros((2, m, ld), dtype=torch.bfloat16, device="cuda"), ld_out=ld)
    rb = f.pack(fmt, dev(torch, B), K, n, q.FMT_OPERAND_B,
                out=torch.zeros((2, n, ld), dtype=torch.bfloat16, device="cuda"), ld_out=ld)
    assert torch.equal(oa, ra) and torch.equal(ob, rb)


@pytest.mark.parametrize("pk", [(101, 2), (7, 4), (2, 8), (3, 3), (251, 2)])
@pytest.mark.parametrize("fmt", [q.FMT_INT8_PLANES, q.FMT_COEFF_U8])
@pytest.mark.parametrize("shape", [(100, 48, 128), (1, 16, 64), (257, 80, 192), (64, 64, 64),
                                   (65, 4096, 64), (130, 144, 128), (130, 40, 70)])
def test_pack_operands_ragged(torch, pk, fmt, shape):
    """The fused launch (K a multiple of 16, n of 64): B tiles stacked two
    deep down K, cut by the edge of K, ragged m for A, full-range int8 and
    uint8 bytes (reduced mod p on the way), against the two single-operand
    packs; the last shape takes two launches."""
    p, k = pk
    m, K, n = shape
    f = q.Field(p, k)
    rng = np.random.default_rng(p * 1000 + m + K + n)
    if fmt == q.FMT_INT8_PLANES:
        A = rng.integers(-128, 128, (k, m, K), dtype=np.int8)
        B = rng.integers(-128, 128, (k, K, n), dtype=np.int8)
    else:
        A = rng.integers(0, 256, (k, m, K), dtype=np.uint8)
        B = rng.integers(0, 256, (k, K, n), dtype=np.uint8)
    ld = (K + 7) // 8 * 8
    oa = torch.full((k, m, ld), 7.0, dtype=torch.bfloat16, device="cuda")
    ob = torch.full((k, n, ld), 7.0, dtype=torch.bfloat16, device="cuda")
    f.pack_operands(fmt, dev(torch, A), dev(torch, B), m, n, K, oa, ob)
    ra = f.pack(fmt, dev(torch, A), m, K, q.FMT_OPERAND_A,
                out=torch.full((k, m, ld), 7.0, dtype=torch.bfloat16, device="cuda"), ld_out=ld)
    rb = f.pack(fmt, dev(torch, B), K, n, q.FMT_OPERAND_B,
                out=torch.full((k, n, ld), 7.0, dtype=torch.bfloat16, device="cuda"), ld_out=ld)
    torch.cuda.synchronize()
    q.sync_status()
    assert torch.equal(oa[:, :, :K], ra[:, :, :K]) and torch.equal(ob[:, :, :K], rb[:, :, :K])
    # nothing written past K in the padded rows
    assert bool((oa[:, :, K:] == 7.0).all()) and bool((ob[:, :, K:] == 7.0).all())


@pytest.mark.parametrize("path", [q.PATH_PLANES, q.PATH_FP64_QADIC, q.PATH_FOLD,
                                  q.PATH_KARATSUBA])
@pytest.mark.parametrize("fmt", [q.FMT_INT8_PLANES, q.FMT_LOG])
@pytest.mark.parametrize("shape", [(200, 130, 72), (256, 192, 64), (33, 65, 7)])
def test_matmul_device_all_paths(torch, orc, path, fmt, shape):
    m, n, K = shape
    p, k = 101, 2
    f = q.Field(p, k)
    if fmt == q.FMT_LOG:
        LA, LB = W.log_matrix(m, K, f.order, salt=61), W.log_matrix(K, n, f.order, salt=62)
        T = orc.antilog(p, f.poly)
        want = orc.gemm(p, f.poly, T[LA.astype(np.int64)], T[LB.astype(np.int64)])
        dA, dB = dev(torch, LA), dev(torch, LB)
    else:
        A, B = W.centred_planes(k, m, K, 50, salt=61), W.centred_planes(k, K, n, 50, salt=62)
        want = orc.gemm(p, f.poly, np.transpose(A, (1, 2, 0)), np.transpose(B, (1, 2, 0)))
        dA, dB = dev(torch, A), dev(torch, B)
    ws = torch.empty(f.matmul_device_workspace_size(path, m, n, K) + 256, dtype=torch.uint8,
                     device="cuda")
    C = f.matmul(path, fmt, dA, dB, m, n, K, ws)
    assert np.array_equal(np.transpose(C.cpu().numpy(), (1, 2, 0)), want)


def test_matmul_device_empty_k_and_short_workspace(torch):
    f = q.Field(31, 2)
    x = torch.zeros(64, dtype=torch.int8, device="cuda")
    ws = torch.empty(f.matmul_device_workspace_size(q.PATH_PLANES, 4, 4, 0) + 256,
                     dtype=torch.uint8, device="cuda")
    C = torch.full((2, 4, 4), 7, dtype=torch.uint8, device="cuda")
    f.matmul(q.PATH_PLANES, q.FMT_INT8_PLANES, x, x, 4, 4, 0, ws, C=C)
    assert not C.any()
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QadicError) as e:
        f.matmul(q.PATH_PLANES, q.FMT_INT8_PLANES, x, x, 4, 4, 8, small)
    assert e.value.status == q.E_NOMEM
