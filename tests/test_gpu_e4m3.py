"""GPU parity of the plane path on fp8 e4m3 operands (QADIC_PATH_PLANES_E4M3,
p <= 31): the pack to e4m3 codes against the bf16 pack, and the tcgen05
kind::f8f6f4 plane GEMM against the oracle, bit-exact, on ragged shapes,
across exact-FP32-chunk reductions and with every partial sum at its bound."""
import numpy as np
import pytest

import paper_0710_0510_gb300 as q
from paper_0710_0510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle_planes(orc, p, poly, A, B):
    """A: (k, m, K), B: (k, K, n) integer planes -> (k, m, n)."""
    C = orc.gemm(p, poly, np.transpose(A, (1, 2, 0)), np.transpose(B, (1, 2, 0)))
    return np.transpose(C, (2, 0, 1))


def run_e4m3(torch, f, fmt, A, B, m, n, K):
    Kp = (K + 15) // 16 * 16
    a = torch.zeros((f.k, m, Kp), dtype=torch.uint8, device="cuda")
    b = torch.zeros((f.k, n, Kp), dtype=torch.uint8, device="cuda")
    f.pack(fmt, dev(torch, A), m, K, q.FMT_OPERAND_A_E4M3, out=a, ld_out=Kp)
    f.pack(fmt, dev(torch, B), K, n, q.FMT_OPERAND_B_E4M3, out=b, ld_out=Kp)
    C = f.gemm(q.PATH_PLANES_E4M3, a, b, m, n, K, lda=Kp, ldb=Kp)
    torch.cuda.synchronize()
    q.sync_status()
    return C.cpu().numpy()


@pytest.mark.parametrize("pk", [(31, 2), (7, 4), (2, 3), (3, 3), (13, 2)])
@pytest.mark.parametrize("fmt", [q.FMT_INT8_PLANES, q.FMT_COEFF_U8, q.FMT_LOG])
@pytest.mark.parametrize("rows,cols", [(64, 128), (45, 96), (130, 64), (7, 40)])
def test_pack_e4m3_equals_bf16_values(torch, pk, fmt, rows, cols):
    """The e4m3 codes decode to the same small integers as the bf16 operands,
    on the vectorised paths (16-byte rows) and the generic ones."""
    p, k = pk
    f = q.Field(p, k)
    rng = np.random.default_rng(p * 100 + rows + cols)
    if fmt == q.FMT_LOG:
        X = W.log_matrix(rows, cols, f.order, salt=rows)
    elif fmt == q.FMT_INT8_PLANES:
        X = rng.integers(-128, 128, (k, rows, cols), dtype=np.int8)
    else:
        X = rng.integers(0, 256, (k, rows, cols), dtype=np.uint8)
    x = dev(torch, X)
    for o8, o16, r_, c_ in ((q.FMT_OPERAND_A_E4M3, q.FMT_OPERAND_A, rows, cols),
                            (q.FMT_OPERAND_B_E4M3, q.FMT_OPERAND_B, cols, rows)):
        ld = (c_ + 15) // 16 * 16
        r8 = torch.full((k, r_, ld), 0x7F, dtype=torch.uint8, device="cuda")
        r16 = torch.zeros((k, r_, ld), dtype=torch.bfloat16, device="cuda")
        f.pack(fmt, x, rows, cols, o8, out=r8, ld_out=ld)
        f.pack(fmt, x, rows, cols, o16, out=r16, ld_out=ld)
        torch.cuda.synchronize()
        q.sync_status()
        got = r8[:, :, :c_].contiguous().view(torch.float8_e4m3fn).float()
        assert torch.equal(got, r16[:, :, :c_].float()), (o8, fmt)
        assert (r8[:, :, c_:] == 0x7F).all()   # the padding is left alone


def test_pack_e4m3_refused_above_p31(torch):
    f = q.Field(37, 2)
    x = torch.zeros((2, 16, 16), dtype=torch.int8, device="cuda")
    with pytest.raises(q.QadicError) as e:
        f.pack(q.FMT_INT8_PLANES, x, 16, 16, q.FMT_OPERAND_A_E4M3)
    assert e.value.status == q.E_UNSUPPORTED


@pytest.mark.parametrize("pk,shape", [((31, 2), (300, 520, 64)), ((31, 2), (128, 130, 1000)),
                                      ((31, 2), (513, 256, 4096)), ((7, 4), (129, 64, 256)),
                                      ((3, 3), (200, 130, 300)), ((2, 4), (77, 65, 90)),
                                      ((13, 3), (257, 192, 1000)), ((5, 2), (1, 1, 1))])
def test_gemm_planes_e4m3(torch, orc, pk, shape):
    """k = 2 with m > 128 on CTA pairs, k = 2 with one tile row and k = 3, 4
    on one CTA per tile; ragged m, n and K (K-blocks of 128 elements)."""
    p, k = pk
    m, n, K = shape
    f = q.Field(p, k)
    h = max((p - 1) // 2, 1)
    A = W.centred_planes(k, m, K, h, salt=m + 5)
    B = W.centred_planes(k, K, n, h, salt=n + 6)
    if p == 2:
        A, B = A % 2, B % 2
    got = run_e4m3(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_planes(orc, p, f.poly, A, B))


def test_gemm_planes_e4m3_crosses_chunks(torch, orc):
    """GF(31^3): shared accumulators, exact chunk (2^24 - 62) / (3 * 15^2) =
    24855 elements, i.e. 194 K-blocks of 128; K = 50000 crosses two in-place
    reductions."""
    p, k = 31, 3
    f = q.Field(p, k)
    m, n, K = 128, 64, 50000
    A = W.centred_planes(k, m, K, 15, salt=91)
    B = W.centred_planes(k, K, n, 15, salt=92)
    got = run_e4m3(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    assert np.array_equal(got, oracle_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("val", [15, -15])
@pytest.mark.parametrize("k,m,extra", [(2, 384, 0), (2, 384, 1), (3, 128, 0)])
def test_gemm_planes_e4m3_sums_at_the_fp32_limit(torch, orc, val, k, m, extra):
    """p = 31, all coefficients at +-15 with one sign: every accumulator grows
    by the largest amount per K step.  k = 2: K the longest with no in-place
    reduction (CTA pairs; each split accumulator ends at the 2^24 bound), and
    one K-block more (one CTA per tile, one reduction).  k = 3: K of three
    exact chunks (two reductions, each at the bound)."""
    p = 31
    f = q.Field(p, k)
    h2 = 15 * 15
    if k == 2:
        K = (2 ** 24 - 2 * p) // h2 // 128 * 128 + 128 * extra
    else:
        K = 3 * f.k_chunk_f32 // 128 * 128
    n = 256
    A = np.full((k, m, K), val, np.int8)
    B = np.full((k, K, n), val, np.int8)
    got = run_e4m3(torch, f, q.FMT_INT8_PLANES, A, B, m, n, K)
    full = oracle_planes(orc, p, f.poly, A[:, :2, :], B[:, :, :2])
    assert np.array_equal(got[:, :2, :2], full)
    assert (got == got[:, :1, :1]).all()


@pytest.mark.parametrize("fmt", [q.FMT_LOG, q.FMT_COEFF_U8, q.FMT_INT8_PLANES])
def test_matmul_device_e4m3_equals_bf16_path(torch, fmt):
    """qadic_matmul with QADIC_PATH_PLANES_E4M3 (pack to e4m3 + GEMM) gives the
    bf16 plane path's result, twice on the same workspace."""
    p, k, m, n, K = 31, 2, 300, 200, 333
    f = q.Field(p, k)
    if fmt == q.FMT_LOG:
        A, B = W.log_matrix(m, K, f.order, salt=3), W.log_matrix(K, n, f.order, salt=4)
    elif fmt == q.FMT_COEFF_U8:
        A, B = W.coeff_planes(k, m, K, p, salt=3), W.coeff_planes(k, K, n, p, salt=4)
    else:
        A, B = W.centred_planes(k, m, K, 15, salt=3), W.centred_planes(k, K, n, 15, salt=4)
    dA, dB = dev(torch, A), dev(torch, B)
    want = None
    for path in (q.PATH_PLANES, q.PATH_PLANES_E4M3):
        ws = torch.empty(max(int(q.lib().qadic_matmul_device_workspace_size(f.handle, path, m, n, K)), 256),
                         dtype=torch.uint8, device="cuda")
        for _ in range(2):
            C = f.matmul(path, fmt, dA, dB, m, n, K, ws)
            torch.cuda.synchronize()
            q.sync_status()
            if want is None:
                want = C.clone()
            assert torch.equal(C, want), path


def test_gemm_e4m3_refuses_misaligned_and_large_p(torch):
    f = q.Field(31, 2)
    a = torch.zeros((2, 64, 24), dtype=torch.uint8, device="cuda")   # ld 24: not a multiple of 16
    with pytest.raises(q.QadicError) as e:
        f.gemm(q.PATH_PLANES_E4M3, a, a, 64, 64, 24, lda=24, ldb=24)
    assert e.value.status == q.E_INVALID
    g = q.Field(101, 2)
    b = torch.zeros((2, 64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QadicError) as e:
        g.gemm(q.PATH_PLANES_E4M3, b, b, 64, 64, 64)
    assert e.value.status == q.E_UNSUPPORTED


@pytest.mark.parametrize("path", [q.PATH_PLANES, q.PATH_PLANES_E4M3])
def test_chained_packs_and_gemms_share_operand_buffers(torch, path):
    """Packs and GEMMs launched back to back on one stream with no host
    synchronisation, two input sets alternating through the same operand
    buffers: each launch may begin while the previous one finishes
    (programmatic dependent launch), so a pack that overwrote operands still
    being read, or a GEMM that read operands not yet written, would change
    some product.  Every product equals the one computed in isolation."""
    p, k, n = 31, 2, 2048
    f = q.Field(p, k)
    X = [(dev(torch, W.centred_planes(k, n, n, 15, salt=40 + 2 * i)),
          dev(torch, W.centred_planes(k, n, n, 15, salt=41 + 2 * i))) for i in range(2)]
    e4 = path == q.PATH_PLANES_E4M3
    dt = torch.uint8 if e4 else torch.bfloat16
    opA = torch.empty((k, n, n), dtype=dt, device="cuda")
    opB = torch.empty((k, n, n), dtype=dt, device="cuda")

    def product(i, C):
        a, b = X[i]
        f.pack_operands(q.FMT_INT8_PLANES, a, b, n, n, n, opA, opB, e4m3=e4)
        return f.gemm(path, opA, opB, n, n, n, C=C)

    want = []
    for i in range(2):
        want.append(product(i, torch.empty((k, n, n), dtype=torch.uint8, device="cuda")))
        torch.cuda.synchronize()
    assert not torch.equal(want[0], want[1])
    outs = [torch.empty((k, n, n), dtype=torch.uint8, device="cuda") for _ in range(12)]
    for j, C in enumerate(outs):
        product(j % 2, C)
    torch.cuda.synchronize()
    q.sync_status()
    for j, C in enumerate(outs):
        assert torch.equal(C, want[j % 2]), j


def test_matmul_device_e4m3_strided_inputs(torch, orc):
    """qadic_matmul on e4m3 with input rows longer than the widths (odd
    strides, each plane rows x ld elements) against the oracle."""
    p, k, m, n, K = 31, 2, 200, 150, 270
    f = q.Field(p, k)
    lda, ldb = K + 5, n + 3
    A = W.centred_planes(k, m, K, 15, salt=61)
    B = W.centred_planes(k, K, n, 15, salt=62)
    Ap = np.full((k, m, lda), 99, np.int8)
    Bp = np.full((k, K, ldb), -99, np.int8)
    Ap[:, :, :K] = A
    Bp[:, :, :n] = B
    ws = torch.empty(max(f.matmul_device_workspace_size(q.PATH_PLANES_E4M3, m, n, K), 256),
                     dtype=torch.uint8, device="cuda")
    C = f.matmul(q.PATH_PLANES_E4M3, q.FMT_INT8_PLANES, dev(torch, Ap), dev(torch, Bp), m, n, K, ws,
                 lda=lda, ldb=ldb)
    torch.cuda.synchronize()
    q.sync_status()
    assert np.array_equal(C.cpu().numpy(), oracle_planes(orc, p, f.poly, A, B))


@pytest.mark.parametrize("fmt", [q.FMT_INT8_PLANES, q.FMT_COEFF_U8, q.FMT_LOG])
@pytest.mark.parametrize("m,n,K", [(256, 256, 256), (130, 192, 96), (77, 100, 45), (64, 64, 4096)])
def test_pack_operands_e4m3_equals_separate_packs(torch, fmt, m, n, K):
    """qadic_pack_operands_e4m3 (one launch for aligned plane inputs with n a
    multiple of 64, two otherwise) writes the bytes of the two single packs."""
    p, k = 7, 4
    f = q.Field(p, k)
    if fmt == q.FMT_LOG:
        A, B = W.log_matrix(m, K, f.order, salt=m), W.log_matrix(K, n, f.order, salt=n)
    elif fmt == q.FMT_COEFF_U8:   # any byte: taken mod p
        A = np.random.default_rng(m).integers(0, 256, (k, m, K), dtype=np.uint8)
        B = np.random.default_rng(n).integers(0, 256, (k, K, n), dtype=np.uint8)
    else:
        A = np.random.default_rng(m).integers(-128, 128, (k, m, K), dtype=np.int8)
        B = np.random.default_rng(n).integers(-128, 128, (k, K, n), dtype=np.int8)
    dA, dB = dev(torch, A), dev(torch, B)
    Kp = (K + 15) // 16 * 16
    fused = [torch.full((k, r, Kp), 0x7F, dtype=torch.uint8, device="cuda") for r in (m, n)]
    single = [torch.full((k, r, Kp), 0x7F, dtype=torch.uint8, device="cuda") for r in (m, n)]
    f.pack_operands(fmt, dA, dB, m, n, K, fused[0], fused[1], e4m3=True)
    f.pack(fmt, dA, m, K, q.FMT_OPERAND_A_E4M3, out=single[0], ld_out=Kp)
    f.pack(fmt, dB, K, n, q.FMT_OPERAND_B_E4M3, out=single[1], ld_out=Kp)
    torch.cuda.synchronize()
    q.sync_status()
    assert torch.equal(fused[0], single[0]) and torch.equal(fused[1], single[1])


def test_pack_operands_e4m3_refusals(torch):
    L = q.lib()
    g = q.Field(37, 2)
    z = torch.zeros(2 * 64 * 64, dtype=torch.uint8, device="cuda")
    st = L.qadic_pack_operands_e4m3(g.handle, q.FMT_INT8_PLANES, q._ptr(z), 64, 64, 64, q._ptr(z), 64,
                                    q._ptr(z), 64, 64, q._ptr(z), 64, None)
    assert st == q.E_UNSUPPORTED
    f = q.Field(31, 2)
    st = L.qadic_pack_operands_e4m3(f.handle, q.FMT_INT8_PLANES, q._ptr(z), 64, 24, 24, q._ptr(z), 24,
                                    q._ptr(z), 64, 64, q._ptr(z), 24, None)
    assert st == q.E_INVALID   # ld_out 24 is not a multiple of 16


def test_stream_handle_is_the_current_stream(torch):
    """The binding passes the stream torch has current (a side stream inside
    `torch.cuda.stream`, the default one outside)."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert (q._stream().value or 0) == s.cuda_stream
    assert (q._stream().value or 0) == torch.cuda.current_stream().cuda_stream
    assert (q._stream(s).value or 0) == s.cuda_stream
