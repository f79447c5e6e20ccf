"""C-ABI library loads and exports every symbol include/qadic.h declares, and
the host-side logic (field construction, bounds, argument checks) agrees
with the oracle.  No GPU: host-only field handles, and calls that fail
their checks before any launch."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_0710_0510_gb300 as q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qadic.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qadic_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(q.build.build())
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    assert set(q._SIGS) == set(declared_functions())


def test_status_strings():
    L = q.lib()
    for s in range(9):
        assert L.qadic_status_string(s)
    assert L.qadic_status_string(0) == b"ok"


FIELDS = [(3, 3), (101, 2), (251, 2), (2, 8), (7, 4), (31, 2), (5, 3), (2, 4)]


@pytest.mark.parametrize("p,k", FIELDS)
def test_host_field_matches_oracle(orc, p, k):
    f = q.Field(p, k, host_only=True)
    assert f.poly == orc.smallest_irreducible(p, k)
    assert f.generator == orc.generator(p, f.poly)
    assert f.order == p ** k and f.zero_code == p ** k - 1
    assert f.log_bytes == (1 if p ** k <= 256 else 2)
    # q: largest 2^s with (2k-1) s <= 51; n_q: Eq. 2
    assert (2 * k - 1) * f.log2_q <= 51 < (2 * k - 1) * (f.log2_q + 1)
    assert f.n_q == (2 ** f.log2_q - 1) // (k * (p - 1) ** 2)
    assert f.k_max_int32 == orc.delayed_k_bound(p, k, 31)
    h = 1 if p == 2 else (p - 1) // 2
    assert 2 * p + k * f.k_chunk_f32 * h * h <= 2 ** 24 < 2 * p + k * (f.k_chunk_f32 + 1) * h * h
    f.close()


@pytest.mark.parametrize("p,k", [(3, 3), (101, 2), (7, 3)])
def test_fp64_block_matches_eq2_reading(orc, p, k):
    f = q.Field(p, k, host_only=True)
    assert (2 ** f.log2_q, f.n_q) == orc.qadic_bounds(p, k, 53)


def test_given_polynomial_accepted_and_reducible_rejected():
    f = q.Field(3, 3, poly=[2, 2, 0, 1], host_only=True)   # X^3 + 2X + 2: no root mod 3
    assert f.poly == [2, 2, 0, 1]
    with pytest.raises(q.QadicError) as e:
        q.Field(3, 3, poly=[1, 0, 0, 1], host_only=True)   # X^3 + 1 = (X+1)^3 mod 3
    assert e.value.status == q.E_REDUCIBLE
    with pytest.raises(q.QadicError) as e:
        q.Field(101, 2, poly=[1, 0, 1], host_only=True)    # X^2 + 1: -1 is a square mod 101
    assert e.value.status == q.E_REDUCIBLE


def test_bad_fields_rejected():
    for p, k, st in [(4, 2, q.E_NOT_PRIME), (9, 1, q.E_NOT_PRIME), (257, 1, q.E_INVALID),
                     (3, 0, q.E_INVALID), (2, 17, q.E_INVALID), (251, 3, q.E_INVALID)]:
        with pytest.raises(q.QadicError) as e:
            q.Field(p, k, host_only=True)
        assert e.value.status == st, (p, k)


def test_irreducibility_test_agrees_with_oracle(orc):
    L = q.lib()
    for p, k in [(2, 4), (3, 3), (3, 4), (5, 2), (7, 2), (2, 6)]:
        for v in range(p ** k):
            poly = [(v // p ** i) % p for i in range(k)] + [1]
            arr = (ctypes.c_uint32 * (k + 1))(*poly)
            h = ctypes.c_void_p()
            st = L.qadic_field_init(ctypes.byref(h), p, k, ctypes.cast(arr, ctypes.c_void_p),
                                    q.FIELD_HOST_ONLY)
            assert (st == q.OK) == orc.irreducible(p, poly), (p, poly)
            if st == q.OK:
                L.qadic_field_destroy(h)


def test_host_only_field_rejects_launches():
    f = q.Field(101, 2, host_only=True)
    L = q.lib()
    st = L.qadic_gemm(f.handle, q.PATH_PLANES, 4, 4, 4, ctypes.c_void_p(16), 8,
                      ctypes.c_void_p(16), 8, ctypes.c_void_p(16), 4, None, 0, None)
    assert st == q.E_INVALID
    st = L.qadic_pack(f.handle, q.FMT_LOG, ctypes.c_void_p(16), 4, 4, 4, q.FMT_QADIC_F64,
                      ctypes.c_void_p(16), 4, None)
    assert st == q.E_INVALID


def test_polymul_plain_fp64_rejected_for_config_sizes():
    """p = 7, k = 4, q = 2^8: (2k-1) log2 q = 56 >= 53, so the single-rounded
    product is refused (overflow rejected rather than miscomputed)."""
    L = q.lib()
    st = L.qadic_polymul_batched(7, 4, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 ctypes.c_void_p(16), 65536, q.POLYMUL_PLAIN_F64, None)
    assert st == q.E_OVERFLOW
    assert b"53" in L.qadic_last_error()


def test_redq_lemma1_limit_rejected():
    L = q.lib()
    # 5 digits of 2^11: 55 bits > 51
    st = L.qadic_redq(7, 11, 5, ctypes.c_void_p(16), ctypes.c_void_p(16), 10, 3, None)
    assert st == q.E_OVERFLOW
    # misaligned pointers
    st = L.qadic_redq(7, 10, 5, ctypes.c_void_p(8), ctypes.c_void_p(16), 10, 3, None)
    assert st == q.E_INVALID
    # q must exceed p
    st = L.qadic_redq(7, 2, 5, ctypes.c_void_p(16), ctypes.c_void_p(16), 10, 3, None)
    assert st == q.E_INVALID


def test_redq_pq_rejections():
    L = q.lib()
    a, b = ctypes.c_void_p(16), ctypes.c_void_p(32)
    # q not a multiple of p
    assert L.qadic_redq_pq(7, 1024, 5, a, b, 10, 0, None) == q.E_INVALID
    # q below p
    assert L.qadic_redq_pq(7, 0, 5, a, b, 10, 0, None) == q.E_INVALID
    # 1183^5 > 2^51 (Lemma 1 limit); 1176^5 is just below it
    assert L.qadic_redq_pq(7, 1183, 5, a, b, 10, 0, None) == q.E_OVERFLOW
    assert b"2^51" in L.qadic_last_error()
    # q^ndigits overflowing 64 bits is rejected, not wrapped
    assert L.qadic_redq_pq(7, 7 * 2 ** 40, 30, a, b, 10, 0, None) == q.E_OVERFLOW
    # unknown flags, misaligned pointers, non-prime p
    assert L.qadic_redq_pq(7, 1176, 5, a, b, 10, 0x1, None) == q.E_INVALID
    assert L.qadic_redq_pq(7, 1176, 5, ctypes.c_void_p(8), b, 10, 0, None) == q.E_INVALID
    assert L.qadic_redq_pq(9, 18, 5, a, b, 10, 0, None) == q.E_INVALID
    assert L.qadic_redq_pq(7, 1176, 5, None, None, 0, 0, None) == q.OK
    # FP32 digits: one floor flag at most, q^2 < 2^21 (q <= 1448), <= 8 digits
    F32 = q.REDQ_F32_DIGITS
    assert L.qadic_redq_pq(7, 1176, 5, a, b, 10, F32 | q.REDQ_INT_FLOOR, None) == q.E_INVALID
    assert L.qadic_redq_pq(3, 1449, 4, a, b, 10, F32, None) == q.E_UNSUPPORTED
    assert L.qadic_redq_pq(2, 2 ** 32, 1, a, b, 10, F32, None) == q.E_UNSUPPORTED
    assert L.qadic_redq_pq(3, 3, 9, a, b, 10, F32, None) == q.E_UNSUPPORTED
    assert L.qadic_redq_pq(181, 1448, 4, None, None, 0, F32, None) == q.OK
    assert L.qadic_redq_pq(3, 3, 8, None, None, 0, F32, None) == q.OK


@pytest.mark.parametrize("p", [2, 3, 7, 31, 101, 251])
@pytest.mark.parametrize("int_words", [False, True])
def test_fqt_parameters_satisfy_eq2(p, int_words):
    """q = 2^s as large as the word allows, n_q the largest count with
    q > n_q (d+1)(p-1)^2 + (p-1), D_q = ceil((N+1)/(d+1)) - 1 (Sec. 6)."""
    for d in range(0, 8):
        D = 2 * d + 1
        s = min(64 // D, 32 // (d + 1)) if int_words else 51 // D
        q_ = 2 ** s
        unit = (d + 1) * (p - 1) ** 2
        try:
            info = q.polymul_fqt_info(p, 500, d, int_words)
        except q.QadicError as e:
            assert e.status == q.E_OVERFLOW
            assert unit + (p - 1) >= q_          # not even one product fits
            continue
        assert info.log2_q == s
        assert (2 * d + 1) * s <= (64 if int_words else 51)
        if int_words:
            assert (d + 1) * s <= 32
        n_q = info.n_q
        assert n_q >= 1 and n_q * unit + (p - 1) < q_
        if n_q < 2 ** 32 - 1:
            assert (n_q + 1) * unit + (p - 1) >= q_
        assert info.D_q == -(-501 // (d + 1)) - 1
        assert info.word_products == (info.D_q + 1) ** 2
        assert info.word_bits == (64 if int_words else 53)


def test_fqt_paper_example_parameters():
    """p = 3, N = 500 with binary64 words: d = 2 packs 3 coefficients into
    q = 2^10 with 85 products between reductions, D_q = 166 (Sec. 6 uses
    this N and p)."""
    info = q.polymul_fqt_info(3, 500, 2)
    assert (info.log2_q, info.n_q, info.D_q) == (10, 85, 166)
    info = q.polymul_fqt_info(3, 500, 0)
    assert info.D_q == 500 and info.word_products == 501 ** 2


def test_polymul_fqt_rejections():
    L = q.lib()
    a = ctypes.c_void_p(16)
    info = q.FqtInfo()
    assert L.qadic_polymul_fqt_info(4, 10, 1, 0, ctypes.byref(info)) == q.E_INVALID
    assert L.qadic_polymul_fqt_info(3, 10, 25, 0, ctypes.byref(info)) == q.E_INVALID
    assert L.qadic_polymul_fqt_info(3, 10, 1, 2, ctypes.byref(info)) == q.E_INVALID
    assert L.qadic_polymul_fqt_info(3, 10, 5, 0, ctypes.byref(info)) == q.E_OVERFLOW
    assert L.qadic_polymul_fqt(3, 10, 1, None, a, a, 4, 0, None) == q.E_INVALID
    assert L.qadic_polymul_fqt(3, 10, 1, a, a, a, -1, 0, None) == q.E_INVALID
    assert L.qadic_polymul_fqt(3, 10, 1, None, None, None, 0, 0, None) == q.OK
    # too long for one CTA's shared memory: refused before any launch
    assert L.qadic_polymul_fqt(3, 1 << 20, 0, a, a, a, 4, 0, None) == q.E_UNSUPPORTED


def test_batched_tile_table_and_selection():
    for k in range(1, 9):
        cfgs = q.batched_tile_configs(k)
        assert len(cfgs) >= 3 and q.batched_selected_tiles(k) == 0
        for bm, bn, bk, smem in cfgs:
            assert bm % 32 == 0 and bn % 16 == 0 and bk % 16 == 0
            assert smem == (k * bm * (bk + 8) + k * bk * (bn + 8)) * 2
            assert smem <= 227 * 1024 // 3           # three CTAs per SM
        assert len(set(cfgs)) == len(cfgs)          # no duplicate candidates
    L = q.lib()
    assert L.qadic_batched_select_tiles(0, 0) == q.E_INVALID
    assert L.qadic_batched_select_tiles(9, 0) == q.E_INVALID
    assert L.qadic_batched_select_tiles(2, 5) == q.E_INVALID
    assert L.qadic_batched_select_tiles(5, 4) == q.E_INVALID
    assert L.qadic_batched_select_tiles(2, -2) == q.E_INVALID
    q.batched_select_tiles(2, 3)
    assert q.batched_selected_tiles(2) == 3
    q.batched_select_tiles(2, -1)
    assert q.batched_selected_tiles(2) == 0


def test_fold_format_and_path_constants_match_header():
    h = open(os.path.join(os.path.dirname(__file__), "..", "include", "qadic.h")).read()
    assert re.search(r"QADIC_FMT_OPERAND_B_FOLD = 6", h) and q.FMT_OPERAND_B_FOLD == 6
    assert re.search(r"QADIC_PATH_FOLD = 2", h) and q.PATH_FOLD == 2
    assert q.fold_n_pad(1) == 256 and q.fold_n_pad(256) == 256 and q.fold_n_pad(257) == 512
    assert re.search(r"QADIC_FMT_OPERAND_A_KARA = 7", h) and q.FMT_OPERAND_A_KARA == 7
    assert re.search(r"QADIC_FMT_OPERAND_B_KARA = 8", h) and q.FMT_OPERAND_B_KARA == 8
    assert re.search(r"QADIC_PATH_KARATSUBA = 3", h) and q.PATH_KARATSUBA == 3
    assert re.search(r"QADIC_FMT_OPERAND_A_E4M3 = 9", h) and q.FMT_OPERAND_A_E4M3 == 9
    assert re.search(r"QADIC_FMT_OPERAND_B_E4M3 = 10", h) and q.FMT_OPERAND_B_E4M3 == 10
    assert re.search(r"QADIC_PATH_PLANES_E4M3 = 4", h) and q.PATH_PLANES_E4M3 == 4


def test_e4m3_workspace_is_one_byte_per_element_padded_to_16():
    """Packed e4m3 operands: k planes of m x K16 and n x K16 bytes, each
    block 256-byte aligned; half the bf16 planes' bytes when K % 16 == 0."""
    f = q.Field(31, 2, host_only=True)
    L = q.lib()
    a256 = lambda x: (x + 255) // 256 * 256
    for m, n, K in ((64, 64, 64), (7, 9, 17), (300, 200, 333)):
        K16 = (K + 15) // 16 * 16
        want = a256(2 * m * K16) + a256(2 * n * K16)
        assert L.qadic_matmul_device_workspace_size(f.handle, q.PATH_PLANES_E4M3, m, n, K) == want
    assert L.qadic_matmul_device_workspace_size(f.handle, q.PATH_PLANES_E4M3, 128, 128, 128) * 2 == \
        L.qadic_matmul_device_workspace_size(f.handle, q.PATH_PLANES, 128, 128, 128)


def test_selftest_rejects_bad_poll_counts():
    L = q.lib()
    assert L.qadic_selftest_bounded_wait(0, None) == q.E_INVALID
    assert L.qadic_selftest_bounded_wait((1 << 26) + 1, None) == q.E_INVALID


def test_zero_counts_are_noops():
    L = q.lib()
    assert L.qadic_redq(7, 10, 5, None, None, 0, 3, None) == q.OK
    assert L.qadic_polymul_batched(7, 4, None, None, None, 0, 0, None) == q.OK


def test_desc_array_is_built_once():
    """A prebuilt descriptor array passes through unchanged; a list becomes
    an array of the same descriptors."""
    d = [q.GemmDesc(0, 3, 4, 5, 16, 32, 48, 5, 4, 4, 0), q.GemmDesc(1, 7, 8, 9, 0, 0, 0, 9, 8, 8, 0)]
    arr = q.desc_array(d)
    assert len(arr) == 2 and arr[1].m == 7 and arr[0].ldb == 4
    assert q.desc_array(arr) is arr
