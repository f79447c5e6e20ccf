"""GPU parity at the benchmark's full sizes, in the launch configuration that
bench.py times (its own workload builders): outputs against the oracle,
entry by entry where the oracle computes them within a minute (GF(3^3)
n = 1024, GF(101^2) n = 4096, all 4096 batched products, both REDQ sweeps),
and for GF(251^2) n = 16384 sampled entries, whole rows and columns, plus
Freivalds checks (C x = A (B x) for random field vectors x), which hold at
any size."""
import numpy as np
import pytest

import bench
import paper_0710_0510_gb300 as q
from paper_0710_0510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def planes_to_mkk(X):
    """(k, rows, cols) planes -> (rows, cols, k) coefficient vectors."""
    return np.ascontiguousarray(np.transpose(X, (1, 2, 0)))


def sampled_entries_agree(orc, f, A, B, C, ii, jj):
    want = orc.gemm_entries(f.p, f.poly, planes_to_mkk(A), planes_to_mkk(B), ii, jj)
    return np.array_equal(C[:, ii, jj].T, want)


def freivalds(orc, f, A, B, C, vectors=2, seed=0):
    """C x == A (B x) over GF(p^k) for random x (all as (rows, cols, k))."""
    rng = np.random.default_rng(seed)
    n = B.shape[1]
    for _ in range(vectors):
        x = rng.integers(0, f.p, (n, 1, f.k))
        Bx = orc.gemm(f.p, f.poly, B, x)
        ABx = orc.gemm(f.p, f.poly, A, Bx)
        Cx = orc.gemm(f.p, f.poly, C, x)
        if not np.array_equal(ABx, Cx):
            return False
    return True


def test_plane_gf101_2_n4096_and_fp64_form(torch, orc):
    """Headline workload: pack + tcgen05 plane GEMM at n = 4096, every entry
    against the oracle (2.7e11 schoolbook multiply-adds on the host cores),
    and the FP64 q-adic form and the end-to-end host path on the same inputs."""
    n = 4096
    f, A, B, C, step = bench.make_plane_workload(torch, q, W, 101, n)
    step(None)
    torch.cuda.synchronize()
    Ch = C.cpu().numpy()
    want = orc.gemm(f.p, f.poly, planes_to_mkk(A), planes_to_mkk(B))
    assert np.array_equal(planes_to_mkk(Ch), want)
    del want
    C64, _ = bench.bench_fp64(None, torch, q, W, f, A, B, n, reps=1)
    assert torch.equal(C64, C)
    # end to end from pinned host buffers, as timed
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty((2, n, n), dtype=torch.uint8).pin_memory()
    ws = torch.empty(f.matmul_workspace_size(q.PATH_PLANES, q.FMT_INT8_PLANES, n, n, n),
                     dtype=torch.uint8, device="cuda")
    for _ in range(2):
        hC.zero_()
        f.matmul_host(q.PATH_PLANES, q.FMT_INT8_PLANES, hA, hB, hC, n, n, n, ws)
        torch.cuda.synchronize()
        assert np.array_equal(hC.numpy(), Ch)
    del C64, ws
    torch.cuda.empty_cache()


def test_plane_e4m3_gf31_2_n4096(torch, orc):
    """The e4m3 comparison workload as bench.py times it (one-launch e4m3
    pack + the kind::f8f6f4 plane GEMM, GF(31^2), n = 4096): 4096 sampled entries,
    two whole rows (a leader CTA's and a peer's half of a 256-row unit) and
    two whole columns against the oracle, every entry against the bf16 plane
    path on the same inputs, and one Freivalds vector."""
    n = 4096
    f, A, B = bench.make_e4m3_inputs(q, W, 31, n)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    a8 = torch.empty((2, n, n), dtype=torch.uint8, device="cuda")
    b8 = torch.empty((2, n, n), dtype=torch.uint8, device="cuda")
    f.pack_operands(q.FMT_INT8_PLANES, dA, dB, n, n, n, a8, b8, e4m3=True)
    C8 = f.gemm(q.PATH_PLANES_E4M3, a8, b8, n, n, n)
    a16 = torch.empty((2, n, n), dtype=torch.bfloat16, device="cuda")
    b16 = torch.empty((2, n, n), dtype=torch.bfloat16, device="cuda")
    f.pack_operands(q.FMT_INT8_PLANES, dA, dB, n, n, n, a16, b16)
    C16 = f.gemm(q.PATH_PLANES, a16, b16, n, n, n)
    torch.cuda.synchronize()
    q.sync_status()
    assert torch.equal(C8, C16)
    Ch = C8.cpu().numpy()
    rng = np.random.default_rng(77)
    ii = rng.integers(0, n, 4096)
    jj = rng.integers(0, n, 4096)
    assert sampled_entries_agree(orc, f, A, B, Ch, ii, jj)
    Am, Bm = planes_to_mkk(A), planes_to_mkk(B)
    for r in (5, 128 + 77):
        want = orc.gemm(f.p, f.poly, Am[r:r + 1], Bm)
        assert np.array_equal(planes_to_mkk(Ch[:, r:r + 1, :]), want), r
    for c in (0, n - 1):
        want = orc.gemm(f.p, f.poly, Am, Bm[:, c:c + 1])
        assert np.array_equal(planes_to_mkk(Ch[:, :, c:c + 1]), want), c
    assert freivalds(orc, f, Am % f.p, Bm % f.p, planes_to_mkk(Ch), vectors=1, seed=5)
    del a8, b8, C8, a16, b16, C16
    torch.cuda.empty_cache()


def test_plane_gf251_2_n16384(torch, orc):
    """The n = 16384 GF(251^2) product: 4096 sampled entries, two whole rows
    (one in a leader CTA's half of a 256-row unit, one in a peer's) and two
    whole columns, and Freivalds checks with 4 random vectors."""
    n = 16384
    f, A, B, C, step = bench.make_plane_workload(torch, q, W, 251, n)
    step(None)
    torch.cuda.synchronize()
    Ch = C.cpu().numpy()
    del C
    torch.cuda.empty_cache()
    rng = np.random.default_rng(12)
    rows, cols = [5, n - 1], [0, n - 77]
    ii = np.concatenate([rng.integers(0, n, 4096)] + [np.full(n, r) for r in rows] +
                        [np.arange(n) for _ in cols])
    jj = np.concatenate([rng.integers(0, n, 4096)] + [np.arange(n) for _ in rows] +
                        [np.full(n, c) for c in cols])
    assert sampled_entries_agree(orc, f, A, B, Ch, ii, jj)
    assert freivalds(orc, f, planes_to_mkk(A), planes_to_mkk(B), planes_to_mkk(Ch), vectors=4)


def test_fp64_gf27_n1024_full(torch, orc):
    """GF(3^3), n = 1024 from log codes: every entry against the oracle, the
    logs converted through the oracle's own generator."""
    f, A, B, C, step = bench.make_fp64_gf27(torch, q, W)
    step(None)
    torch.cuda.synchronize()
    T = orc.antilog(3, f.poly)
    want = orc.gemm(3, f.poly, T[A.astype(np.int64)], T[B.astype(np.int64)])
    assert np.array_equal(planes_to_mkk(C.cpu().numpy()), want)


def test_redq_sweep_2_28_words(torch, orc):
    """The 2^28-word sweep (p = 7, q = 2^10, 5 digits) in every table mode
    and floor, and the q = 1176 (7 | q) variant, all words compared."""
    count = 1 << 28
    w = W.redq_words(count, 5, 10)
    want = torch.from_numpy(orc.redq(7, 1024, 4, w)).cuda()
    d = torch.from_numpy(w).cuda()
    del w
    out = torch.empty_like(d)
    for mode in (0, 1, 2, 3):
        for int_floor in (False, True):
            out.zero_()
            q.redq(7, 10, 5, d, out=out, table_mode=mode, int_floor=int_floor)
            assert torch.equal(out, want), (mode, int_floor)
    del d, want
    wq = W.redq_words_q(count, 5, bench.PQ_Q)
    want = torch.from_numpy(orc.redq(7, bench.PQ_Q, 4, wq)).cuda()
    d = torch.from_numpy(wq).cuda()
    del wq
    for kw in (dict(int_floor=False), dict(int_floor=True), dict(f32_digits=True)):
        out.zero_()
        q.redq_pq(7, bench.PQ_Q, 5, d, out=out, **kw)
        assert torch.equal(out, want), kw
    del d, want, out
    torch.cuda.empty_cache()


def test_batched_4096_products(torch, orc):
    """4096 uneven products over GF(2^8), GF(7^4), GF(31^2) in one
    graph-replayed launch: every product in full against the oracle."""
    fields, dims, fidx, offs, hA, hB, dC, descs, ws = bench.make_batched(torch, q, W)
    q.batched_gemm(fields, descs, ws, graph=True)
    torch.cuda.synchronize()
    Ch = dC.cpu().numpy()

    def operands(i):
        m, n, K = (int(x) for x in dims[i])
        f = fields[fidx[i]]
        a, b, c = offs[i]
        A = planes_to_mkk(hA[a:a + f.k * m * K].reshape(f.k, m, K))
        B = planes_to_mkk(hB[b:b + f.k * K * n].reshape(f.k, K, n))
        C = planes_to_mkk(Ch[c:c + f.k * m * n].reshape(f.k, m, n))
        return f, A, B, C

    for i in range(len(descs)):
        f, A, B, C = operands(i)
        assert np.array_equal(C, orc.gemm(f.p, f.poly, A, B)), i


def test_fold_and_karatsuba_forms_n4096(torch, orc):
    """The fold-before and Karatsuba forms as bench.py times them (GF(101^2),
    n = 4096): equal to the plane product, itself checked against the oracle
    on sampled entries."""
    n = 4096
    f, A, B, C, step = bench.make_plane_workload(torch, q, W, 101, n)
    step(None)
    torch.cuda.synchronize()
    rng = np.random.default_rng(21)
    ii, jj = rng.integers(0, n, 256), rng.integers(0, n, 256)
    assert sampled_entries_agree(orc, f, A, B, C.cpu().numpy(), ii, jj)
    for fn in (bench.bench_fold, bench.bench_karatsuba):
        r = fn(None, torch, q, W, f, A, B, n, C, steps=1)
        assert r["bitexact_vs_plane"], fn.__name__
    torch.cuda.empty_cache()


def test_polymul_2_24_pairs_sampled(torch, orc):
    """The labelled 2^24-pair scaling run of the batched polynomial products,
    both product modes: a sample of pairs, and the last ones."""
    count = 1 << 24
    a, b = W.polymul_pairs(count, 7, 4, salt=1)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    idx = np.concatenate([np.random.default_rng(4).choice(count, 20000, replace=False),
                          np.arange(count - 1000, count)])
    want = orc.polymul(7, a[idx], b[idx])
    for int_words in (False, True):
        out = q.polymul_batched(7, 4, da, db, int_words=int_words).cpu().numpy()
        assert np.array_equal(out[idx], want), int_words
