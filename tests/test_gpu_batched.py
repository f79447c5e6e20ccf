"""GPU parity of the batched persistent kernel (qadic_batched_gemm) against
the oracle, product by product, bit-exact."""
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


class Batch:
    """Products laid out in three flat device buffers (A, B, C)."""

    def __init__(self, torch, fields, shapes, fidx, seed, converted=True):
        rng = np.random.default_rng(seed)
        self.fields, self.shapes, self.fidx = fields, shapes, fidx
        self.A, self.B, offs = [], [], []
        oa = ob = oc = 0
        for (m, n, K), fi in zip(shapes, fidx):
            f = fields[fi]
            self.A.append(rng.integers(0, f.p, (f.k, m, K), dtype=np.uint8))
            self.B.append(rng.integers(0, f.p, (f.k, K, n), dtype=np.uint8))
            offs.append((oa, ob, oc))
            oa += f.k * m * K
            ob += f.k * K * n
            oc += f.k * m * n
        self.dA = torch.from_numpy(np.concatenate([a.ravel() for a in self.A])).cuda()
        self.dB = torch.from_numpy(np.concatenate([b.ravel() for b in self.B])).cuda()
        self.dC = torch.zeros(oc, dtype=torch.uint8, device="cuda")
        self.offs = offs
        self.descs = []
        for i, ((m, n, K), fi) in enumerate(zip(shapes, fidx)):
            a, b, c = offs[i]
            self.descs.append(q.GemmDesc(fi, m, n, K, self.dA.data_ptr() + a,
                                         self.dB.data_ptr() + b, self.dC.data_ptr() + c,
                                         K, n, n, 0))
        # with the fields: room for converted operands (the cp.async path);
        # without: the work list only (operand bytes staged through registers)
        ws = q.batched_workspace_size(self.descs, fields if converted else None)
        self.ws = torch.empty(ws, dtype=torch.uint8, device="cuda")

    def run(self, graph=False):
        q.batched_gemm(self.fields, self.descs, self.ws, graph=graph)

    def result(self, i):
        m, n, K = self.shapes[i]
        f = self.fields[self.fidx[i]]
        c = self.offs[i][2]
        return self.dC[c:c + f.k * m * n].cpu().numpy().reshape(f.k, m, n)

    def expected(self, orc, i):
        f = self.fields[self.fidx[i]]
        C = orc.gemm(f.p, f.poly, np.transpose(self.A[i], (1, 2, 0)),
                     np.transpose(self.B[i], (1, 2, 0)))
        return np.transpose(C, (2, 0, 1))


def mixed_fields():
    return [q.Field(2, 8), q.Field(7, 4), q.Field(31, 2)]


@pytest.mark.parametrize("converted", [True, False])
def test_batched_mixed_fields(torch, orc, converted):
    fields = mixed_fields()
    dims, fidx = W.batched_shapes(60, salt=1)
    shapes = [tuple(int(x) for x in d) for d in dims]
    shapes[:5] = [(1, 1, 1), (16, 16, 16), (256, 256, 256), (65, 17, 33), (3, 200, 7)]
    bt = Batch(torch, fields, shapes, [int(x) for x in fidx], seed=5, converted=converted)
    bt.run()
    q.sync_status()
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i)), (i, shapes[i], fidx[i])


def test_batched_paths_agree_and_sizes(torch, orc):
    """The tensor-core path (converted operands) and the register-staged path
    give the same bytes; the size query with fields covers the converted
    operands in their blocked layout on top of the work list."""
    fields = mixed_fields()
    dims, fidx = W.batched_shapes(30, salt=7)
    shapes = [tuple(int(x) for x in d) for d in dims]
    fi = [int(x) for x in fidx]
    a = Batch(torch, fields, shapes, fi, seed=6, converted=True)
    b = Batch(torch, fields, shapes, fi, seed=6, converted=False)
    a.run(graph=True)
    b.run(graph=True)
    for i in range(len(shapes)):
        assert np.array_equal(a.result(i), b.result(i)), i
    small = q.batched_workspace_size(a.descs)
    big = q.batched_workspace_size(a.descs, fields)
    r8 = lambda x: (x + 7) // 8 * 8
    cdiv = lambda a, b: -(-a // b)
    conv = items = tiles = 0
    for (m, n, K), f in zip(shapes, fi):
        k = fields[f].k
        # tensor-core blocks: 32-byte K-blocks of 32 fp8 (p <= 31) or 16 bf16
        # elements; A as k planes of m rounded up to 8 rows, B^T as k planes
        # of BN-column tiles (BN = 128, 64, 32, 32, 16, ... for k = 1, 2, 3, 4, 5..)
        ks = cdiv(K, 32 if fields[f].p <= 31 else 16)
        bn = 128 if k == 1 else 64 if k == 2 else 32 if k <= 4 else 16
        a_bytes = k * r8(m) * 32 * ks
        b_bytes = k * bn * 32 * ks * cdiv(n, bn)
        conv += a_bytes + b_bytes
        items += cdiv(a_bytes // 16, 4096) + cdiv(k * ks * 2 * n, 4096)
        tiles += cdiv(m, 128) * cdiv(n, bn)
    # the work list holds 48-byte tile records on this path (8-byte ones with
    # the smallest tile shape in the work-list-only size)
    small_tiles = sum(cdiv(m, 32) * cdiv(n, 16) for m, n, K in shapes)
    header = small - 8 * small_tiles
    assert big >= header - 512 + 48 * tiles + conv
    # + 256-byte alignment of each operand and section, + the conversion items (8 bytes each)
    assert big <= header + 48 * tiles + conv + 2 * 256 * len(shapes) + 8 * items + 1024


@pytest.mark.parametrize("pk", [(3, 3), (5, 5), (2, 6), (101, 2), (3, 7), (13, 3), (2, 1)])
def test_batched_other_fields(torch, orc, pk):
    fields = [q.Field(*pk)]
    shapes = [(33, 47, 95), (64, 64, 64), (100, 3, 250), (1, 70, 129)]
    bt = Batch(torch, fields, shapes, [0] * len(shapes), seed=pk[0])
    bt.run()
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i)), (pk, shapes[i])


def test_batched_exact_chunks_p251(torch, orc):
    """GF(251^2): the exact FP32 chunk is 536 -> 16 K-blocks of 32, so
    K = 2000 crosses three in-register reductions; all-max inputs push every
    chunk to the bound."""
    f = q.Field(251, 2)
    shapes = [(64, 64, 2000), (50, 70, 1100)]
    bt = Batch(torch, [f], shapes, [0, 0], seed=2)
    bt.A[0][:] = 126                      # centred -125 for every coefficient
    bt.B[0][:] = 126
    bt.dA[: bt.A[0].size] = torch.from_numpy(bt.A[0].ravel()).cuda()
    bt.dB[: bt.B[0].size] = torch.from_numpy(bt.B[0].ravel()).cuda()
    bt.run()
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i))


def test_batched_graph_replay(torch, orc):
    fields = mixed_fields()
    dims, fidx = W.batched_shapes(40, salt=2)
    shapes = [tuple(int(x) for x in d) for d in dims]
    bt = Batch(torch, fields, shapes, [int(x) for x in fidx], seed=9)
    bt.run(graph=True)
    first = [bt.result(i) for i in range(len(shapes))]
    bt.dC.zero_()
    bt.run(graph=True)                     # replay of the cached graph
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), first[i])
        assert np.array_equal(first[i], bt.expected(orc, i))
    # new input data behind the same pointers is picked up by the replay
    new = np.random.default_rng(3).integers(0, fields[bt.fidx[0]].p, bt.A[0].shape,
                                            dtype=np.uint8)
    bt.A[0] = new
    bt.dA[: new.size] = torch.from_numpy(new.ravel()).cuda()
    bt.run(graph=True)
    assert np.array_equal(bt.result(0), bt.expected(orc, 0))


def test_batched_matches_plane_gemm(torch, orc):
    """One GF(101^2) product through both the batched kernel and the
    tensor-core plane GEMM."""
    f = q.Field(101, 2)
    m, n, K = 192, 160, 300
    bt = Batch(torch, [f], [(m, n, K)], [0], seed=4)
    bt.run()
    a = f.pack(q.FMT_COEFF_U8, torch.from_numpy(bt.A[0]).cuda(), m, K, q.FMT_OPERAND_A,
               out=torch.zeros((2, m, 304), dtype=torch.bfloat16, device="cuda"), ld_out=304)
    b = f.pack(q.FMT_COEFF_U8, torch.from_numpy(bt.B[0]).cuda(), K, n, q.FMT_OPERAND_B,
               out=torch.zeros((2, n, 304), dtype=torch.bfloat16, device="cuda"), ld_out=304)
    C = f.gemm(q.PATH_PLANES, a, b, m, n, K, lda=304, ldb=304).cpu().numpy()
    assert np.array_equal(bt.result(0), C)


def test_batched_rejects_bad_descriptors(torch):
    f = q.Field(31, 2)
    x = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    ws = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    good = q.GemmDesc(0, 4, 4, 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 4, 4, 0)
    for bad in (q.GemmDesc(1, 4, 4, 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 4, 4, 0),
                q.GemmDesc(0, 0, 4, 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 4, 4, 0),
                q.GemmDesc(0, 4, 4, 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), 3, 4, 4, 0),
                q.GemmDesc(0, 4, 4, 4, 0, x.data_ptr(), x.data_ptr(), 4, 4, 4, 0)):
        with pytest.raises(q.QadicError) as e:
            q.batched_gemm([f], [good, bad], ws)
        assert e.value.status == q.E_INVALID
    with pytest.raises(q.QadicError) as e:
        q.batched_gemm([f], [good], ws[:64])
    assert e.value.status == q.E_NOMEM


# ------------------------------------------------- tile configurations ----

@pytest.fixture
def restore_tiles():
    yield
    for k in range(1, 9):
        q.batched_select_tiles(k, -1)


@pytest.mark.parametrize("converted", [True, False])
@pytest.mark.parametrize("pk", [(101, 1), (31, 2), (3, 3), (7, 4), (5, 5), (2, 6), (2, 8), (3, 8)])
def test_batched_every_tile_configuration(torch, orc, restore_tiles, pk, converted):
    """Each (BM, BN, BK) candidate of the autotuner computes the same exact
    products on both paths: ragged shapes, K across exact-chunk boundaries."""
    f = q.Field(*pk)
    shapes = [(1, 1, 1), (33, 47, 95), (64, 64, 64), (100, 3, 250), (1, 70, 129), (77, 65, 640)]
    for c in range(len(q.batched_tile_configs(f.k))):
        q.batched_select_tiles(f.k, c)
        bt = Batch(torch, [f], shapes, [0] * len(shapes), seed=pk[0] + c, converted=converted)
        bt.run(graph=bool(c % 2))
        for i in range(len(shapes)):
            assert np.array_equal(bt.result(i), bt.expected(orc, i)), (pk, c, shapes[i])


@pytest.mark.parametrize("converted", [True, False])
def test_batched_p251_chunks_every_configuration(torch, orc, restore_tiles, converted):
    """GF(251^2) (exact chunk 536 = 16 blocks of 32 or 8 of 64), all-max
    inputs, K = 2000, under every configuration for k = 2."""
    f = q.Field(251, 2)
    for c in range(len(q.batched_tile_configs(2))):
        q.batched_select_tiles(2, c)
        bt = Batch(torch, [f], [(64, 64, 2000), (50, 70, 1100)], [0, 0], seed=2,
                   converted=converted)
        bt.A[0][:] = 126
        bt.B[0][:] = 126
        bt.dA[: bt.A[0].size] = torch.from_numpy(bt.A[0].ravel()).cuda()
        bt.dB[: bt.B[0].size] = torch.from_numpy(bt.B[0].ravel()).cuda()
        bt.run()
        for i in range(2):
            assert np.array_equal(bt.result(i), bt.expected(orc, i)), c


@pytest.mark.parametrize("converted", [True, False])
def test_batched_gf256_chunks_every_configuration(torch, orc, restore_tiles, converted):
    """GF(2^8), whose converted path runs on f16 operands and accumulators:
    all-one planes (every plane product is 1, the largest sums), K across the
    f16 chunk of 2047/8 = 255 elements, every configuration for k = 8."""
    f = q.Field(2, 8)
    shapes = [(64, 64, 2000), (50, 70, 1100), (33, 16, 255), (32, 16, 256), (17, 9, 257)]
    for c in range(len(q.batched_tile_configs(8))):
        q.batched_select_tiles(8, c)
        bt = Batch(torch, [f], shapes, [0] * len(shapes), seed=3, converted=converted)
        for i in range(len(shapes)):
            bt.A[i][:] = 1
            bt.B[i][:] = 1
        bt.dA[:] = torch.from_numpy(np.concatenate([x.ravel() for x in bt.A])).cuda()
        bt.dB[:] = torch.from_numpy(np.concatenate([x.ravel() for x in bt.B])).cuda()
        bt.run(graph=bool(c % 2))
        for i in range(len(shapes)):
            assert np.array_equal(bt.result(i), bt.expected(orc, i)), (c, shapes[i])


@pytest.mark.parametrize("converted", [True, False])
@pytest.mark.parametrize("pk", [(31, 2), (7, 4), (2, 8)])
def test_batched_fp8_fields_all_max(torch, orc, pk, converted):
    """The fields whose coefficients run as fp8 e4m3 (p <= 31), every
    coefficient at -h (the same sign: every plane product is h^2 > 0), K up
    to 4096: the plane sums reach k K h^2 (1.8e6 for GF(31^2)), so any loss
    of low-order bits in the tensor-core accumulation shows."""
    p, k = pk
    f = q.Field(p, k)
    h = (p - 1) // 2 if p > 2 else 1
    code = p - h if p > 2 else 1          # least non-negative representative of -h (p = 2: 1)
    shapes = [(64, 64, 4096), (33, 17, 4096), (16, 16, 1000), (130, 70, 2049)]
    bt = Batch(torch, [f], shapes, [0] * len(shapes), seed=p, converted=converted)
    for i in range(len(shapes)):
        bt.A[i][:] = code
        bt.B[i][:] = code
    bt.dA[:] = torch.from_numpy(np.concatenate([x.ravel() for x in bt.A])).cuda()
    bt.dB[:] = torch.from_numpy(np.concatenate([x.ravel() for x in bt.B])).cuda()
    bt.run()
    q.sync_status()
    for i in range(len(shapes)):
        got = bt.result(i)
        m, n, K = shapes[i]
        want = bt.expected(orc, i) if m * n * K <= 64 * 64 * 4096 else None
        if want is None:   # every entry is the same: compare one against the oracle
            one = orc.gemm(p, f.poly, np.transpose(bt.A[i][:, :1, :], (1, 2, 0)),
                           np.transpose(bt.B[i][:, :, :1], (1, 2, 0)))
            want = np.broadcast_to(np.transpose(one, (2, 0, 1)), got.shape)
        assert np.array_equal(got, want), (pk, shapes[i])


@pytest.mark.parametrize("converted", [True, False])
def test_batched_maximum_sizes(torch, orc, converted):
    """The largest product the batched entry point takes (m = n = K = 4096)
    beside small ones, GF(31^2) and GF(2^8): sampled entries and whole edge
    rows and columns against the oracle."""
    f31, f2 = q.Field(31, 2), q.Field(2, 8)
    shapes = [(4096, 4096, 4096), (1, 4096, 4096), (4096, 1, 7), (17, 33, 4096)]
    fidx = [0, 1, 0, 1]
    bt = Batch(torch, [f31, f2], shapes, fidx, seed=21, converted=converted)
    bt.run()
    rng = np.random.default_rng(22)
    for i, (m, n, K) in enumerate(shapes):
        f = bt.fields[fidx[i]]
        C = bt.result(i)
        ii = np.concatenate([rng.integers(0, m, 64), np.full(min(n, 64), m - 1), np.arange(min(m, 64))])
        jj = np.concatenate([rng.integers(0, n, 64), np.arange(min(n, 64)), np.full(min(m, 64), n - 1)])
        want = orc.gemm_entries(f.p, f.poly, np.transpose(bt.A[i], (1, 2, 0)),
                                np.transpose(bt.B[i], (1, 2, 0)), ii, jj)
        assert np.array_equal(C[:, ii, jj].T, want), (i, shapes[i])


@pytest.mark.parametrize("converted", [True, False])
def test_graph_cache_after_field_destroyed(torch, orc, converted):
    """A graph cached for a destroyed field is not replayed for a new field
    (its handle may reuse the old address) with the same descriptors and
    workspace."""
    shapes = [(40, 24, 70), (1, 1, 1)]
    f1 = q.Field(2, 8)
    bt = Batch(torch, [f1], shapes, [0, 0], seed=12, converted=converted)
    bt.run(graph=True)
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i))
    f1.close()
    f2 = q.Field(3, 8)
    bt.fields = [f2]
    descs = bt.descs
    q.batched_gemm([f2], descs, bt.ws, graph=True)
    torch.cuda.synchronize()
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i)), i


def test_graph_replay_after_another_list_in_the_same_workspace(torch, orc):
    """graph(X), graph(Y), graph(X) on one workspace: the third call replays
    X's cached graph and must first restore X's work list."""
    fields = mixed_fields()
    dims, fidx = W.batched_shapes(30, salt=4)
    shapes = [tuple(int(x) for x in d) for d in dims]
    x = Batch(torch, fields, shapes, [int(v) for v in fidx], seed=11)
    y = Batch(torch, fields, shapes[::-1], [int(v) for v in fidx][::-1], seed=12)
    ws = torch.empty(max(x.ws.numel(), y.ws.numel()), dtype=torch.uint8, device="cuda")
    x.ws = y.ws = ws
    x.run(graph=True)
    y.run(graph=True)
    x.dC.zero_()
    x.run(graph=True)
    for i in range(len(shapes)):
        assert np.array_equal(x.result(i), x.expected(orc, i)), i
        assert np.array_equal(y.result(i), y.expected(orc, i)), i


def test_autotune_selects_measured_configurations(torch, orc, restore_tiles):
    fields = mixed_fields()
    dims, fidx = W.batched_shapes(200, salt=6)
    shapes = [tuple(int(v) for v in d) for d in dims]
    bt = Batch(torch, fields, shapes, [int(v) for v in fidx], seed=13)
    chosen = q.batched_autotune(fields, bt.descs, bt.ws, reps=2)
    assert set(chosen) == {f.k for f in fields}
    for k, c in chosen.items():
        assert 0 <= c < len(q.batched_tile_configs(k))
        assert q.batched_selected_tiles(k) == c
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i)), i
    bt.dC.zero_()
    bt.run(graph=True)
    for i in range(0, len(shapes), 7):
        assert np.array_equal(bt.result(i), bt.expected(orc, i)), i


@pytest.mark.parametrize("converted", [True, False])
def test_batched_unreduced_bytes(torch, orc, converted):
    """Operand bytes anywhere in [0, 255] are taken mod p (canonical and
    unreduced bytes side by side in the same rows and columns), on both
    paths."""
    fields = mixed_fields()
    shapes = [(70, 96, 64), (33, 130, 48), (128, 64, 100), (5, 257, 17), (64, 64, 64), (90, 32, 40)]
    fidx = [0, 1, 2, 0, 1, 0]
    bt = Batch(torch, fields, shapes, fidx, seed=9, converted=converted)
    rng = np.random.default_rng(10)
    for i, (m, n, K) in enumerate(shapes):
        f = fields[fidx[i]]
        a = rng.integers(0, 256, (f.k, m, K), dtype=np.uint8)
        b = rng.integers(0, 256, (f.k, K, n), dtype=np.uint8)
        a[:, ::2] %= f.p             # every other row canonical
        b[:, :, ::3] %= f.p          # every third column canonical
        oa, ob, _ = bt.offs[i]
        bt.dA[oa:oa + a.size] = torch.from_numpy(a.ravel()).cuda()
        bt.dB[ob:ob + b.size] = torch.from_numpy(b.ravel()).cuda()
        bt.A[i], bt.B[i] = a % f.p, b % f.p
    bt.run()
    q.sync_status()
    for i in range(len(shapes)):
        assert np.array_equal(bt.result(i), bt.expected(orc, i)), (i, shapes[i])


@pytest.mark.parametrize("converted", [True, False])
def test_batched_strided_unaligned_operands(torch, orc, converted):
    """Row strides above the widths (odd ones among them) and operand bases
    at every offset mod 4: the conversion's word loads of B columns (one or
    two aligned words per K row, four columns per thread) and the ragged
    last column group, on both paths."""
    fields = mixed_fields()
    shapes = [(70, 97, 64), (33, 130, 48), (128, 61, 100), (5, 257, 17), (64, 66, 64),
              (90, 3, 40), (17, 1, 33), (129, 255, 255)]
    fidx = [0, 1, 2, 0, 1, 2, 0, 1]
    pads = [(3, 5), (1, 0), (0, 7), (2, 2), (5, 1), (0, 13), (1, 3), (4, 9)]
    rng = np.random.default_rng(31)
    As, Bs, descs, offs = [], [], [], []
    ra = rb = rc = 0
    layout = []
    for (m, n, K), fi, (pa, pb) in zip(shapes, fidx, pads):
        f = fields[fi]
        lda, ldb = K + pa, n + pb
        ra += 1 + (ra % 3)     # bases at varied offsets mod 4
        rb += 1 + (rb % 3)
        layout.append((ra, rb, rc, lda, ldb))
        ra += f.k * m * lda
        rb += f.k * K * ldb
        rc += f.k * m * n
        As.append(rng.integers(0, f.p, (f.k, m, K), dtype=np.uint8))
        Bs.append(rng.integers(0, f.p, (f.k, K, n), dtype=np.uint8))
    hA = np.full(ra + 64, 0xEE, np.uint8)
    hB = np.full(rb + 64, 0xEE, np.uint8)
    for (m, n, K), fi, A, B, (oa, ob, oc, lda, ldb) in zip(shapes, fidx, As, Bs, layout):
        f = fields[fi]
        va = hA[oa:oa + f.k * m * lda].reshape(f.k, m, lda)
        va[:, :, :K] = A
        vb = hB[ob:ob + f.k * K * ldb].reshape(f.k, K, ldb)
        vb[:, :, :n] = B
    dA = torch.from_numpy(hA).cuda()
    dB = torch.from_numpy(hB).cuda()
    dC = torch.zeros(rc, dtype=torch.uint8, device="cuda")
    for (m, n, K), fi, (oa, ob, oc, lda, ldb) in zip(shapes, fidx, layout):
        descs.append(q.GemmDesc(fi, m, n, K, dA.data_ptr() + oa, dB.data_ptr() + ob,
                                dC.data_ptr() + oc, lda, ldb, n, 0))
    ws = torch.empty(q.batched_workspace_size(descs, fields if converted else None),
                     dtype=torch.uint8, device="cuda")
    q.batched_gemm(fields, descs, ws)
    torch.cuda.synchronize()
    q.sync_status()
    for (m, n, K), fi, A, B, (oa, ob, oc, lda, ldb) in zip(shapes, fidx, As, Bs, layout):
        f = fields[fi]
        got = dC[oc:oc + f.k * m * n].cpu().numpy().reshape(f.k, m, n)
        want = orc.gemm(f.p, f.poly, np.transpose(A, (1, 2, 0)), np.transpose(B, (1, 2, 0)))
        assert np.array_equal(got, np.transpose(want, (2, 0, 1))), (m, n, K, fi)
