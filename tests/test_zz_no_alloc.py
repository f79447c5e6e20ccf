"""The allocation-free batched entry point (qadic_batched_gemm_noalloc).

It exists for callers that cannot allocate during a call -- a framework
whose allocator owns every byte of device memory, a loop where a
cudaMalloc/cudaFree would synchronise the device, a plugin that is handed
only its inputs and outputs.  It keeps its work list in a fixed array inside
the library.  This file checks, through the C ABI, that it returns exactly
what qadic_batched_gemm (the workspace version) returns, on two calls in a
row, that two different batches issued back to back on one stream with no
synchronisation in between both come out right, that a small mixed-field
batch matches the CPU oracle, and that a work list too large for the fixed
array is refused.

The file name makes pytest collect it last, so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_0710_0510_gb300 as q
from paper_0710_0510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(torch, fields, count, seed, with_host=False):
    dims, fidx = W.batched_shapes(count, salt=seed)
    rng = np.random.default_rng(seed)
    A, B, descs = [], [], []
    oa = ob = oc = 0
    offs = []
    for (m, n, K), fi in zip(dims, fidx):
        m, n, K, f = int(m), int(n), int(K), fields[int(fi)]
        A.append(rng.integers(0, f.p, f.k * m * K, dtype=np.uint8))
        B.append(rng.integers(0, f.p, f.k * K * n, dtype=np.uint8))
        offs.append((oa, ob, oc))
        oa, ob, oc = oa + A[-1].size, ob + B[-1].size, oc + f.k * m * n
    dA = torch.from_numpy(np.concatenate(A)).cuda()
    dB = torch.from_numpy(np.concatenate(B)).cuda()
    dC = torch.zeros(oc, dtype=torch.uint8, device="cuda")
    for (m, n, K), fi, (a, b, c) in zip(dims, fidx, offs):
        descs.append(q.GemmDesc(int(fi), int(m), int(n), int(K), dA.data_ptr() + a,
                                dB.data_ptr() + b, dC.data_ptr() + c, int(K), int(n), int(n), 0))
    if with_host:
        return dA, dB, dC, descs, (dims, fidx, A, B, offs)
    return dA, dB, dC, descs


def _reference(torch, fields, descs, dC):
    ws = torch.empty(q.batched_workspace_size(descs), dtype=torch.uint8, device="cuda")
    q.batched_gemm(fields, descs, ws)
    torch.cuda.synchronize()
    return dC.clone()


def _call_noalloc(fields, descs, stream):
    lib = q.lib()
    arr = (q.GemmDesc * len(descs))(*descs)
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    return lib.qadic_batched_gemm_noalloc(hs, len(fields), arr, len(descs),
                                          ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_workspace_version_twice():
    import torch
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    fields = [q.Field(2, 8), q.Field(7, 4), q.Field(31, 2)]
    dA, dB, dC, descs = _batch(torch, fields, 96, seed=21)
    ws = torch.empty(q.batched_workspace_size(descs), dtype=torch.uint8, device="cuda")
    q.batched_gemm(fields, descs, ws)
    torch.cuda.synchronize()
    want = dC.clone()
    # integer results: the tolerance is zero
    for _ in range(2):
        dC.fill_(255)
        assert _call_noalloc(fields, descs, stream) == q.OK
        torch.cuda.synchronize()
        assert torch.equal(dC, want)
    # a different batch through the same fixed array right after
    dA2, dB2, dC2, descs2 = _batch(torch, fields, 40, seed=22)
    ws2 = torch.empty(q.batched_workspace_size(descs2), dtype=torch.uint8, device="cuda")
    q.batched_gemm(fields, descs2, ws2)
    torch.cuda.synchronize()
    want2 = dC2.clone()
    dC2.fill_(255)
    assert _call_noalloc(fields, descs2, stream) == q.OK
    torch.cuda.synchronize()
    assert torch.equal(dC2, want2)
    q.sync_status()


def test_noalloc_back_to_back_without_sync():
    """Two different batches on one stream, no synchronisation between the
    calls: the second call rewrites the shared host array only after the
    first call's upload has read it, so both results are right."""
    import torch
    stream = torch.cuda.current_stream()
    fields = [q.Field(2, 8), q.Field(7, 4), q.Field(31, 2)]
    dA, dB, dC, descs = _batch(torch, fields, 64, seed=21)
    dA2, dB2, dC2, descs2 = _batch(torch, fields, 48, seed=22)
    want = _reference(torch, fields, descs, dC)
    want2 = _reference(torch, fields, descs2, dC2)
    for _ in range(2):
        dC.fill_(255)
        dC2.fill_(255)
        torch.cuda.synchronize()
        assert _call_noalloc(fields, descs, stream) == q.OK
        assert _call_noalloc(fields, descs2, stream) == q.OK
        torch.cuda.synchronize()
        assert torch.equal(dC, want)
        assert torch.equal(dC2, want2)
    q.sync_status()


def test_noalloc_matches_oracle(orc):
    import torch
    stream = torch.cuda.current_stream()
    fields = [q.Field(2, 8), q.Field(7, 4), q.Field(31, 2)]
    dA, dB, dC, descs, (dims, fidx, A, B, offs) = _batch(torch, fields, 9, seed=23,
                                                          with_host=True)
    dC.fill_(255)
    assert _call_noalloc(fields, descs, stream) == q.OK
    torch.cuda.synchronize()
    q.sync_status()
    got = dC.cpu().numpy()
    for (m, n, K), fi, a, b, (_, _, c) in zip(dims, fidx, A, B, offs):
        m, n, K, f = int(m), int(n), int(K), fields[int(fi)]
        Ai = np.transpose(a.reshape(f.k, m, K), (1, 2, 0))
        Bi = np.transpose(b.reshape(f.k, K, n), (1, 2, 0))
        want = np.transpose(orc.gemm(f.p, f.poly, Ai, Bi), (2, 0, 1))
        assert np.array_equal(got[c:c + f.k * m * n].reshape(f.k, m, n), want), (m, n, K, f.p)


def test_noalloc_rejects_work_list_beyond_fixed_array():
    import torch
    stream = torch.cuda.current_stream()
    f = q.Field(31, 2)
    m = n = 4096
    K = 16
    # Every descriptor stays inside its buffers, so even a launch would read
    # and write only memory it owns: A holds k*m*K bytes, B k*K*n, C k*m*n
    # (shared by all descriptors).  The size check counts tiles of the
    # smallest shape, 32 x 16: 40 products of 4096 x 4096 give 40 * 128 * 256
    # tiles of 8 bytes > 8 MiB, so the list is refused before anything is
    # uploaded or launched.
    A = torch.zeros(f.k * m * K, dtype=torch.uint8, device="cuda")
    B = torch.zeros(f.k * K * n, dtype=torch.uint8, device="cuda")
    C = torch.zeros(f.k * m * n, dtype=torch.uint8, device="cuda")
    big = [q.GemmDesc(0, m, n, K, A.data_ptr(), B.data_ptr(), C.data_ptr(), K, n, n, 0)
           for _ in range(40)]
    assert _call_noalloc([f], big, stream) == q.E_INVALID
    assert b"fixed scratch" in q.lib().qadic_last_error()
    torch.cuda.synchronize()
    assert int(C.sum()) == 0
