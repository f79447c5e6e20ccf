"""The allocation-free batched entry point (qadic_batched_gemm_noalloc).

It exists for callers that cannot allocate during a call -- a framework
whose allocator owns every byte of device memory, a loop where a
cudaMalloc/cudaFree would synchronise the device, a plugin that is handed
only its inputs and outputs.  It keeps its work list in a fixed array inside
the library.  This file checks, through the C ABI, that it returns exactly
what qadic_batched_gemm (the workspace version) returns, on two calls in a
row, and that a work list too large for the fixed array is refused.

The file name makes pytest collect it last, so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_0710_0510_gb300 as q
from paper_0710_0510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(torch, fields, count, seed):
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
    return dA, dB, dC, descs


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


def test_noalloc_rejects_work_list_beyond_fixed_array():
    import torch
    stream = torch.cuda.current_stream()
    f = q.Field(31, 2)
    x = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    # 40 products of 4096 x 4096 -> 40 * 128 * 256 tiles of 8 bytes > 8 MiB;
    # refused before anything is read or launched
    big = [q.GemmDesc(0, 4096, 4096, 4096, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                      4096, 4096, 4096, 0) for _ in range(40)]
    assert _call_noalloc([f], big, stream) == q.E_INVALID
    assert b"fixed scratch" in q.lib().qadic_last_error()
