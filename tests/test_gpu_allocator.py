"""The device-allocator hook on a GPU: a field whose tables come from torch's
caching allocator computes the same product as one built with cudaMalloc,
and every table goes back to the allocator at destroy."""
import numpy as np
import pytest

import paper_0710_0510_gb300 as q
from paper_0710_0510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_field_tables_from_torch_allocator(orc):
    import torch
    assert torch.cuda.is_available()
    live = {}

    def alloc(nbytes):
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        live[ptr] = nbytes
        return ptr

    def free(ptr, nbytes):
        assert live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)

    p, k, m, n, K = 101, 2, 130, 144, 200
    A = W.centred_planes(k, m, K, 50, salt=31)
    B = W.centred_planes(k, K, n, 50, salt=32)
    want = np.transpose(orc.gemm(p, orc.smallest_irreducible(p, k), np.transpose(A, (1, 2, 0)),
                                 np.transpose(B, (1, 2, 0))), (2, 0, 1))
    q.set_device_allocator(alloc, free)
    try:
        f = q.Field(p, k)
        assert len(live) == 6            # every device table came from the hook
    finally:
        q.set_device_allocator(None, None)
    a = f.pack(q.FMT_INT8_PLANES, torch.from_numpy(A).cuda(), m, K, q.FMT_OPERAND_A)
    b = f.pack(q.FMT_INT8_PLANES, torch.from_numpy(B).cuda(), K, n, q.FMT_OPERAND_B)
    C = f.gemm(q.PATH_PLANES, a, b, m, n, K).cpu().numpy()
    q.sync_status()
    assert np.array_equal(C, want)
    # fields built after the default came back do not use the hook
    g = q.Field(7, 4)
    assert len(live) == 6
    g.close()
    torch.cuda.synchronize()
    f.close()
    assert live == {}
