"""Failure paths that are decided on the host, before anything reaches a GPU:
allocation failure injected through the device-allocator hook, and batched
work lists that the work queue cannot index.  CPU only: every call here must
return its status without a CUDA launch (on a machine with no GPU, reaching
a CUDA call would turn the status into QADIC_E_CUDA instead)."""
import ctypes

import pytest

import paper_0710_0510_gb300 as q


def _cuda_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# The fake allocator below hands out addresses that are not device memory; on
# a machine with a GPU the library would go on to copy tables to them, so
# these host-only checks run only where no CUDA device exists.
pytestmark = pytest.mark.skipif(_cuda_present(), reason="host-only checks: no CUDA device allowed")


class CountingAllocator:
    """Hands out fake, never-dereferenced addresses, failing from call `fail_at` on."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.freed = []

    def alloc(self, nbytes):
        self.calls += 1
        if self.fail_at is not None and self.calls >= self.fail_at:
            return 0
        ptr = 0x10000000 * self.calls
        self.live[ptr] = nbytes
        return ptr

    def free(self, ptr, nbytes):
        assert self.live.pop(ptr) == nbytes
        self.freed.append(ptr)


@pytest.fixture
def allocator():
    made = []

    def make(fail_at=None):
        a = CountingAllocator(fail_at)
        q.set_device_allocator(a.alloc, a.free)
        made.append(a)
        return a

    yield make
    q.set_device_allocator(None, None)


def _init(p, k, flags=0):
    h = ctypes.c_void_p()
    st = q.lib().qadic_field_init(ctypes.byref(h), p, k, None, flags)
    return st, h


@pytest.mark.parametrize("fail_at", [1, 2, 4, 6])
def test_allocation_failure_returns_nomem_and_frees_earlier_tables(allocator, fail_at):
    a = allocator(fail_at)
    st, h = _init(3, 3)
    assert st == q.E_NOMEM
    assert not h.value
    assert b"device allocation" in q.lib().qadic_last_error()
    # every table obtained before the failing one went back through the hook
    assert a.calls == fail_at and a.live == {} and len(a.freed) == fail_at - 1


def test_allocator_cuda_error_is_passed_through(allocator):
    seen = []

    def alloc_cb(out, nbytes, ctx):
        seen.append(nbytes)
        return q.E_CUDA

    def free_cb(ptr, nbytes, ctx):
        raise AssertionError("nothing was allocated")

    refs = (q.ALLOC_FN(alloc_cb), q.FREE_FN(free_cb))
    q._ALLOCATOR_REFS.append(refs)     # outlives every field built with it
    assert q.lib().qadic_set_device_allocator(refs[0], refs[1], None) == q.OK
    st, h = _init(101, 2)
    assert st == q.E_CUDA and len(seen) == 1


def test_all_tables_come_from_the_hook(allocator):
    """Every table allocated through the hook and none leaked: with no GPU
    the upload after the allocations fails (QADIC_E_CUDA) and all six tables
    are handed back (a real allocator is tested under -m gpu)."""
    a = allocator()
    st, h = _init(7, 4)
    assert st == q.E_CUDA
    assert a.calls == 6 and a.live == {} and len(a.freed) == 6


def test_host_only_fields_never_touch_the_allocator(allocator):
    a = allocator(fail_at=1)
    st, h = _init(31, 2, q.FIELD_HOST_ONLY)
    assert st == q.OK and a.calls == 0
    assert q.lib().qadic_field_destroy(h) == q.OK


def test_allocator_arguments_checked():
    L = q.lib()
    assert L.qadic_set_device_allocator(q.ALLOC_FN(lambda o, n, c: 0), q.FREE_FN(), None) == \
        q.E_INVALID
    assert L.qadic_set_device_allocator(q.ALLOC_FN(), q.FREE_FN(), None) == q.OK


def _host_fields():
    return [q.Field(2, 8, host_only=True), q.Field(31, 2, host_only=True)]


def _call_batched(fields, descs, ws_ptr=None, ws_bytes=0):
    arr = (q.GemmDesc * len(descs))(*descs)
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    return q.lib().qadic_batched_gemm(hs, len(fields), arr, len(descs), ctypes.c_void_p(ws_ptr),
                                      ws_bytes, 0, None)


def _call_noalloc(fields, descs):
    arr = (q.GemmDesc * len(descs))(*descs)
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    return q.lib().qadic_batched_gemm_noalloc(hs, len(fields), arr, len(descs), None)


def test_batched_queue_refuses_lists_it_cannot_index():
    """4200 products of 4096 x 4096 make 4200 * 32768 tiles of the smallest
    shape (> 2^27): refused as QADIC_E_INVALID by both batched entry points,
    before the workspace is looked at."""
    fields = _host_fields()
    big = [q.GemmDesc(i % 2, 4096, 4096, 16, 256, 256, 256, 16, 4096, 4096, 0)
           for i in range(4200)]
    assert _call_batched(fields, big) == q.E_INVALID
    assert b"work queue" in q.lib().qadic_last_error()
    assert _call_noalloc(fields, big) == q.E_INVALID
    assert b"work queue" in q.lib().qadic_last_error()


def test_batched_impossible_descriptors_refused():
    fields = _host_fields()
    ok = dict(field=0, m=8, n=8, K=8, A=256, B=256, C=256, lda=8, ldb=8, ldc=8, reserved=0)
    cases = [
        dict(ok, field=2),                 # no such field
        dict(ok, field=-1),
        dict(ok, m=0), dict(ok, n=4097), dict(ok, K=-3),
        dict(ok, A=0), dict(ok, C=0),
        dict(ok, lda=7), dict(ok, ldb=7), dict(ok, ldc=7),
    ]
    for c in cases:
        d = q.GemmDesc(*[c[f] for f, _ in q.GemmDesc._fields_])
        assert _call_batched(fields, [q.GemmDesc(**ok), d]) == q.E_INVALID, c
        assert _call_noalloc(fields, [d]) == q.E_INVALID, c


def test_batched_short_workspace_is_nomem():
    fields = _host_fields()
    d = [q.GemmDesc(1, 64, 64, 64, 256, 256, 256, 64, 64, 64, 0)]
    need = q.batched_workspace_size(d)
    assert _call_batched(fields, d, 256, need - 1) == q.E_NOMEM
    assert _call_batched(fields, d, None, 0) == q.E_NOMEM
    assert b"workspace" in q.lib().qadic_last_error()
    assert _call_batched(fields, d, 256 + 16, need) == q.E_INVALID    # not 256-byte aligned


def test_matmul_host_short_workspace_is_nomem():
    f = q.Field(101, 2, host_only=True)
    L = q.lib()
    need = L.qadic_matmul_workspace_size(f.handle, q.PATH_PLANES, q.FMT_INT8_PLANES, 64, 64, 64)
    assert need > 0
    buf = ctypes.create_string_buffer(16)
    st = L.qadic_matmul_host(f.handle, q.PATH_PLANES, q.FMT_INT8_PLANES, 64, 64, 64, buf, buf, buf,
                             ctypes.c_void_p(256), need - 1, None)
    assert st == q.E_NOMEM
