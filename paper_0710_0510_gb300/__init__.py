"""GF(p^k) matrix multiplication through the q-adic transform on GB300.

Python binding of ``libqadic.so`` (C ABI in ``include/qadic.h``).  This module
only marshals arguments: torch tensors supply device memory and the current
CUDA stream, and every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: without the built library or a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

# qadic_status
OK, E_INVALID, E_NOT_PRIME, E_REDUCIBLE, E_OVERFLOW, E_UNSUPPORTED, E_CUDA, E_DEVICE_TIMEOUT, \
    E_NOMEM = range(9)
# qadic_format
FMT_LOG, FMT_COEFF_U8, FMT_INT8_PLANES, FMT_QADIC_F64, FMT_OPERAND_A, FMT_OPERAND_B, \
    FMT_OPERAND_B_FOLD, FMT_OPERAND_A_KARA, FMT_OPERAND_B_KARA, FMT_OPERAND_A_E4M3, \
    FMT_OPERAND_B_E4M3 = range(11)
# qadic_path
PATH_FP64_QADIC, PATH_PLANES, PATH_FOLD, PATH_KARATSUBA, PATH_PLANES_E4M3 = 0, 1, 2, 3, 4
REDQ_INT_FLOOR = 0x100
REDQ_F32_DIGITS = 0x200
POLYMUL_PLAIN_F64 = 0x1
POLYMUL_INT_WORDS = 0x2
BATCHED_GRAPH = 0x1
FIELD_HOST_ONLY = 0x1
FQT_INT_WORDS = 0x1

_lock = threading.Lock()
_lib = None


def fold_n_pad(n: int) -> int:
    """Rows of one output block in a FMT_OPERAND_B_FOLD plane."""
    return (n + 255) // 256 * 256


class QadicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"qadic status {status}: {message}")
        self.status = status


class Info(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("poly", ctypes.c_uint32 * 17), ("generator", ctypes.c_uint32 * 16),
                ("order", ctypes.c_uint32), ("zero_code", ctypes.c_uint32),
                ("log_bytes", ctypes.c_uint32), ("log2_q", ctypes.c_uint32),
                ("n_q", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("k_max_int32", ctypes.c_int64), ("k_chunk_f32", ctypes.c_int64)]


class GemmDesc(ctypes.Structure):
    _fields_ = [("field", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("K", ctypes.c_int32), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("lda", ctypes.c_int32), ("ldb", ctypes.c_int32),
                ("ldc", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TileConfig(ctypes.Structure):
    _fields_ = [("bm", ctypes.c_int32), ("bn", ctypes.c_int32), ("bk", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32)]


class FqtInfo(ctypes.Structure):
    _fields_ = [("log2_q", ctypes.c_uint32), ("n_q", ctypes.c_uint32), ("D_q", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32), ("word_products", ctypes.c_uint64)]


# qadic_set_device_allocator callbacks: alloc(&ptr, bytes, ctx) -> status, free(ptr, bytes, ctx)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                            ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_SIGS = {
    "qadic_set_device_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, ctypes.c_void_p]),
    "qadic_field_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32]),
    "qadic_field_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "qadic_field_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Info)]),
    "qadic_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_void_p]),
    "qadic_gemm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_void_p]),
    "qadic_pack_operands": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p]),
    "qadic_pack_operands_e4m3": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_int64, ctypes.c_void_p]),
    "qadic_matmul_device_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int,
                                                             ctypes.c_int64, ctypes.c_int64,
                                                             ctypes.c_int64]),
    "qadic_matmul": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p]),
    "qadic_matmul_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int64, ctypes.c_int64,
                                                      ctypes.c_int64]),
    "qadic_matmul_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "qadic_redq": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_void_p]),
    "qadic_redq_pq": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_uint32, ctypes.c_void_p]),
    "qadic_polymul_fqt_info": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.POINTER(FqtInfo)]),
    "qadic_polymul_fqt": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p]),
    "qadic_batched_tile_configs": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(TileConfig),
                                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "qadic_batched_select_tiles": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int32]),
    "qadic_batched_selected_tiles": (ctypes.c_int, [ctypes.c_uint32,
                                                    ctypes.POINTER(ctypes.c_int32)]),
    "qadic_batched_autotune": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                              ctypes.POINTER(GemmDesc), ctypes.c_int64,
                                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "qadic_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_void_p]),
    "qadic_polymul_batched": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_uint32, ctypes.c_void_p]),
    "qadic_batched_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(GemmDesc), ctypes.c_int64]),
    "qadic_batched_workspace_size_fields": (ctypes.c_size_t, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                                              ctypes.POINTER(GemmDesc), ctypes.c_int64]),
    "qadic_batched_gemm": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                          ctypes.POINTER(GemmDesc), ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                          ctypes.c_void_p]),
    "qadic_batched_gemm_noalloc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                                  ctypes.POINTER(GemmDesc), ctypes.c_int64,
                                                  ctypes.c_void_p]),
    "qadic_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "qadic_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qadic_last_error": (ctypes.c_char_p, []),
}


def lib(load: bool = True):
    """The loaded ``libqadic.so`` (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None and load:
            path = _build.build()
            handle = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(status: int):
    if status != OK:
        msg = lib().qadic_last_error().decode(errors="replace")
        raise QadicError(status, msg)


_TORCH_CUDA = None   # torch, once a CUDA device has been seen (checked once per process)


def _torch():
    global _TORCH_CUDA
    if _TORCH_CUDA is None:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: libqadic has no CPU path")
        _TORCH_CUDA = torch
    return _TORCH_CUDA


_RAW_STREAM = None


def _stream(stream=None):
    """The CUDA stream handle to pass: `stream`'s, else the current one (read
    as a raw handle where torch exposes it, which skips building a Stream
    object on every call)."""
    global _RAW_STREAM
    torch = _torch()
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    if _RAW_STREAM is None:
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        dev = getattr(torch._C, "_cuda_getDevice", None)
        _RAW_STREAM = (lambda: raw(dev())) if raw is not None and dev is not None else False
    if _RAW_STREAM:
        return ctypes.c_void_p(_RAW_STREAM())
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Field:
    """GF(p^k) on the current CUDA device (``qadic_field_init``)."""

    def __init__(self, p: int, k: int, poly=None, host_only: bool = False):
        if not host_only:
            _torch()
        L = lib()
        h = ctypes.c_void_p()
        arr = None
        if poly is not None:
            arr = (ctypes.c_uint32 * len(poly))(*poly)
        _check(L.qadic_field_init(ctypes.byref(h), p, k,
                                  ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None,
                                  FIELD_HOST_ONLY if host_only else 0))
        self._h = h
        info = Info()
        _check(L.qadic_field_info(h, ctypes.byref(info)))
        self.p, self.k = info.p, info.k
        self.poly = [info.poly[i] for i in range(self.k + 1)]
        self.generator = [info.generator[i] for i in range(self.k)]
        self.order = info.order
        self.zero_code = info.zero_code
        self.log_bytes = info.log_bytes
        self.log2_q = info.log2_q
        self.n_q = info.n_q
        self.k_max_int32 = info.k_max_int32
        self.k_chunk_f32 = info.k_chunk_f32

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qadic_field_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def pack(self, in_fmt: int, x, rows: int, cols: int, out_fmt: int, out=None, ld_in=None,
             ld_out=None, stream=None):
        """DQT pack (``qadic_pack``).  Allocates ``out`` when not given."""
        torch = _torch()
        if out is None:
            if out_fmt == FMT_QADIC_F64:
                out = torch.empty((rows, cols), dtype=torch.float64, device=x.device)
            elif out_fmt == FMT_OPERAND_A:
                out = torch.empty((self.k, rows, cols), dtype=torch.bfloat16, device=x.device)
            elif out_fmt == FMT_OPERAND_B:
                out = torch.empty((self.k, cols, rows), dtype=torch.bfloat16, device=x.device)
            elif out_fmt == FMT_COEFF_U8:
                out = torch.empty((self.k, rows, cols), dtype=torch.uint8, device=x.device)
            elif out_fmt == FMT_OPERAND_A_KARA:
                out = torch.empty((3, rows, cols), dtype=torch.bfloat16, device=x.device)
            elif out_fmt == FMT_OPERAND_B_KARA:
                out = torch.empty((3, cols, rows), dtype=torch.bfloat16, device=x.device)
            elif out_fmt == FMT_OPERAND_A_E4M3:
                out = torch.empty((self.k, rows, cols), dtype=torch.uint8, device=x.device)
            elif out_fmt == FMT_OPERAND_B_E4M3:
                out = torch.empty((self.k, cols, rows), dtype=torch.uint8, device=x.device)
            elif out_fmt == FMT_OPERAND_B_FOLD:
                out = torch.empty((self.k, self.k * fold_n_pad(cols), (rows + 7) // 8 * 8),
                                  dtype=torch.bfloat16, device=x.device)
            else:
                raise ValueError("unsupported output format")
        if ld_in is None:
            ld_in = cols
        if ld_out is None:
            if out_fmt == FMT_OPERAND_B_FOLD:
                ld_out = out.shape[-1]
            else:
                ld_out = rows if out_fmt in (FMT_OPERAND_B, FMT_OPERAND_B_KARA,
                                             FMT_OPERAND_B_E4M3) else cols
        _check(lib().qadic_pack(self._h, in_fmt, _ptr(x), rows, cols, ld_in, out_fmt, _ptr(out),
                                ld_out, _stream(stream)))
        return out

    def gemm(self, path: int, A, B, m: int, n: int, K: int, C=None, lda=None, ldb=None,
             ldc=None, stream=None):
        """C = A B over GF(p^k) (``qadic_gemm``); C: (k, m, n) uint8."""
        torch = _torch()
        if C is None:
            C = torch.empty((self.k, m, n), dtype=torch.uint8, device=A.device)
        if lda is None:
            lda = K
        if ldb is None:
            ldb = n if path == PATH_FP64_QADIC else (B.shape[-1] if path == PATH_FOLD else K)
        if ldc is None:
            ldc = n
        _check(lib().qadic_gemm(self._h, path, m, n, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc,
                                None, 0, _stream(stream)))
        return C

    def pack_operands(self, in_fmt: int, A, B, m: int, n: int, K: int, outA, outB,
                      lda_in=None, ldb_in=None, lda_out=None, ldb_out=None, stream=None,
                      e4m3: bool = False):
        """A -> OPERAND_A and B -> OPERAND_B in one call (``qadic_pack_operands``);
        with e4m3, the E4M3 operand formats (``qadic_pack_operands_e4m3``)."""
        fn = lib().qadic_pack_operands_e4m3 if e4m3 else lib().qadic_pack_operands
        _check(fn(
            self._h, in_fmt, _ptr(A), m, K, K if lda_in is None else lda_in, _ptr(outA),
            outA.shape[-1] if lda_out is None else lda_out, _ptr(B), n,
            n if ldb_in is None else ldb_in, _ptr(outB),
            outB.shape[-1] if ldb_out is None else ldb_out, _stream(stream)))
        return outA, outB

    def matmul_device_workspace_size(self, path: int, m: int, n: int, K: int) -> int:
        return int(lib().qadic_matmul_device_workspace_size(self._h, path, m, n, K))

    def matmul(self, path: int, in_fmt: int, A, B, m: int, n: int, K: int, workspace, C=None,
               lda=None, ldb=None, ldc=None, stream=None):
        """Pack + GEMM on device operands in one call (``qadic_matmul``)."""
        torch = _torch()
        if C is None:
            C = torch.empty((self.k, m, n), dtype=torch.uint8, device=A.device)
        _check(lib().qadic_matmul(self._h, path, in_fmt, m, n, K, _ptr(A),
                                  K if lda is None else lda, _ptr(B), n if ldb is None else ldb,
                                  _ptr(C), n if ldc is None else ldc, _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)))
        return C

    def matmul_workspace_size(self, path: int, in_fmt: int, m: int, n: int, K: int) -> int:
        return int(lib().qadic_matmul_workspace_size(self._h, path, in_fmt, m, n, K))

    def matmul_host(self, path: int, in_fmt: int, A_host, B_host, C_host, m: int, n: int, K: int,
                    workspace, stream=None):
        """End to end from host buffers (``qadic_matmul_host``)."""
        _check(lib().qadic_matmul_host(self._h, path, in_fmt, m, n, K, _ptr(A_host), _ptr(B_host),
                                       _ptr(C_host), _ptr(workspace), workspace.numel(),
                                       _stream(stream)))
        return C_host


def redq(p: int, log2_q: int, ndigits: int, words, out=None, table_mode: int = 3,
         int_floor: bool = False, stream=None):
    """REDQ over packed FP64 words (``qadic_redq``)."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(words)
    mode = table_mode | (REDQ_INT_FLOOR if int_floor else 0)
    _check(lib().qadic_redq(p, log2_q, ndigits, _ptr(words), _ptr(out), words.numel(), mode,
                            _stream(stream)))
    return out


def redq_pq(p: int, q: int, ndigits: int, words, out=None, int_floor: bool = False,
            stream=None, f32_digits: bool = False):
    """REDQ for q a multiple of p, no correction step (``qadic_redq_pq``);
    ``f32_digits`` selects QADIC_REDQ_F32_DIGITS."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(words)
    flags = (REDQ_INT_FLOOR if int_floor else 0) | (REDQ_F32_DIGITS if f32_digits else 0)
    _check(lib().qadic_redq_pq(p, q, ndigits, _ptr(words), _ptr(out), words.numel(),
                               flags, _stream(stream)))
    return out


def polymul_fqt_info(p: int, N: int, d: int, int_words: bool = False) -> FqtInfo:
    """Parameters of the d-FQT product (``qadic_polymul_fqt_info``, host only)."""
    info = FqtInfo()
    _check(lib().qadic_polymul_fqt_info(p, N, d, FQT_INT_WORDS if int_words else 0,
                                        ctypes.byref(info)))
    return info


def polymul_fqt(p: int, d: int, a, b, out=None, int_words: bool = False, stream=None):
    """Long polynomial products by the d-FQT (``qadic_polymul_fqt``);
    a, b: (count, N+1) uint8, returns (count, 2N+1) uint8."""
    torch = _torch()
    count, n1 = a.shape
    if out is None:
        out = torch.empty((count, 2 * n1 - 1), dtype=torch.uint8, device=a.device)
    _check(lib().qadic_polymul_fqt(p, n1 - 1, d, _ptr(a), _ptr(b), _ptr(out), count,
                                   FQT_INT_WORDS if int_words else 0, _stream(stream)))
    return out


def polymul_batched(p: int, k: int, a, b, out=None, plain_f64: bool = False,
                    int_words: bool = False, stream=None):
    """Batched Alg. 1 + Alg. 2 (``qadic_polymul_batched``); a, b: (count, k) uint8."""
    torch = _torch()
    count = a.shape[0]
    if out is None:
        out = torch.empty((count, 2 * k - 1), dtype=torch.uint8, device=a.device)
    _check(lib().qadic_polymul_batched(p, k, _ptr(a), _ptr(b), _ptr(out), count,
                                       (POLYMUL_PLAIN_F64 if plain_f64 else 0) |
                                       (POLYMUL_INT_WORDS if int_words else 0), _stream(stream)))
    return out


def desc_array(descs):
    """The descriptors as the ctypes array the C calls take; a caller that
    launches the same batch repeatedly can build it once and pass it instead
    of the list (building it costs about 0.2 us per descriptor)."""
    if isinstance(descs, ctypes.Array):
        return descs
    return (GemmDesc * len(descs))(*descs)


def batched_workspace_size(descs, fields=None) -> int:
    """Workspace bytes of ``batched_gemm``: with ``fields``, room for the
    converted operands too (``qadic_batched_workspace_size_fields``, the
    faster path); without, the work list alone (operands staged through
    registers)."""
    arr = desc_array(descs)
    if fields is None:
        return int(lib().qadic_batched_workspace_size(arr, len(descs)))
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    n = int(lib().qadic_batched_workspace_size_fields(hs, len(fields), arr, len(descs)))
    if n == 0:
        raise QadicError(1, "batched_workspace_size: invalid fields or descriptors")
    return n


def batched_gemm(fields, descs, workspace, graph: bool = False, stream=None):
    """Many independent products in one persistent launch (``qadic_batched_gemm``)."""
    arr = desc_array(descs)
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    _check(lib().qadic_batched_gemm(hs, len(fields), arr, len(descs), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(),
                                    BATCHED_GRAPH if graph else 0, _stream(stream)))


def batched_tile_configs(k: int):
    """The batched kernel's tile configurations for degree k
    (``qadic_batched_tile_configs``): list of (bm, bn, bk, smem_bytes)."""
    n = ctypes.c_int32()
    arr = (TileConfig * 8)()
    _check(lib().qadic_batched_tile_configs(k, arr, 8, ctypes.byref(n)))
    return [(c.bm, c.bn, c.bk, c.smem_bytes) for c in arr[:n.value]]


def batched_select_tiles(k: int, index: int):
    _check(lib().qadic_batched_select_tiles(k, index))


def batched_selected_tiles(k: int) -> int:
    i = ctypes.c_int32()
    _check(lib().qadic_batched_selected_tiles(k, ctypes.byref(i)))
    return i.value


def batched_autotune(fields, descs, workspace, reps: int = 3, stream=None):
    """Time every tile configuration on this batch and keep the fastest per k
    (``qadic_batched_autotune``); returns {k: chosen index}."""
    arr = desc_array(descs)
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    chosen = (ctypes.c_int32 * 9)()
    _check(lib().qadic_batched_autotune(hs, len(fields), arr, len(descs), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), reps,
                                        chosen, _stream(stream)))
    return {k: chosen[k] for k in range(9) if chosen[k] >= 0}


def batched_gemm_noalloc(fields, descs, stream=None):
    """Same products as batched_gemm without any allocation
    (``qadic_batched_gemm_noalloc``: fixed library-owned scratch, calls that
    overlap on the GPU race)."""
    arr = desc_array(descs)
    hs = (ctypes.c_void_p * len(fields))(*[f.handle for f in fields])
    _check(lib().qadic_batched_gemm_noalloc(hs, len(fields), arr, len(descs), _stream(stream)))


# Every callback pair ever installed stays alive for the life of the process:
# a field built while a pair was installed calls that pair's free at destroy,
# possibly long after another allocator (or the default) replaced it.
_ALLOCATOR_REFS = []


def set_device_allocator(alloc=None, free=None):
    """Install the device allocator for field tables (``qadic_set_device_allocator``):
    ``alloc(bytes) -> int`` returns a device address (0 for out of memory),
    ``free(ptr, bytes)`` releases one; both None restores cudaMalloc/cudaFree."""
    if alloc is None and free is None:
        _check(lib().qadic_set_device_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def c_alloc(out, nbytes, ctx):
        try:
            ptr = int(alloc(int(nbytes)) or 0)
        except MemoryError:
            ptr = 0
        out[0] = ptr or None
        return OK if ptr else E_NOMEM

    def c_free(ptr, nbytes, ctx):
        free(int(ptr or 0), int(nbytes))

    refs = (ALLOC_FN(c_alloc), FREE_FN(c_free))
    _ALLOCATOR_REFS.append(refs)
    _check(lib().qadic_set_device_allocator(refs[0], refs[1], None))


def selftest_bounded_wait(polls: int, stream=None):
    """Let a bounded device wait run out on purpose (``qadic_selftest_bounded_wait``):
    the next sync_status() raises QadicError with E_DEVICE_TIMEOUT."""
    _check(lib().qadic_selftest_bounded_wait(polls, _stream(stream)))


def sync_status(stream=None):
    _check(lib().qadic_sync_status(_stream(stream)))
