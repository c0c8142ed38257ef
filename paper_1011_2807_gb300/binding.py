"""Thin ctypes binding of libknnjoin.so (include/knn_join.h).

Marshalling only: every step of the join runs in the library's CUDA kernels.  The
names match the C entry points.  PyTorch provides device memory (outputs, and the
library's own buffers through the allocator hook) and streams.

A CSR argument is either a host CSR (numpy ``indptr``/``indices``/``values``, e.g.
:class:`paper_1011_2807_gb300.synth.CSR`) or a :class:`DeviceCSR` of CUDA tensors.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libknnjoin.so")

KNN_OK, KNN_EINVAL, KNN_ENOMEM, KNN_ECUDA, KNN_ETIMEOUT, KNN_EUNSUPPORTED = range(6)
KNN_U8, KNN_F32 = 0, 1
KNN_MODE_IIIB, KNN_MODE_IIB, KNN_MODE_BF = 0, 1, 2
_MODES = {"iiib": KNN_MODE_IIIB, "iib": KNN_MODE_IIB, "bf": KNN_MODE_BF}


def _mode(mode: str) -> int:
    try:
        return _MODES[mode]
    except KeyError:
        raise ValueError(f"mode must be one of {sorted(_MODES)}") from None
KNN_MAX_K = 64


class KnnError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"knn status {status}: {message}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("dim", ctypes.c_int32), ("dtype", ctypes.c_int),
                ("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class _BuildOpts(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("n_levels", ctypes.c_int32)]


class _IndexInfo(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("dim", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("dtype", ctypes.c_int),
                ("max_row_nnz", ctypes.c_int32), ("device_bytes", ctypes.c_size_t),
                ("host_bytes", ctypes.c_size_t)]


class _JoinOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("threads", ctypes.c_int32), ("s_groups", ctypes.c_int32),
                ("init_threshold", ctypes.c_void_p), ("n_found", ctypes.c_void_p),
                ("postings_scanned", ctypes.c_void_p), ("outputs_on_host", ctypes.c_int32),
                ("skip_validation", ctypes.c_int32), ("level_margin", ctypes.c_float),
                ("stats", ctypes.c_void_p), ("blocks_per_launch", ctypes.c_int32),
                ("no_fixed_point", ctypes.c_int32)]

KNN_STATS = ("block_steps", "candidates", "completed", "pushed", "merges", "rounds",
             "residual_features", "postings", "shared_adds", "fixed_point_rows")


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None
_alloc_cbs = None


_last_alloc_error = ""


def _torch_alloc(nbytes, stream, ctx):
    global _last_alloc_error
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception as e:   # reported by the library as KNN_ENOMEM
        _last_alloc_error = repr(e)
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    torch.cuda.caching_allocator_delete(int(ptr))


def lib():
    """Loads libknnjoin.so; raises if it was not built (there is no CPU fallback)."""
    global _lib, _alloc_cbs
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.knn_last_error.restype = ctypes.c_char_p
        L.knn_version.restype = ctypes.c_char_p
        L.knn_kernel_launch_count.restype = ctypes.c_int64
        L.knn_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]
        L.knn_join_build_index.argtypes = [P(_Csr), P(_BuildOpts), ctypes.c_void_p, P(ctypes.c_void_p)]
        L.knn_index_get_info.argtypes = [ctypes.c_void_p, P(_IndexInfo)]
        L.knn_index_destroy.argtypes = [ctypes.c_void_p]
        L.knn_index_destroy.restype = None
        L.knn_index_to_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.knn_join.argtypes = [ctypes.c_void_p, P(_Csr), ctypes.c_int32, P(_JoinOpts),
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.knn_join_noalloc.argtypes = [ctypes.c_void_p, P(_Csr), ctypes.c_int32, P(_JoinOpts),
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _alloc_cbs = (_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free))
        _check(L, L.knn_set_allocator(_alloc_cbs[0], _alloc_cbs[1], None))
        _lib = L
        return L


def _check(L, status):
    if status != KNN_OK:
        msg = L.knn_last_error().decode()
        if status == KNN_ENOMEM and _last_alloc_error:
            msg += f" (allocator: {_last_alloc_error})"
        raise KnnError(status, msg)


def knn_last_error() -> str:
    return lib().knn_last_error().decode()


def knn_version() -> str:
    return lib().knn_version().decode()


def knn_kernel_launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().knn_kernel_launch_count())


# ----------------------------------------------------------------------------------
# CSR marshalling
# ----------------------------------------------------------------------------------

@dataclasses.dataclass
class DeviceCSR:
    """CSR held in CUDA tensors (int64 indptr, int32 indices, uint8/float32 values)."""

    indptr: torch.Tensor
    indices: torch.Tensor
    values: torch.Tensor
    dim: int

    @property
    def n_rows(self) -> int:
        return int(self.indptr.shape[0] - 1)

    @staticmethod
    def from_host(x, device="cuda") -> "DeviceCSR":
        return DeviceCSR(torch.from_numpy(np.ascontiguousarray(x.indptr, np.int64)).to(device),
                         torch.from_numpy(np.ascontiguousarray(x.indices, np.int32)).to(device),
                         torch.from_numpy(np.ascontiguousarray(x.values)).to(device), int(x.dim))


def _dtype_code(vdtype) -> int:
    if vdtype in (np.uint8, torch.uint8):
        return KNN_U8
    if vdtype in (np.float32, torch.float32):
        return KNN_F32
    raise TypeError(f"values must be uint8 or float32, got {vdtype}")


def _csr(x, keep: list) -> _Csr:
    if isinstance(x, DeviceCSR):
        for t, dt in ((x.indptr, torch.int64), (x.indices, torch.int32)):
            if t.dtype != dt or not t.is_contiguous():
                raise TypeError("DeviceCSR needs contiguous int64 indptr and int32 indices")
        if not x.values.is_contiguous():
            raise TypeError("values must be contiguous")
        on_dev = int(x.indptr.is_cuda)
        keep.append(x)
        return _Csr(x.n_rows, int(x.dim), _dtype_code(x.values.dtype), x.indptr.data_ptr(),
                    x.indices.data_ptr(), x.values.data_ptr(), on_dev)
    indptr = np.ascontiguousarray(x.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(x.indices, dtype=np.int32)
    values = np.ascontiguousarray(x.values)
    keep.extend([indptr, indices, values])
    return _Csr(indptr.shape[0] - 1, int(x.dim), _dtype_code(values.dtype), indptr.ctypes.data,
                indices.ctypes.data, values.ctypes.data, 0)


def _stream_ptr(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


# ----------------------------------------------------------------------------------
# index
# ----------------------------------------------------------------------------------

class Index:
    """Owns a knn_index handle (freed on close() or garbage collection)."""

    def __init__(self, handle: int, dtype: int):
        self._h = handle
        self.dtype = dtype

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("index is closed")
        return self._h

    def to_host(self, stream=None) -> "Index":
        """Moves the index into pinned host memory (knn_index_to_host); returns self."""
        L = lib()
        _check(L, L.knn_index_to_host(self.handle, _stream_ptr(stream) if stream is not None else None))
        return self

    def info(self) -> dict:
        inf = _IndexInfo()
        L = lib()
        _check(L, L.knn_index_get_info(self.handle, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _IndexInfo._fields_}

    def close(self):
        if self._h:
            lib().knn_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def knn_join_build_index(S, block_size: int = 0, n_levels: int = 0, stream=None) -> Index:
    """Builds the index of S (see include/knn_join.h)."""
    L = lib()
    keep = []
    c = _csr(S, keep)
    opts = _BuildOpts(int(block_size), int(n_levels))
    h = ctypes.c_void_p()
    _check(L, L.knn_join_build_index(ctypes.byref(c), ctypes.byref(opts), _stream_ptr(stream),
                                     ctypes.byref(h)))
    return Index(h.value, c.dtype)


# ----------------------------------------------------------------------------------
# join
# ----------------------------------------------------------------------------------

def knn_join(index: Index, R, k: int, *, mode: str = "iiib", threads: int = 0, s_groups: int = 0,
             init_threshold: torch.Tensor | None = None, n_found: torch.Tensor | None = None,
             postings_scanned: torch.Tensor | None = None, out_ids=None, out_scores=None,
             outputs_on_host: bool = False, skip_validation: bool = False, level_margin: float = 0.0,
             stats: torch.Tensor | None = None, blocks_per_launch: int = 0, fixed_point: bool = True,
             stream=None):
    """Exact top-k of every row of R; returns (ids, scores).

    Device outputs are torch tensors on the current device unless ``out_ids`` /
    ``out_scores`` are given.  With ``outputs_on_host`` the outputs are pinned CPU
    tensors (or numpy arrays) filled by the library's device-to-host copies.
    """
    L = lib()
    keep = []
    c = _csr(R, keep)
    n = c.n_rows
    sdt = torch.int32 if index.dtype == KNN_U8 else torch.float32
    if out_ids is None:
        if outputs_on_host:
            out_ids = torch.empty((n, k), dtype=torch.int32, pin_memory=True)
            out_scores = torch.empty((n, k), dtype=sdt, pin_memory=True)
        else:
            out_ids = torch.empty((n, k), dtype=torch.int32, device="cuda")
            out_scores = torch.empty((n, k), dtype=sdt, device="cuda")
    opts = _JoinOpts(_mode(mode), int(threads), int(s_groups),
                     _ptr(init_threshold), _ptr(n_found), _ptr(postings_scanned),
                     int(bool(outputs_on_host)), int(bool(skip_validation)), float(level_margin),
                     _ptr(stats), int(blocks_per_launch), int(not fixed_point))
    ip = out_ids.ctypes.data if isinstance(out_ids, np.ndarray) else out_ids.data_ptr()
    sp = out_scores.ctypes.data if isinstance(out_scores, np.ndarray) else out_scores.data_ptr()
    _check(L, L.knn_join(index.handle, ctypes.byref(c), int(k), ctypes.byref(opts), ip, sp,
                         _stream_ptr(stream)))
    return out_ids, out_scores


def knn_join_noalloc(index: Index, R: DeviceCSR, k: int, out_ids: torch.Tensor, out_scores: torch.Tensor, *,
                     mode: str = "iiib", threads: int = 0, init_threshold: torch.Tensor | None = None,
                     n_found: torch.Tensor | None = None, skip_validation: bool = False,
                     level_margin: float = 0.0, blocks_per_launch: int = 0, stream=None):
    """knn_join without any device allocation by the library.

    For callers that cannot let a library allocate device memory during a call (a
    process that has split the GPU between its own fixed pools, or a latency-critical
    loop).  R and both outputs must already be in device memory; the library works in
    its own fixed scratch array, so n_rows * k is limited (see include/knn_join.h) and
    calls whose GPU work overlaps must be serialised by the caller.
    """
    L = lib()
    if not isinstance(R, DeviceCSR) or not R.indptr.is_cuda:
        raise TypeError("knn_join_noalloc needs a DeviceCSR on the GPU")
    keep = []
    c = _csr(R, keep)
    opts = _JoinOpts(_mode(mode), int(threads), 1,
                     _ptr(init_threshold), _ptr(n_found), None, 0, int(bool(skip_validation)),
                     float(level_margin), None, int(blocks_per_launch))
    _check(L, L.knn_join_noalloc(index.handle, ctypes.byref(c), int(k), ctypes.byref(opts),
                                 out_ids.data_ptr(), out_scores.data_ptr(), _stream_ptr(stream)))
    return out_ids, out_scores


# ----------------------------------------------------------------------------------
# learned start threshold
# ----------------------------------------------------------------------------------

class _ModelOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64)]


class _TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("quantile", ctypes.c_float), ("seed", ctypes.c_uint64)]


class _LearnedOpts(ctypes.Structure):
    _fields_ = [("join", _JoinOpts), ("tau_scale", ctypes.c_float), ("tau", ctypes.c_void_p)]


class _LearnedStats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("fallback_rows", ctypes.c_int64)]


SKETCH_WIDTH = 528   # padded sketch row (516 used)
HIDDEN = 256


def _model_lib():
    L = lib()
    if not getattr(L, "_model_ready", False):
        P = ctypes.POINTER
        L.knn_threshold_model_create.argtypes = [P(_ModelOpts), ctypes.c_void_p, P(ctypes.c_void_p)]
        L.knn_threshold_model_destroy.argtypes = [ctypes.c_void_p]
        L.knn_threshold_model_destroy.restype = None
        L.knn_threshold_model_train.argtypes = [ctypes.c_void_p, P(_Csr), ctypes.c_void_p, P(_TrainOpts),
                                                P(ctypes.c_float), ctypes.c_void_p]
        L.knn_threshold_model_predict.argtypes = [ctypes.c_void_p, P(_Csr), ctypes.c_void_p, ctypes.c_void_p]
        L.knn_threshold_model_calibrate.argtypes = [ctypes.c_void_p, P(_Csr), ctypes.c_void_p, ctypes.c_float,
                                                    P(ctypes.c_float), ctypes.c_void_p]
        L.knn_threshold_model_get_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                     P(ctypes.c_size_t)]
        L.knn_threshold_model_set_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        L.knn_join_learned.argtypes = [ctypes.c_void_p, ctypes.c_void_p, P(_Csr), ctypes.c_int32,
                                       P(_LearnedOpts), ctypes.c_void_p, ctypes.c_void_p, P(_LearnedStats),
                                       ctypes.c_void_p]
        L.knn_gemm_bf16.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_void_p]
        L.knn_threshold_sketch.argtypes = [ctypes.c_void_p, P(_Csr), ctypes.c_void_p, ctypes.c_void_p]
        L.knn_threshold_model_forward_backward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                           ctypes.c_int64, ctypes.c_float, ctypes.c_void_p,
                                                           ctypes.c_void_p, ctypes.c_void_p]
        L.knn_threshold_model_params.argtypes = [ctypes.c_void_p, P(ctypes.c_void_p), P(ctypes.c_int64)]
        L._model_ready = True
    return L


class ThresholdModel:
    """knn_model handle: sketch -> 516-256-256-1 MLP (BF16 weights) predicting log k-th score."""

    def __init__(self, seed: int = 0, stream=None):
        L = _model_lib()
        h = ctypes.c_void_p()
        _check(L, L.knn_threshold_model_create(ctypes.byref(_ModelOpts(int(seed))), _stream_ptr(stream),
                                               ctypes.byref(h)))
        self._h = h.value

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("model is closed")
        return self._h

    def train(self, Q, kth_scores: torch.Tensor, epochs: int = 0, batch: int = 0, lr: float = 0.0,
              quantile: float = 0.0, seed: int = 0, stream=None) -> float:
        L = _model_lib()
        keep = []
        c = _csr(Q, keep)
        loss = ctypes.c_float(0.0)
        o = _TrainOpts(int(epochs), int(batch), float(lr), float(quantile), int(seed))
        kth = kth_scores.contiguous().float()
        _check(L, L.knn_threshold_model_train(self.handle, ctypes.byref(c), kth.data_ptr(), ctypes.byref(o),
                                              ctypes.byref(loss), _stream_ptr(stream)))
        return float(loss.value)

    def calibrate(self, Q, kth_scores: torch.Tensor, miss_rate: float, stream=None) -> float:
        """Sets (and returns) the prediction multiplier for a target fallback rate."""
        L = _model_lib()
        keep = []
        c = _csr(Q, keep)
        kth = kth_scores.contiguous().float()
        out = ctypes.c_float(0.0)
        _check(L, L.knn_threshold_model_calibrate(self.handle, ctypes.byref(c), kth.data_ptr(), float(miss_rate),
                                                  ctypes.byref(out), _stream_ptr(stream)))
        return float(out.value)

    def predict(self, R, stream=None) -> torch.Tensor:
        L = _model_lib()
        keep = []
        c = _csr(R, keep)
        out = torch.empty(c.n_rows, dtype=torch.float32, device="cuda")
        _check(L, L.knn_threshold_model_predict(self.handle, ctypes.byref(c), out.data_ptr(), _stream_ptr(stream)))
        return out

    def sketch(self, R, stream=None) -> torch.Tensor:
        L = _model_lib()
        keep = []
        c = _csr(R, keep)
        out = torch.empty((c.n_rows, SKETCH_WIDTH), dtype=torch.bfloat16, device="cuda")
        _check(L, L.knn_threshold_sketch(self.handle, ctypes.byref(c), out.data_ptr(), _stream_ptr(stream)))
        return out

    def params(self) -> torch.Tensor:
        """fp32 parameters (a copy): W1 [256,528], b1, W2 [256,256], b2, w3 [256], b3 [1]."""
        L = _model_lib()
        p = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check(L, L.knn_threshold_model_params(self.handle, ctypes.byref(p), ctypes.byref(n)))
        torch.cuda.synchronize()

        class _Dev:   # a view of the library's device array for torch.as_tensor
            __cuda_array_interface__ = {"shape": (n.value,), "typestr": "<f4", "data": (p.value, False),
                                        "version": 3}
        return torch.as_tensor(_Dev(), device="cuda").clone()

    def forward_backward(self, x_bf16: torch.Tensor, target: torch.Tensor, quantile: float, stream=None):
        L = _model_lib()
        B = x_bf16.shape[0]
        pred = torch.empty(B, dtype=torch.float32, device="cuda")
        n = ctypes.c_int64()
        p = ctypes.c_void_p()
        _check(L, L.knn_threshold_model_params(self.handle, ctypes.byref(p), ctypes.byref(n)))
        grads = torch.empty(n.value, dtype=torch.float32, device="cuda")
        _check(L, L.knn_threshold_model_forward_backward(self.handle, x_bf16.contiguous().data_ptr(),
                                                         target.contiguous().float().data_ptr(), B,
                                                         float(quantile), pred.data_ptr(), grads.data_ptr(),
                                                         _stream_ptr(stream)))
        return pred, grads

    def get_params(self) -> bytes:
        L = _model_lib()
        need = ctypes.c_size_t()
        _check(L, L.knn_threshold_model_get_params(self.handle, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(L, L.knn_threshold_model_get_params(self.handle, buf, need.value, ctypes.byref(need)))
        return buf.raw

    def set_params(self, data: bytes):
        L = _model_lib()
        buf = ctypes.create_string_buffer(data, len(data))
        _check(L, L.knn_threshold_model_set_params(self.handle, buf, len(data)))

    def close(self):
        if self._h:
            _model_lib().knn_threshold_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def knn_gemm_bf16(A: torch.Tensor, sa, B: torch.Tensor, sb, C: torch.Tensor, sc, M, N, K, accumulate=False,
                  stream=None):
    """C (+)= A @ B on tensor cores with explicit element strides (test hook)."""
    L = _model_lib()
    _check(L, L.knn_gemm_bf16(M, N, K, A.data_ptr(), sa[0], sa[1], B.data_ptr(), sb[0], sb[1], C.data_ptr(),
                              sc[0], sc[1], int(accumulate), _stream_ptr(stream)))


def knn_join_learned(index: Index, model: "ThresholdModel | None", R, k: int, *, tau: torch.Tensor | None = None,
                     tau_scale: float = 0.0, mode: str = "iiib", threads: int = 0, s_groups: int = 0,
                     postings_scanned: torch.Tensor | None = None, stats_out: torch.Tensor | None = None,
                     level_margin: float = 0.0, blocks_per_launch: int = 0, out_ids=None, out_scores=None,
                     stream=None):
    """Exact top-k from predicted start thresholds with verify-and-fallback.

    Returns (ids, scores, {"rows": n, "fallback_rows": m}).
    """
    L = _model_lib()
    keep = []
    c = _csr(R, keep)
    n = c.n_rows
    sdt = torch.int32 if index.dtype == KNN_U8 else torch.float32
    if out_ids is None:
        out_ids = torch.empty((n, k), dtype=torch.int32, device="cuda")
        out_scores = torch.empty((n, k), dtype=sdt, device="cuda")
    jo = _JoinOpts(_mode(mode), int(threads), int(s_groups), None, None,
                   _ptr(postings_scanned), 0, 0, float(level_margin), _ptr(stats_out), int(blocks_per_launch))
    lo = _LearnedOpts(jo, float(tau_scale), _ptr(tau))
    st = _LearnedStats()
    _check(L, L.knn_join_learned(index.handle, model.handle if model is not None else None, ctypes.byref(c),
                                 int(k), ctypes.byref(lo), out_ids.data_ptr(), out_scores.data_ptr(),
                                 ctypes.byref(st), _stream_ptr(stream)))
    return out_ids, out_scores, {"rows": int(st.rows), "fallback_rows": int(st.fallback_rows)}


# ----------------------------------------------------------------------------------
# batched joins
# ----------------------------------------------------------------------------------

class _Job(ctypes.Structure):
    _fields_ = [("index", ctypes.c_void_p), ("R", _Csr), ("k", ctypes.c_int32), ("out_ids", ctypes.c_void_p),
                ("out_scores", ctypes.c_void_p)]


class _BatchOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("threads", ctypes.c_int32), ("blocks_per_group", ctypes.c_int32),
                ("level_margin", ctypes.c_float), ("use_graph", ctypes.c_int32),
                ("skip_validation", ctypes.c_int32), ("stats", ctypes.c_void_p), ("wait_spins", ctypes.c_int64),
                ("test_never_publish", ctypes.c_int32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("work_items", ctypes.c_int64), ("ctas", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("shared_bytes", ctypes.c_int64), ("graph", ctypes.c_int32), ("kernels_per_launch", ctypes.c_int32)]


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        P = ctypes.POINTER
        L.knn_batch_create.argtypes = [ctypes.c_int32, P(_Job), P(_BatchOpts), ctypes.c_void_p, P(ctypes.c_void_p)]
        L.knn_batch_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.knn_batch_get_info.argtypes = [ctypes.c_void_p, P(_BatchInfo)]
        L.knn_batch_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.knn_batch_destroy.argtypes = [ctypes.c_void_p]
        L.knn_batch_destroy.restype = None
        L.knn_join_batched.argtypes = [ctypes.c_int32, P(_Job), P(_BatchOpts), ctypes.c_void_p]
        L._batch_ready = True
    return L


def _jobs_array(jobs, keep):
    """jobs: list of (Index, DeviceCSR, k[, out_ids, out_scores]) -> ctypes array, outputs."""
    arr = (_Job * len(jobs))()
    outs = []
    for i, jb in enumerate(jobs):
        index, R, k = jb[0], jb[1], int(jb[2])
        if not isinstance(R, DeviceCSR):
            raise TypeError("batched jobs need DeviceCSR queries")
        c = _csr(R, keep)
        sdt = torch.int32 if index.dtype == KNN_U8 else torch.float32
        if len(jb) > 3:
            ids, sc = jb[3], jb[4]
        else:
            ids = torch.empty((c.n_rows, k), dtype=torch.int32, device="cuda")
            sc = torch.empty((c.n_rows, k), dtype=sdt, device="cuda")
        keep.extend([ids, sc])
        arr[i] = _Job(index.handle, c, k, ids.data_ptr(), sc.data_ptr())
        outs.append((ids, sc))
    return arr, outs


class Batch:
    """A prepared knn_batch (work items, scratch, optionally a captured CUDA graph)."""

    def __init__(self, jobs, *, mode="iiib", threads=0, blocks_per_group=0, level_margin=0.0, use_graph=True,
                 skip_validation=False, stats: torch.Tensor | None = None, wait_spins: int = 0,
                 test_never_publish: bool = False, stream=None):
        L = _batch_lib()
        self._keep = []
        arr, self.outputs = _jobs_array(jobs, self._keep)
        self._keep.append(arr)
        o = _BatchOpts(_mode(mode), int(threads), int(blocks_per_group),
                       float(level_margin), int(bool(use_graph)), int(bool(skip_validation)), _ptr(stats),
                       int(wait_spins), int(bool(test_never_publish)))
        h = ctypes.c_void_p()
        _check(L, L.knn_batch_create(len(jobs), arr, ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h.value

    def launch(self, stream=None):
        L = _batch_lib()
        _check(L, L.knn_batch_launch(self._h, _stream_ptr(stream)))
        return self.outputs

    def check(self, stream=None):
        """Synchronises and raises KnnError (KNN_ETIMEOUT) if a bounded wait gave up."""
        L = _batch_lib()
        _check(L, L.knn_batch_check(self._h, _stream_ptr(stream)))

    def info(self) -> dict:
        L = _batch_lib()
        inf = _BatchInfo()
        _check(L, L.knn_batch_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _BatchInfo._fields_}

    def close(self):
        if self._h:
            _batch_lib().knn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def knn_join_batched(jobs, *, mode="iiib", threads=0, blocks_per_group=0, level_margin=0.0, stream=None):
    """Runs the jobs [(Index, DeviceCSR, k), ...] in one persistent launch; returns [(ids, scores)]."""
    L = _batch_lib()
    keep = []
    arr, outs = _jobs_array(jobs, keep)
    o = _BatchOpts(_mode(mode), int(threads), int(blocks_per_group),
                   float(level_margin), 0, 0, None, 0, 0)
    _check(L, L.knn_join_batched(len(jobs), arr, ctypes.byref(o), _stream_ptr(stream)))
    return outs


def knn_merge_topk(parts, offsets, k: int, stream=None):
    """knn_merge_topk: parts = [(ids, scores), ...] (device [n_rows, k] tensors, as
    knn_join returns them, ids relative to each shard), offsets = each shard's first S
    id; returns the global (ids, scores) [n_rows, k]."""
    L = lib()
    if not getattr(L, "_merge_ready", False):
        L.knn_merge_topk.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
        L._merge_ready = True
    n = len(parts)
    if n != len(offsets):
        raise ValueError("one offset per part")
    ids0, sc0 = parts[0]
    n_rows = ids0.shape[0]
    for ids, sc in parts:
        if ids.shape != (n_rows, k) or sc.shape != (n_rows, k) or not ids.is_cuda or not sc.is_cuda:
            raise ValueError("every part must be a pair of device tensors [n_rows, k]")
    dtype = KNN_F32 if sc0.dtype == torch.float32 else KNN_U8
    parts = [(ids.contiguous(), sc.contiguous()) for ids, sc in parts]
    pid = (ctypes.c_void_p * n)(*[ids.data_ptr() for ids, _ in parts])
    psc = (ctypes.c_void_p * n)(*[sc.data_ptr() for _, sc in parts])
    off = (ctypes.c_int64 * n)(*[int(o) for o in offsets])
    out_ids = torch.empty((n_rows, k), dtype=torch.int32, device=ids0.device)
    out_sc = torch.empty((n_rows, k), dtype=sc0.dtype, device=ids0.device)
    _check(L, L.knn_merge_topk(n, pid, psc, off, int(n_rows), int(k), dtype, out_ids.data_ptr(), out_sc.data_ptr(),
                               _stream_ptr(stream)))
    return out_ids, out_sc


# ----------------------------------------------------------------------------------
# MS/MS spectra as sparse vectors (Section 5's preprocessing; host code, no GPU)
# ----------------------------------------------------------------------------------
_SPECTRA_FORMATS = {"auto": 0, "mgf": 1, "ms2": 2}
_SPECTRA_MERGE = {"max": 0, "sum": 1}
_SPECTRA_WEIGHTS = {"f32": 0, "u8": 1}


class _SpectraOpts(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int), ("mz_scale", ctypes.c_double), ("merge", ctypes.c_int),
                ("weights", ctypes.c_int), ("dim", ctypes.c_int32), ("min_intensity", ctypes.c_double),
                ("chunk_bytes", ctypes.c_int64)]


class _SpectraInfo(ctypes.Structure):
    _fields_ = [("n_spectra", ctypes.c_int64), ("n_peaks", ctypes.c_int64), ("n_features", ctypes.c_int64),
                ("n_dropped", ctypes.c_int64), ("n_merged", ctypes.c_int64), ("dim", ctypes.c_int32),
                ("dtype", ctypes.c_int)]


def _spectra_lib():
    L = lib()
    if not getattr(L, "_spectra_ready", False):
        P = ctypes.POINTER
        L.knn_spectra_parse.argtypes = [ctypes.c_char_p, ctypes.c_size_t, P(_SpectraOpts), P(ctypes.c_void_p)]
        L.knn_spectra_read.argtypes = [ctypes.c_char_p, P(_SpectraOpts), P(ctypes.c_void_p)]
        L.knn_spectra_csr.argtypes = [ctypes.c_void_p, P(_Csr)]
        L.knn_spectra_get_info.argtypes = [ctypes.c_void_p, P(_SpectraInfo)]
        L.knn_spectra_free.argtypes = [ctypes.c_void_p]
        L.knn_spectra_free.restype = None
        L._spectra_ready = True
    return L


def _spectra_opts(fmt, mz_scale, merge, weights, dim, min_intensity, chunk_bytes):
    try:
        return _SpectraOpts(_SPECTRA_FORMATS[fmt], float(mz_scale), _SPECTRA_MERGE[merge],
                            _SPECTRA_WEIGHTS[weights], int(dim), float(min_intensity), int(chunk_bytes))
    except KeyError as e:
        raise ValueError(f"unknown option value {e}") from None


def _spectra_take(L, handle):
    """Copies the library's host CSR out of `handle` (then freed): (CSR, info dict)."""
    from .synth import CSR
    try:
        c = _Csr()
        _check(L, L.knn_spectra_csr(handle, ctypes.byref(c)))
        inf = _SpectraInfo()
        _check(L, L.knn_spectra_get_info(handle, ctypes.byref(inf)))
        n, nnz = int(c.n_rows), int(inf.n_features)
        vdt = np.uint8 if c.dtype == KNN_U8 else np.float32

        def take(ptr, count, dt):
            if count == 0 or not ptr:
                return np.zeros(count, dt)
            return np.frombuffer((ctypes.c_char * (count * np.dtype(dt).itemsize)).from_address(ptr), dt).copy()

        csr = CSR(take(c.indptr, n + 1, np.int64), take(c.indices, nnz, np.int32), take(c.values, nnz, vdt),
                  int(c.dim))
        info = {f: getattr(inf, f) for f, _ in _SpectraInfo._fields_}
        return csr, info
    finally:
        L.knn_spectra_free(handle)


def spectra_parse(text, *, fmt: str = "auto", mz_scale: float = 10.0, merge: str = "max", weights: str = "f32",
                  dim: int = 0, min_intensity: float = 0.0, chunk_bytes: int = 0):
    """knn_spectra_parse: MGF or MS2 text (str or bytes) -> (CSR on the host, info dict)."""
    L = _spectra_lib()
    data = text.encode() if isinstance(text, str) else bytes(text)
    o = _spectra_opts(fmt, mz_scale, merge, weights, dim, min_intensity, chunk_bytes)
    h = ctypes.c_void_p()
    _check(L, L.knn_spectra_parse(data, len(data), ctypes.byref(o), ctypes.byref(h)))
    return _spectra_take(L, h.value)


def spectra_read(path, *, fmt: str = "auto", mz_scale: float = 10.0, merge: str = "max", weights: str = "f32",
                 dim: int = 0, min_intensity: float = 0.0, chunk_bytes: int = 0):
    """knn_spectra_read: an MGF or MS2 file -> (CSR on the host, info dict)."""
    L = _spectra_lib()
    o = _spectra_opts(fmt, mz_scale, merge, weights, dim, min_intensity, chunk_bytes)
    h = ctypes.c_void_p()
    _check(L, L.knn_spectra_read(os.fsencode(path), ctypes.byref(o), ctypes.byref(h)))
    return _spectra_take(L, h.value)
