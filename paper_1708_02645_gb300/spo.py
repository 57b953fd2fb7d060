"""Thin ctypes binding of libspo (include/spo.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  If
libspo.so has not been built, loading raises SpoError; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

F64, F32, BF16, F16 = 0, 1, 2, 3
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}
KIND_V, KIND_VGL, KIND_VGH = 0, 1, 2
KINDS = {"v": KIND_V, "vgl": KIND_VGL, "vgh": KIND_VGH}
ALGO_AUTO, ALGO_GATHER, ALGO_SORTED_GATHER, ALGO_BRICK = 0, 1, 2, 3
ALGOS = {"auto": ALGO_AUTO, "gather": ALGO_GATHER, "sorted_gather": ALGO_SORTED_GATHER,
         "brick": ALGO_BRICK}
ROWS = {KIND_V: 1, KIND_VGL: 5, KIND_VGH: 10}
PARAMS = {"brick_vec": 0, "brick_tile": 1, "brick_schedule": 2}
STATUS = {0: "SPO_OK", 1: "SPO_EINVAL", 2: "SPO_ENOMEM", 3: "SPO_ECUDA", 4: "SPO_ETIMEOUT",
          5: "SPO_EUNSUPPORTED"}

# every symbol include/spo.h declares: (name, restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
SIGNATURES = [
    ("spo_create", _INT, [_P, _P, _INT, _I64, _INT, _INT, ctypes.POINTER(_P)]),
    ("spo_destroy", _INT, [_P]),
    ("spo_eval_v", _INT, [_P, _P, _I64, _P, _P]),
    ("spo_eval_vgl", _INT, [_P, _P, _I64, _P, _P]),
    ("spo_eval_vgh", _INT, [_P, _P, _I64, _P, _P]),
    ("spo_eval", _INT, [_P, _INT, _P, _I64, _P, _P]),
    ("spo_eval_ex", _INT, [_P, _INT, _P, _I64, _P, _P, _INT]),
    ("spo_bin", _INT, [_P, _P, _I64, _P]),
    ("spo_eval_binned", _INT, [_P, _INT, _P, _I64, _P, _P, _INT]),
    ("spo_reserve", _INT, [_P, _I64, _P]),
    ("spo_eval_noalloc", _INT, [_P, _INT, _P, _I64, _P, _P]),
    ("spo_eval_ratio", _INT, [_P, _P, _I64, _P, _I64, _I64, _P, _P, _P, _P]),
    ("spo_autotune", _INT, [_P, _INT, _I64, _P, _P]),
    ("spo_batch_create", _INT, [_P, _INT, _I64, _INT, ctypes.POINTER(_P)]),
    ("spo_batch_eval", _INT, [_P, _INT, _P, _INT, _P]),
    ("spo_batch_graph", _INT, [_P, _INT, _P, _INT, _P]),
    ("spo_batch_launch", _INT, [_P, _P]),
    ("spo_batch_destroy", _INT, [_P]),
    ("spo_eval_batch", _INT, [_P, _INT, _P, _INT, _INT, _P]),
    ("spo_device_status", _INT, [ctypes.POINTER(ctypes.c_uint), _INT, _P]),
    ("spo_eval_host", _INT, [_P, _INT, _P, _I64, _P, _P]),
    ("spo_set_param", _INT, [_P, _INT, _I64]),
    ("spo_get_param", _INT, [_P, _INT, ctypes.POINTER(_I64)]),
    ("spo_auto_algo", _INT, [_P, _INT, _I64, ctypes.POINTER(_INT)]),
    ("spo_footprint", _INT, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    ("spo_info", _INT, [_P, _P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_INT)]),
    ("spo_selftest_wait", _INT, [ctypes.c_uint64, _P, ctypes.POINTER(_INT)]),
    ("spo_prefilter", _INT, [_P, _I64, _P, _INT, _P]),
    ("spo_surrogate_create", _INT, [_P, ctypes.c_uint64, ctypes.POINTER(_P)]),
    ("spo_surrogate_train", _INT, [_P, _P, _I64, _I64, ctypes.c_float, _P, ctypes.c_uint64, _P,
                                   ctypes.POINTER(ctypes.c_float)]),
    ("spo_surrogate_eval", _INT, [_P, _INT, _P, _I64, _P, _INT, _P]),
    ("spo_surrogate_grad", _INT, [_P, _P, _P, _I64, _P, _INT, ctypes.POINTER(ctypes.c_float), _P, _P,
                                  _P, _P]),
    ("spo_surrogate_set_train_precision", _INT, [_P, _INT]),
    ("spo_surrogate_set_level_lr", _INT, [_P, ctypes.c_float]),
    ("spo_surrogate_set_optimizer", _INT, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_float]),
    ("spo_surrogate_nparams", _INT, [_P, ctypes.POINTER(_I64)]),
    ("spo_surrogate_state", _INT, [_P, _P, _P, _P, ctypes.POINTER(_I64), _INT]),
    ("spo_surrogate_footprint", _INT, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    ("spo_surrogate_params", _INT, [_P, _P, _P, _P, _INT]),
    ("spo_surrogate_destroy", _INT, [_P]),
    ("spo_rows", _INT, [_INT]),
    ("spo_status_str", ctypes.c_char_p, [_INT]),
    ("spo_last_error", ctypes.c_char_p, []),
    ("spo_abi_version", _INT, []),
]


class SpoError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The in-tree libspo.so, or the library named by SPO_LIBRARY (another
    build of it, such as the index-checking debug build)."""
    return os.environ.get("SPO_LIBRARY") or _build.LIB


def load() -> ctypes.CDLL:
    """Load libspo.so (raises SpoError-like RuntimeError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libspo.so is not built ({path}); build it with "
                    "paper_1708_02645_gb300.build.build() — there is no CPU fallback")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != 0:
        detail = load().spo_last_error().decode(errors="replace")
        raise SpoError(status, where, detail)


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dtype_of(coefs, src_dtype):
    if src_dtype is not None:
        return DTYPES[src_dtype] if isinstance(src_dtype, str) else int(src_dtype)
    torch = _torch()
    if isinstance(coefs, torch.Tensor):
        m = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
        if coefs.dtype not in m:
            raise TypeError(f"unsupported coefficient dtype {coefs.dtype}")
        return m[coefs.dtype]
    m = {np.dtype(np.float64): F64, np.dtype(np.float32): F32, np.dtype(np.float16): F16}
    if coefs.dtype not in m:
        raise TypeError(f"unsupported coefficient dtype {coefs.dtype} (pass src_dtype for raw bf16)")
    return m[coefs.dtype]


def device_status(clear: bool = True, stream=None) -> int:
    """Device-side status word of the current device (bit 0: a bounded wait
    on a TMA copy gave up; bit 1: an index check of a -DSPO_CHECK_BOUNDS build
    failed).  Raises SpoError(SPO_ETIMEOUT) if bit 0 is set, SpoError(SPO_EINVAL)
    if bit 1 is."""
    flags = ctypes.c_uint()
    _check(load().spo_device_status(ctypes.byref(flags), int(clear), _stream_handle(stream)),
           "spo_device_status")
    return int(flags.value)


class _Tuning(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("brick_tile", ctypes.c_int32),
                ("brick_vec", ctypes.c_int32), ("brick_schedule", ctypes.c_int32),
                ("ms", ctypes.c_float), ("from_cache", ctypes.c_int32)]


ALGO_NAMES = {v: k for k, v in ALGOS.items()}


class OrbitalSet:
    """One B-spline orbital set resident on the current CUDA device.

    coefs: [nx, ny, nz, N] coefficients, numpy (host) or torch (host or
    device), FP64/FP32/FP16, torch BF16, or a raw uint16 numpy array with
    src_dtype="bf16".  storage: "f32", "bf16" or "f16".
    """

    def __init__(self, coefs, storage: str = "f32", src_dtype=None):
        lib = load()
        torch = _torch()
        sd = _dtype_of(coefs, src_dtype)
        on_device = isinstance(coefs, torch.Tensor) and coefs.is_cuda
        if isinstance(coefs, torch.Tensor):
            coefs = coefs.contiguous()
            keep = coefs
            ptr = coefs.data_ptr()
        else:
            keep = np.ascontiguousarray(coefs)
            ptr = keep.ctypes.data
        if len(keep.shape) != 4:
            raise ValueError("coefs must be [nx, ny, nz, N]")
        nx, ny, nz, N = (int(s) for s in keep.shape)
        grid = _Grid(nx, ny, nz)
        h = ctypes.c_void_p()
        _check(lib.spo_create(ctypes.byref(grid), ctypes.c_void_p(ptr), sd, N, DTYPES[storage],
                              int(on_device), ctypes.byref(h)), "spo_create")
        self._h = h
        self.grid = (nx, ny, nz)
        self.N = N
        self.storage = storage
        self.device = torch.cuda.current_device()
        del keep

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("orbital set already destroyed")
        return self._h

    def set_param(self, name: str, value: int):
        """Tuning parameter ("brick_vec": 2 or 4, "brick_tile": 32 or 64,
        "brick_schedule": 0 or 1); outputs do not change."""
        _check(load().spo_set_param(self.handle, PARAMS[name], int(value)), "spo_set_param")

    def get_param(self, name: str) -> int:
        v = _I64()
        _check(load().spo_get_param(self.handle, PARAMS[name], ctypes.byref(v)), "spo_get_param")
        return int(v.value)

    def autotune(self, kind="vgh", P: int = 98304, stream=None) -> dict:
        """spo_autotune: time the strategies for this kind and batch size,
        apply the fastest, and return it."""
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        t = _Tuning()
        _check(load().spo_autotune(self.handle, k, int(P), _stream_handle(stream), ctypes.byref(t)),
               "spo_autotune")
        return {"algo": ALGO_NAMES[t.algo], "brick_tile": t.brick_tile, "brick_vec": t.brick_vec,
                "brick_schedule": t.brick_schedule, "ms": t.ms, "from_cache": bool(t.from_cache)}

    def footprint(self) -> int:
        b = ctypes.c_size_t()
        _check(load().spo_footprint(self.handle, ctypes.byref(b)), "spo_footprint")
        return int(b.value)

    def auto_algo(self, kind, P: int) -> str:
        """The strategy algo="auto" takes for this kind and batch size."""
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        a = _INT()
        _check(load().spo_auto_algo(self.handle, k, int(P), ctypes.byref(a)), "spo_auto_algo")
        return {v: n for n, v in ALGOS.items()}[a.value]

    def info(self):
        g = _Grid()
        n, npad, st = _I64(), _I64(), _INT()
        _check(load().spo_info(self.handle, ctypes.byref(g), ctypes.byref(n), ctypes.byref(npad),
                               ctypes.byref(st)), "spo_info")
        return {"grid": (g.nx, g.ny, g.nz), "N": n.value, "Np": npad.value, "storage": st.value}

    def out_shape(self, P: int, kind) -> tuple:
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        return (P, self.N) if k == KIND_V else (P, ROWS[k], self.N)

    def _check_pos(self, pos):
        torch = _torch()
        if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dtype == torch.float32):
            raise TypeError("pos must be a float32 CUDA tensor")
        if pos.dim() != 2 or pos.shape[1] != 3 or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous [P, 3] tensor")
        return int(pos.shape[0])

    def _out_for(self, pos, P, k, out):
        torch = _torch()
        if out is None:
            return torch.empty(self.out_shape(P, k), dtype=torch.float32, device=pos.device)
        if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
                and out.numel() == P * ROWS[k] * self.N):
            raise ValueError("out must be a contiguous float32 CUDA tensor of the output shape")
        return out

    def eval(self, pos, kind="vgh", out=None, stream=None, algo="auto"):
        """Evaluate at device positions pos [P, 3] (FP32 torch CUDA tensor).
        Returns out (allocated if None): [P, N], [P, 5, N] or [P, 10, N].
        algo: "auto", "gather", "sorted_gather" or "brick" (same values)."""
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        P = self._check_pos(pos)
        out = self._out_for(pos, P, k, out)
        _check(load().spo_eval_ex(self.handle, k, ctypes.c_void_p(pos.data_ptr()), P,
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream), a),
               "spo_eval_ex")
        return out

    def bin(self, pos, stream=None):
        """Sort pos by brick into this set's scratch for the stream."""
        P = self._check_pos(pos)
        _check(load().spo_bin(self.handle, ctypes.c_void_p(pos.data_ptr()), P,
                              _stream_handle(stream)), "spo_bin")

    def eval_binned(self, pos, kind="vgh", out=None, stream=None, algo="brick"):
        """Evaluate from the binning of the last bin(pos) on the stream."""
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        P = self._check_pos(pos)
        out = self._out_for(pos, P, k, out)
        _check(load().spo_eval_binned(self.handle, k, ctypes.c_void_p(pos.data_ptr()), P,
                                      ctypes.c_void_p(out.data_ptr()), _stream_handle(stream), a),
               "spo_eval_binned")
        return out

    def eval_ratio(self, pos, rows, row_of=None, ratio=None, v_out=None, stream=None):
        """Determinant ratios rho_p = rows[row_of[p]] . phi(pos_p) (eq.
        md_lemma).  rows: FP32 CUDA [R, ld >= N]; row_of: int32 CUDA [P] or
        None (row p); v_out: optional FP32 CUDA [P, N] for the values."""
        torch = _torch()
        P = self._check_pos(pos)
        if not (rows.is_cuda and rows.dtype == torch.float32 and rows.dim() == 2
                and rows.stride(1) == 1):
            raise TypeError("rows must be a row-major float32 CUDA matrix")
        if row_of is not None and not (row_of.is_cuda and row_of.dtype == torch.int32
                                       and row_of.is_contiguous() and row_of.numel() == P):
            raise TypeError("row_of must be a contiguous int32 CUDA vector of length P")
        if ratio is None:
            ratio = torch.empty((P,), dtype=torch.float32, device=pos.device)
        if v_out is not None:
            v_out = self._out_for(pos, P, KIND_V, v_out)
        _check(load().spo_eval_ratio(
            self.handle, ctypes.c_void_p(pos.data_ptr()), P, ctypes.c_void_p(rows.data_ptr()),
            int(rows.shape[0]), int(rows.stride(0)),
            ctypes.c_void_p(row_of.data_ptr() if row_of is not None else None),
            ctypes.c_void_p(ratio.data_ptr()),
            ctypes.c_void_p(v_out.data_ptr() if v_out is not None else None),
            _stream_handle(stream)), "spo_eval_ratio")
        return ratio

    def eval_noalloc(self, pos, kind="vgh", out=None, stream=None):
        """spo_eval_noalloc: the library allocates nothing (pass `out` to
        allocate nothing at all); scratch is a fixed per-device array, so
        calls must not overlap on the GPU.  P <= 262,144."""
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        P = self._check_pos(pos)
        out = self._out_for(pos, P, k, out)
        _check(load().spo_eval_noalloc(self.handle, k, ctypes.c_void_p(pos.data_ptr()), P,
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "spo_eval_noalloc")
        return out

    def reserve(self, P: int, stream=None):
        """Pre-allocate binning scratch for batches of up to P positions."""
        _check(load().spo_reserve(self.handle, int(P), _stream_handle(stream)), "spo_reserve")

    def eval_v(self, pos, out=None, stream=None):
        return self.eval(pos, "v", out, stream)

    def eval_vgl(self, pos, out=None, stream=None):
        return self.eval(pos, "vgl", out, stream)

    def eval_vgh(self, pos, out=None, stream=None):
        return self.eval(pos, "vgh", out, stream)

    def eval_host(self, pos, kind="vgh", out=None, stream=None):
        """Evaluate host positions (numpy or CPU tensor, FP32 [P, 3]) into a
        host output (numpy/CPU tensor, allocated if None).  Synchronous."""
        torch = _torch()
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        if isinstance(pos, torch.Tensor):
            if pos.is_cuda or pos.dtype != torch.float32 or not pos.is_contiguous():
                raise TypeError("pos must be a contiguous float32 CPU tensor")
            pptr, P = pos.data_ptr(), int(pos.shape[0])
        else:
            pos = np.ascontiguousarray(pos, dtype=np.float32)
            pptr, P = pos.ctypes.data, int(pos.shape[0])
        if out is None:
            out = np.empty(self.out_shape(P, k), dtype=np.float32)
        if isinstance(out, torch.Tensor):
            if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() \
                    or out.numel() != P * ROWS[k] * self.N:
                raise ValueError("out must be a contiguous float32 CPU tensor of the output shape")
            optr = out.data_ptr()
        else:
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != P * ROWS[k] * self.N:
                raise ValueError("out must be a contiguous float32 array of the output shape")
            optr = out.ctypes.data
        _check(load().spo_eval_host(self.handle, k, ctypes.c_void_p(pptr), P, ctypes.c_void_p(optr),
                                    _stream_handle(stream)), "spo_eval_host")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(load().spo_destroy(self._h), "spo_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _Work(ctypes.Structure):
    _fields_ = [("set", ctypes.c_int32), ("reserved", ctypes.c_int32), ("P", ctypes.c_int64),
                ("pos", ctypes.c_void_p), ("out", ctypes.c_void_p)]


def selftest_wait(limit_ns: int = 50_000_000, stream=None) -> bool:
    """Run a bounded device-side wait that cannot succeed; True when the
    time-out was detected and reported through the device status word."""
    t = ctypes.c_int()
    _check(load().spo_selftest_wait(int(limit_ns), _stream_handle(stream), ctypes.byref(t)),
           "spo_selftest_wait")
    return bool(t.value)


def prefilter(samples, stream=None):
    """Interpolating B-spline coefficients from periodic grid samples, in
    place: samples is a CUDA tensor [nx, ny, nz, N] (float64 or float32)."""
    torch = _torch()
    if not samples.is_cuda or not samples.is_contiguous() or samples.dim() != 4:
        raise TypeError("samples must be a contiguous CUDA tensor [nx, ny, nz, N]")
    dt = {torch.float64: F64, torch.float32: F32}.get(samples.dtype)
    if dt is None:
        raise TypeError("samples must be float64 or float32")
    g = _Grid(*[int(x) for x in samples.shape[:3]])
    _check(load().spo_prefilter(ctypes.byref(g), int(samples.shape[3]), ctypes.c_void_p(samples.data_ptr()),
                                dt, _stream_handle(stream)), "spo_prefilter")
    return samples


def eval_batch(sets, items, kind="vgh", stream=None):
    """One-call batched evaluation (spo_eval_batch): items are (set index,
    pos [P, 3] CUDA FP32, out CUDA FP32)."""
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    arr = (ctypes.c_void_p * len(sets))(*[s.handle.value for s in sets])
    table = (_Work * max(1, len(items)))()
    for i, (si, pos, out) in enumerate(items):
        table[i].set = int(si)
        table[i].reserved = 0
        table[i].P = int(pos.shape[0])
        table[i].pos = pos.data_ptr()
        table[i].out = out.data_ptr()
    _check(load().spo_eval_batch(arr, len(sets), table, len(items), k, _stream_handle(stream)),
           "spo_eval_batch")


class Batch:
    """A batched-crowd plan over several OrbitalSets (same storage type):
    many walkers, each (set index, pos [P, 3] CUDA FP32, out CUDA FP32),
    evaluated with one binning and one kernel launch, optionally recorded
    into a CUDA graph and replayed."""

    def __init__(self, sets, max_positions: int, max_items: int):
        self.sets = list(sets)          # keep the sets alive
        arr = (ctypes.c_void_p * len(self.sets))(*[s.handle.value for s in self.sets])
        h = ctypes.c_void_p()
        _check(load().spo_batch_create(arr, len(self.sets), int(max_positions), int(max_items),
                                       ctypes.byref(h)), "spo_batch_create")
        self._h = h

    def _table(self, items):
        table = (_Work * max(1, len(items)))()
        for i, (k, pos, out) in enumerate(items):
            table[i].set = int(k)
            table[i].reserved = 0
            table[i].P = int(pos.shape[0])
            table[i].pos = pos.data_ptr()
            table[i].out = out.data_ptr()
        return table

    def eval(self, items, kind="vgh", stream=None):
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        table = self._table(items)
        _check(load().spo_batch_eval(self._h, k, table, len(items), _stream_handle(stream)),
               "spo_batch_eval")

    def graph(self, items, kind="vgh", stream=None):
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        table = self._table(items)
        _check(load().spo_batch_graph(self._h, k, table, len(items), _stream_handle(stream)),
               "spo_batch_graph")

    def launch(self, stream=None):
        _check(load().spo_batch_launch(self._h, _stream_handle(stream)), "spo_batch_launch")

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(load().spo_batch_destroy(self._h), "spo_batch_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _SurrogateSpec(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("log2_table", ctypes.c_int32),
                ("features", ctypes.c_int32), ("r_min", ctypes.c_int32), ("r_max", ctypes.c_int32),
                ("hidden", ctypes.c_int32), ("layers", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("N", ctypes.c_int64)]


class Surrogate:
    """Learned surrogate of an orbital set (hashed grid + softplus
    perceptron) on the current CUDA device.

    spec: any object with the fields levels, log2_table, features, r_min,
    r_max, hidden, layers, N.  eval() gives V [P, N] or VGL [P, 5, N];
    precision 0 evaluates the FP32 master parameters, 1 the FP16-grid /
    BF16-weight inference copy."""

    def __init__(self, spec, seed: int = 0):
        self.spec = spec
        c = _SurrogateSpec(int(spec.levels), int(spec.log2_table), int(spec.features),
                           int(spec.r_min), int(spec.r_max), int(spec.hidden), int(spec.layers), 0,
                           int(spec.N))
        h = ctypes.c_void_p()
        _check(load().spo_surrogate_create(ctypes.byref(c), int(seed), ctypes.byref(h)),
               "spo_surrogate_create")
        self._h = h
        self.widths = [spec.levels * spec.features] + [spec.hidden] * spec.layers + [spec.N]

    def _param_buffers(self):
        T = 1 << self.spec.log2_table
        grid = np.zeros((self.spec.levels, T, self.spec.features), dtype=np.float32)
        W = [np.zeros((o, i), dtype=np.float32) for i, o in zip(self.widths[:-1], self.widths[1:])]
        b = [np.zeros(o, dtype=np.float32) for o in self.widths[1:]]
        return grid, W, b

    def _params_call(self, grid, W, b, to_device):
        Wp = (ctypes.c_void_p * len(W))(*[w.ctypes.data for w in W])
        bp = (ctypes.c_void_p * len(b))(*[v.ctypes.data for v in b])
        _check(load().spo_surrogate_params(self._h, grid.ctypes.data, Wp, bp, int(to_device)),
               "spo_surrogate_params")

    def set_params(self, grid, W, b):
        """Load FP32 master parameters (grid [levels, T, F], W[l] [out, in], b[l] [out])."""
        g0, W0, b0 = self._param_buffers()
        grid = np.ascontiguousarray(np.asarray(grid, dtype=np.float32).reshape(g0.shape))
        W = [np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(w0.shape)) for w, w0 in zip(W, W0)]
        b = [np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(v0.shape)) for v, v0 in zip(b, b0)]
        if len(W) != len(W0) or len(b) != len(b0):
            raise ValueError("wrong number of layers")
        self._params_call(grid, W, b, True)

    def get_params(self):
        grid, W, b = self._param_buffers()
        self._params_call(grid, W, b, False)
        return grid, W, b

    def train(self, teacher: "OrbitalSet", steps: int, batch: int, lr: float, channel_weights=None,
              seed: int = 0, stream=None) -> float:
        """Adam steps on teacher VGL targets; returns the last step's loss."""
        cw = None
        if channel_weights is not None:
            cw = (ctypes.c_float * 5)(*[float(x) for x in channel_weights])
        loss = ctypes.c_float()
        _check(load().spo_surrogate_train(self._h, teacher.handle, int(steps), int(batch), float(lr),
                                          cw, int(seed), _stream_handle(stream), ctypes.byref(loss)),
               "spo_surrogate_train")
        return float(loss.value)

    def grad(self, pos, target, channel_weights=None, precision=0, stream=None):
        """Loss and FP32 gradients (grid, W list, b list) for device positions
        [P, 3] and device targets [P, 5, N]; the parameters are unchanged.
        precision 1: the products as tensor-core training computes them."""
        torch = _torch()
        for t in (pos, target):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise TypeError("pos and target must be contiguous CUDA float32 tensors")
        grid, W, b = self._param_buffers()
        Wp = (ctypes.c_void_p * len(W))(*[w.ctypes.data for w in W])
        bp = (ctypes.c_void_p * len(b))(*[v.ctypes.data for v in b])
        cw = None
        if channel_weights is not None:
            cw = (ctypes.c_float * 5)(*[float(x) for x in channel_weights])
        loss = ctypes.c_float()
        _check(load().spo_surrogate_grad(self._h, ctypes.c_void_p(pos.data_ptr()),
                                         ctypes.c_void_p(target.data_ptr()), int(pos.shape[0]), cw,
                                         int(precision), ctypes.byref(loss), grid.ctypes.data, Wp, bp,
                                         _stream_handle(stream)), "spo_surrogate_grad")
        return float(loss.value), grid, W, b

    def eval(self, pos, out=None, kind="vgl", precision: int = 1, stream=None):
        torch = _torch()
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        if pos.dtype != torch.float32 or not pos.is_cuda or not pos.is_contiguous():
            raise TypeError("pos must be a contiguous CUDA float32 tensor [P, 3]")
        P = pos.shape[0]
        shape = (P, self.spec.N) if k == KIND_V else (P, 5, self.spec.N)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=pos.device)
        _check(load().spo_surrogate_eval(self._h, k, ctypes.c_void_p(pos.data_ptr()), int(P),
                                         ctypes.c_void_p(out.data_ptr()), int(precision),
                                         _stream_handle(stream)), "spo_surrogate_eval")
        return out

    def footprint(self) -> int:
        n = ctypes.c_size_t()
        _check(load().spo_surrogate_footprint(self._h, ctypes.byref(n)), "spo_surrogate_footprint")
        return int(n.value)

    def set_train_precision(self, precision: int):
        """1: training products on the tensor cores (BF16), 0: FP32."""
        _check(load().spo_surrogate_set_train_precision(self._h, int(precision)),
               "spo_surrogate_set_train_precision")

    def set_level_lr(self, power: float):
        """Scale the grid's rate of level l by (R_0 / R_l)^power."""
        _check(load().spo_surrogate_set_level_lr(self._h, float(power)), "spo_surrogate_set_level_lr")

    def set_optimizer(self, beta1=0.9, beta2=0.99, eps=1e-15, grid_lr_mult=1.0):
        _check(load().spo_surrogate_set_optimizer(self._h, float(beta1), float(beta2), float(eps),
                                                  float(grid_lr_mult)), "spo_surrogate_set_optimizer")

    def state(self):
        """(params, m, v, step): the FP32 training state."""
        n = ctypes.c_int64()
        _check(load().spo_surrogate_nparams(self._h, ctypes.byref(n)), "spo_surrogate_nparams")
        params, m, v = (np.empty(n.value, dtype=np.float32) for _ in range(3))
        step = ctypes.c_int64()
        _check(load().spo_surrogate_state(self._h, params.ctypes.data, m.ctypes.data, v.ctypes.data,
                                          ctypes.byref(step), 0), "spo_surrogate_state")
        return params, m, v, int(step.value)

    def restore(self, params, m, v, step):
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.float32)) for x in (params, m, v)]
        st = ctypes.c_int64(int(step))
        _check(load().spo_surrogate_state(self._h, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                          arrs[2].ctypes.data, ctypes.byref(st), 1), "spo_surrogate_state")

    def save(self, path, **meta):
        """Checkpoint: `path` (flat binary: params, m, v as FP32) and
        `path`.json (spec, step, parameter count, caller's metadata)."""
        import json
        params, m, v, step = self.state()
        with open(path, "wb") as f:
            for a in (params, m, v):
                f.write(a.tobytes())
        spec = {k: int(getattr(self.spec, k)) for k in
                ("levels", "log2_table", "features", "r_min", "r_max", "hidden", "layers", "N")}
        with open(path + ".json", "w") as f:
            json.dump({"format": "spo-surrogate-checkpoint-1", "spec": spec, "step": step,
                       "nparams": int(params.size), "dtype": "float32",
                       "arrays": ["params", "adam_m", "adam_v"], "meta": meta}, f, indent=1)

    def load_checkpoint(self, path):
        import json
        with open(path + ".json") as f:
            head = json.load(f)
        for k, v in head["spec"].items():
            if int(getattr(self.spec, k)) != v:
                raise ValueError(f"checkpoint spec {k}={v} differs from this surrogate's")
        n = head["nparams"]
        raw = np.fromfile(path, dtype=np.float32)
        if raw.size != 3 * n:
            raise ValueError("checkpoint size does not match its header")
        self.restore(raw[:n], raw[n:2 * n], raw[2 * n:], head["step"])
        return head

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(load().spo_surrogate_destroy(self._h), "spo_surrogate_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
