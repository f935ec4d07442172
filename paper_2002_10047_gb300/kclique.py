"""Python binding of libkclique.so (C ABI in include/kclique.h).

Argument marshalling only: every step of orientation and counting runs in the
library's CUDA kernels. PyTorch provides device memory and streams. There is
no CPU fallback: if the library is not built or no CUDA device is present,
every call raises.

The functions carry the C names (``kc_orient``, ``kc_count``,
``kc_count_per_vertex``, ...) and the short forms ``orient``, ``count``,
``count_per_vertex`` of Algorithm 1's interface (Section 3.2 of Shi,
Dhulipala, Shun, "Parallel Clique Counting and Peeling Algorithms").
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

KC_OK, KC_EINVAL, KC_ERANGE, KC_ENOMEM, KC_ETIMEDOUT, KC_ECUDA, KC_ECAPACITY = range(7)
KC_KMAX = 32
KC_ORIENT_DEGREE = 0
KC_ORIENT_GP = 1
KC_VALIDATE_SYMMETRY = 0x100
_METHODS = {"degree": KC_ORIENT_DEGREE, "gp": KC_ORIENT_GP}


class KcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class KcOverflow(KcError):
    pass


class KcTimeout(KcError):
    pass


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("nnz", ctypes.c_uint64),
                ("d_row_ptr", ctypes.c_void_p), ("d_col", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("sum_out_sq", ctypes.c_uint64), ("sum_arc_head", ctypes.c_uint64),
                ("triangles", ctypes.c_uint64), ("max_out", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libkclique.so is not built ({path}); run paper_2002_10047_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, I, U32, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
        lib.kc_orient.argtypes = [ctypes.POINTER(_Csr), I, ctypes.POINTER(P), P]
        lib.kc_dag_free.argtypes = [P]
        lib.kc_dag_free.restype = None
        lib.kc_dag_n.argtypes = [P]
        lib.kc_dag_n.restype = U32
        lib.kc_dag_m.argtypes = [P]
        lib.kc_dag_m.restype = U64
        lib.kc_dag_max_out_degree.argtypes = [P]
        lib.kc_dag_max_out_degree.restype = U32
        lib.kc_dag_export.argtypes = [P, P, P, P]
        lib.kc_count.argtypes = [P, I, ctypes.POINTER(U64), P]
        lib.kc_count_per_vertex.argtypes = [P, I, P, P, P]
        lib.kc_count_per_arc.argtypes = [P, I, P, P, P]
        lib.kc_dag_get_stats.argtypes = [P, ctypes.POINTER(_Stats), P]
        lib.kc_measure_word_op_rate.argtypes = [ctypes.POINTER(ctypes.c_double), P]
        lib.kc_measure_word_op_rate.restype = I
        lib.kc_kernel_launches.argtypes = []
        lib.kc_kernel_launches.restype = U64
        lib.kc_strerror.argtypes = [I]
        lib.kc_strerror.restype = ctypes.c_char_p
        lib.kc_last_cuda_error.argtypes = []
        lib.kc_last_cuda_error.restype = ctypes.c_char_p
        for f in (lib.kc_orient, lib.kc_dag_export, lib.kc_count, lib.kc_count_per_vertex,
                  lib.kc_count_per_arc, lib.kc_dag_get_stats):
            f.restype = I
        _lib = lib
        return lib


def _check(rc: int):
    if rc == KC_OK:
        return
    lib = _load()
    msg = lib.kc_strerror(rc).decode()
    if rc == KC_ECUDA:
        msg += ": " + lib.kc_last_cuda_error().decode()
    cls = KcOverflow if rc == KC_ERANGE else (KcTimeout if rc == KC_ETIMEDOUT else KcError)
    raise cls(rc, msg)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _require_cuda(t: torch.Tensor, name: str, dtypes):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Dag:
    """Handle to an oriented graph owned by the library (freed with the object)."""

    def __init__(self, handle: int, device: torch.device):
        self._h = ctypes.c_void_p(handle)
        self.device = device

    @property
    def handle(self):
        return self._h

    @property
    def n(self) -> int:
        return int(_load().kc_dag_n(self._h))

    @property
    def m(self) -> int:
        return int(_load().kc_dag_m(self._h))

    @property
    def max_out_degree(self) -> int:
        return int(_load().kc_dag_max_out_degree(self._h))

    def export(self, stream=None):
        """(ptr int64[n+1], col int32[m]) device tensors of the out-lists."""
        ptr = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        col = torch.empty(max(self.m, 1), dtype=torch.int32, device=self.device)
        _check(_load().kc_dag_export(self._h, ptr.data_ptr(), col.data_ptr(), _stream(stream)))
        return ptr, col[:self.m]

    def free(self):
        if self._h and self._h.value:
            _load().kc_dag_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kc_orient(row_ptr: torch.Tensor, col: torch.Tensor, n: int | None = None, method: str = "degree",
              validate_symmetry: bool = False, stream=None) -> Dag:
    """Orient(G): rank and direct a simple undirected CSR held in device memory."""
    _require_cuda(row_ptr, "row_ptr", (torch.int64,))
    _require_cuda(col, "col", (torch.int32,))
    n = row_ptr.numel() - 1 if n is None else n
    if row_ptr.numel() != n + 1:
        raise ValueError("row_ptr must have n+1 entries")
    g = _Csr(n, col.numel(), row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0)
    flags = _METHODS[method] | (KC_VALIDATE_SYMMETRY if validate_symmetry else 0)
    h = ctypes.c_void_p()
    _check(_load().kc_orient(ctypes.byref(g), flags, ctypes.byref(h), _stream(stream)))
    return Dag(h.value, row_ptr.device)


def kc_count(dag: Dag, k: int, stream=None) -> int:
    """arb-count: number of k-cliques (exact uint64; raises KcOverflow if it does not fit)."""
    t = ctypes.c_uint64()
    _check(_load().kc_count(dag.handle, int(k), ctypes.byref(t), _stream(stream)))
    return int(t.value)


def kc_count_per_vertex(dag: Dag, k: int, out: torch.Tensor | None = None, stream=None):
    """arb-count-v: (total, out) with out[v] = k-cliques containing v (int64 storage of uint64)."""
    if out is None:
        out = torch.empty(max(dag.n, 1), dtype=torch.int64, device=dag.device)
    _require_cuda(out, "out", (torch.int64,))
    if out.numel() < dag.n:
        raise ValueError("out must have n entries")
    t = ctypes.c_uint64()
    _check(_load().kc_count_per_vertex(dag.handle, int(k), out.data_ptr(), ctypes.byref(t), _stream(stream)))
    return int(t.value), out[:dag.n]


def kc_count_per_arc(dag: Dag, k: int, out: torch.Tensor | None = None, stream=None):
    """(total, out) with out[e] = k-cliques whose two lowest vertices are arc e of the exported DAG."""
    if out is None:
        out = torch.empty(max(dag.m, 1), dtype=torch.int64, device=dag.device)
    _require_cuda(out, "out", (torch.int64,))
    if out.numel() < dag.m:
        raise ValueError("out must have m entries")
    t = ctypes.c_uint64()
    _check(_load().kc_count_per_arc(dag.handle, int(k), out.data_ptr(), ctypes.byref(t), _stream(stream)))
    return int(t.value), out[:dag.m]


def kc_dag_get_stats(dag: Dag, stream=None) -> dict:
    st = _Stats()
    _check(_load().kc_dag_get_stats(dag.handle, ctypes.byref(st), _stream(stream)))
    return {"sum_out_sq": int(st.sum_out_sq), "sum_arc_head": int(st.sum_arc_head),
            "triangles": int(st.triangles), "max_out": int(st.max_out)}


def kc_measure_word_op_rate(stream=None) -> float:
    """Measured 64-bit AND + popcount operations per second on the current device."""
    r = ctypes.c_double()
    _check(_load().kc_measure_word_op_rate(ctypes.byref(r), _stream(stream)))
    return float(r.value)


def kc_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_load().kc_kernel_launches())


# short forms of the spec interface
orient = kc_orient
count = kc_count
count_per_vertex = kc_count_per_vertex
count_per_arc = kc_count_per_arc
dag_stats = kc_dag_get_stats


def csr_to_device(g, device="cuda"):
    """(row_ptr int64, col int32) device tensors of a host CSR with .row_ptr/.col numpy arrays."""
    rp = torch.from_numpy(g.row_ptr.astype("int64", copy=False)).to(device)
    col = torch.from_numpy(g.col.view("int32") if g.col.dtype.name == "uint32" else g.col.astype("int32")).to(device)
    return rp, col


def as_uint64(t: torch.Tensor):
    """Host numpy uint64 view of an int64 tensor holding uint64 counts."""
    return t.detach().cpu().numpy().view("uint64")
