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
KC_ORIENT_BE = 2
KC_VALIDATE_SYMMETRY = 0x100
KC_CORE_BITS = 0x200
KC_NO_CORE_BITS = 0x400
KC_LIGHT_BY_DEGREE = 1
KC_LIGHT_BY_ID = 2
_METHODS = {"degree": KC_ORIENT_DEGREE, "gp": KC_ORIENT_GP, "be": KC_ORIENT_BE}


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


class _Batch(ctypes.Structure):
    _fields_ = [("num_graphs", ctypes.c_uint32), ("d_vertex_offsets", ctypes.c_void_p),
                ("d_k", ctypes.c_void_p), ("k_min", ctypes.c_uint8)]


class _Params(ctypes.Structure):
    _fields_ = [("light_max", ctypes.c_uint32), ("compact_max", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("light_order", ctypes.c_uint32)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("grid_share_pct", ctypes.c_uint32), ("hbm_budget", ctypes.c_uint64)]


class _RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("slot", ctypes.c_int), ("total", ctypes.c_uint64),
                ("queue_ns", ctypes.c_uint64), ("run_ns", ctypes.c_uint64), ("latency_ns", ctypes.c_uint64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "admitted", "completed", "peak_in_flight",
                                                "peak_bytes", "bytes_in_use", "queued")]


class _PeelResult(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("best_rounds", ctypes.c_uint32), ("best_cliques", ctypes.c_uint64),
                ("best_vertices", ctypes.c_uint64), ("total", ctypes.c_uint64)]


class _Stats(ctypes.Structure):
    _fields_ = [("sum_out_sq", ctypes.c_uint64), ("sum_arc_head", ctypes.c_uint64),
                ("triangles", ctypes.c_uint64), ("max_out", ctypes.c_uint32),
                ("core_vertices", ctypes.c_uint32), ("build_scanned", ctypes.c_uint64),
                ("build_lookups", ctypes.c_uint64)]


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
        lib.kc_count_roots.argtypes = [P, I, P, U32, P, P, P]
        lib.kc_count_budget.argtypes = [P, I, P, U64, ctypes.POINTER(U64), P]
        lib.kc_dag_get_stats.argtypes = [P, ctypes.POINTER(_Stats), P]
        BP, PP = ctypes.POINTER(_Batch), ctypes.POINTER(_Params)
        lib.kc_count_batched.argtypes = [P, BP, PP, P, ctypes.POINTER(U64), P]
        lib.kc_plan_create.argtypes = [P, BP, PP, P, ctypes.POINTER(P), P]
        lib.kc_plan_launch.argtypes = [P, P]
        lib.kc_plan_result.argtypes = [P, ctypes.POINTER(U64), P]
        lib.kc_plan_free.argtypes = [P]
        lib.kc_plan_free.restype = None
        lib.kc_autotune_batched.argtypes = [P, BP, P, PP, ctypes.POINTER(ctypes.c_float), P]
        lib.kc_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(P)]
        lib.kc_server_submit.argtypes = [P, P, I, I, U64, ctypes.POINTER(U64)]
        lib.kc_server_wait.argtypes = [P, U64, I, ctypes.POINTER(_RequestResult)]
        lib.kc_server_fetch_per_vertex.argtypes = [P, U64, P, P]
        lib.kc_server_release.argtypes = [P, U64]
        lib.kc_server_get_stats.argtypes = [P, ctypes.POINTER(_ServerStats)]
        lib.kc_server_destroy.argtypes = [P]
        lib.kc_server_destroy.restype = None
        for f in (lib.kc_server_create, lib.kc_server_submit, lib.kc_server_wait, lib.kc_server_fetch_per_vertex,
                  lib.kc_server_release, lib.kc_server_get_stats):
            f.restype = I
        lib.kc_peel.argtypes = [ctypes.POINTER(_Csr), P, I, P, ctypes.POINTER(_PeelResult), P]
        lib.kc_count_colorful.argtypes = [ctypes.POINTER(_Csr), I, U32, U64, I, ctypes.POINTER(U64),
                                          ctypes.POINTER(ctypes.c_double), P]
        lib.kc_count_colorful.restype = I
        lib.kc_peel.restype = I
        lib.kc_peel_approx.argtypes = [ctypes.POINTER(_Csr), P, I, U32, U32, P, ctypes.POINTER(_PeelResult), P]
        lib.kc_peel_approx.restype = I
        lib.kc_checked_sum.argtypes = [P, U64, ctypes.POINTER(U64), P]
        lib.kc_checked_sum.restype = I
        lib.kc_measure_word_op_rate.argtypes = [ctypes.POINTER(ctypes.c_double), P]
        lib.kc_measure_word_op_rate.restype = I
        lib.kc_set_bulk_build.argtypes = [ctypes.c_int]
        lib.kc_set_bulk_build.restype = None
        lib.kc_set_core_policy.argtypes = [U32, U32]
        lib.kc_set_core_policy.restype = None
        lib.kc_dag_core_vertices.argtypes = [P]
        lib.kc_dag_core_vertices.restype = U32
        lib.kc_debug_fail_allocations_after.argtypes = [ctypes.c_int64]
        lib.kc_debug_fail_allocations_after.restype = None
        lib.kc_kernel_launches.argtypes = []
        lib.kc_kernel_launches.restype = U64
        lib.kc_strerror.argtypes = [I]
        lib.kc_strerror.restype = ctypes.c_char_p
        lib.kc_last_cuda_error.argtypes = []
        lib.kc_last_cuda_error.restype = ctypes.c_char_p
        for f in (lib.kc_orient, lib.kc_dag_export, lib.kc_count, lib.kc_count_per_vertex,
                  lib.kc_count_per_arc, lib.kc_count_roots, lib.kc_count_budget, lib.kc_dag_get_stats, lib.kc_count_batched, lib.kc_plan_create,
                  lib.kc_plan_launch, lib.kc_plan_result, lib.kc_autotune_batched):
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

    @property
    def core_vertices(self) -> int:
        """Vertices in the dense core (0: the handle has none)."""
        return int(_load().kc_dag_core_vertices(self._h))

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
              validate_symmetry: bool = False, stream=None, core: bool | None = None) -> Dag:
    """Orient(G): rank and direct a simple undirected CSR held in device memory.
    core: build the dense-core bit matrix always (True), never (False) or where
    it pays (None)."""
    _require_cuda(row_ptr, "row_ptr", (torch.int64,))
    _require_cuda(col, "col", (torch.int32,))
    n = row_ptr.numel() - 1 if n is None else n
    if row_ptr.numel() != n + 1:
        raise ValueError("row_ptr must have n+1 entries")
    g = _Csr(n, col.numel(), row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0)
    flags = _METHODS[method] | (KC_VALIDATE_SYMMETRY if validate_symmetry else 0)
    if core is not None:
        flags |= KC_CORE_BITS if core else KC_NO_CORE_BITS
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


def kc_count_roots(dag: Dag, k: int, roots: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """(total over the roots, out) with out[i] = k-cliques whose lowest vertex is roots[i]
    (roots: int32 device tensor of distinct vertex ids; out: int64 storage of uint64)."""
    _require_cuda(roots, "roots", (torch.int32,))
    r = roots.numel()
    if out is None:
        out = torch.empty(max(r, 1), dtype=torch.int64, device=roots.device)
    _require_cuda(out, "out", (torch.int64,))
    if out.numel() < r:
        raise ValueError("out must have one entry per root")
    t = ctypes.c_uint64()
    _check(_load().kc_count_roots(dag.handle, int(k), roots.data_ptr() if r else None, r,
                                  out.data_ptr(), ctypes.byref(t), _stream(stream)))
    return int(t.value), out[:r]


def kc_count_budget(dag: Dag, k: int, budget_us: int, out: torch.Tensor | None = None, stream=None):
    """A count (out None) or per-vertex count (out: int64 device tensor of n entries) whose pass
    stops with KcTimeout once budget_us microseconds have passed since it started on the GPU."""
    ptr = None
    if out is not None:
        _require_cuda(out, "out", (torch.int64,))
        if out.numel() < dag.n:
            raise ValueError("out must have n entries")
        ptr = out.data_ptr()
    t = ctypes.c_uint64()
    _check(_load().kc_count_budget(dag.handle, int(k), ptr, int(budget_us), ctypes.byref(t), _stream(stream)))
    return int(t.value)


class Batch:
    """A batch of disjoint graphs in one oriented union (kc_batch): graph g owns
    vertices [offsets[g], offsets[g+1]) and counts its ks[g]-cliques."""

    def __init__(self, offsets: torch.Tensor, ks: torch.Tensor):
        _require_cuda(offsets, "offsets", (torch.int64,))
        _require_cuda(ks, "ks", (torch.uint8,))
        if offsets.numel() != ks.numel() + 1 or ks.numel() == 0:
            raise ValueError("offsets must have num_graphs+1 entries, ks num_graphs >= 1")
        self.offsets, self.ks = offsets, ks
        self.num_graphs = ks.numel()
        self.k_min = int(ks.min().item())
        self._c = _Batch(self.num_graphs, offsets.data_ptr(), ks.data_ptr(), self.k_min)

    @property
    def ref(self):
        return ctypes.byref(self._c)


def _params(params):
    if params is None:
        return None
    if isinstance(params, dict):
        params = (params.get("light_max", 0), params.get("compact_max", 0), params.get("chunk", 0),
                  params.get("light_order", 0))
    return ctypes.byref(_Params(*[int(x) for x in params]))


def _totals(batch: Batch, out):
    if out is None:
        out = torch.empty(batch.num_graphs, dtype=torch.int64, device=batch.offsets.device)
    _require_cuda(out, "out", (torch.int64,))
    if out.numel() < batch.num_graphs:
        raise ValueError("out must have num_graphs entries")
    return out


def kc_count_batched(dag: Dag, batch: Batch, params=None, out: torch.Tensor | None = None, stream=None):
    """(sum, out) with out[g] = graph g's ks[g]-clique count (int64 storage of uint64)."""
    out = _totals(batch, out)
    t = ctypes.c_uint64()
    _check(_load().kc_count_batched(dag.handle, batch.ref, _params(params), out.data_ptr(), ctypes.byref(t),
                                    _stream(stream)))
    return int(t.value), out[:batch.num_graphs]


class Plan:
    """kc_plan: a prepared batched pass; launch() only enqueues (capturable)."""

    def __init__(self, dag: Dag, batch: Batch, params=None, out: torch.Tensor | None = None, stream=None):
        self.dag, self.batch = dag, batch  # keep the buffers alive
        self.out = _totals(batch, out)
        h = ctypes.c_void_p()
        _check(_load().kc_plan_create(dag.handle, batch.ref, _params(params), self.out.data_ptr(),
                                      ctypes.byref(h), _stream(stream)))
        self._h = h

    def launch(self, stream=None):
        _check(_load().kc_plan_launch(self._h, _stream(stream)))

    def result(self, stream=None) -> int:
        t = ctypes.c_uint64()
        _check(_load().kc_plan_result(self._h, ctypes.byref(t), _stream(stream)))
        return int(t.value)

    def free(self):
        if self._h and self._h.value:
            _load().kc_plan_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kc_autotune_batched(dag: Dag, batch: Batch, out: torch.Tensor | None = None, stream=None):
    """(params dict, best ms per launch) of the fastest tunables for this batch."""
    out = _totals(batch, out)
    p, ms = _Params(), ctypes.c_float()
    _check(_load().kc_autotune_batched(dag.handle, batch.ref, out.data_ptr(), ctypes.byref(p), ctypes.byref(ms),
                                       _stream(stream)))
    return ({"light_max": int(p.light_max), "compact_max": int(p.compact_max), "chunk": int(p.chunk),
             "light_order": int(p.light_order)}, float(ms.value))


class Server:
    """kc_server: continuous-batching request loop on device-resident DAGs.

    submit() queues a request and returns its id; wait() returns a dict with the
    request's status, total and host-clock times (seconds); per-vertex results
    are fetched with fetch_per_vertex() and then release()d."""

    def __init__(self, slots: int = 8, hbm_budget: int = 8 << 30, grid_share_pct: int = 0):
        cfg = _ServerConfig(int(slots), int(grid_share_pct), int(hbm_budget))
        h = ctypes.c_void_p()
        _check(_load().kc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._dags = {}

    def submit(self, dag: Dag, k: int, per_vertex: bool = False, timeout_us: int = 0) -> int:
        rid = ctypes.c_uint64()
        _check(_load().kc_server_submit(self._h, dag.handle, int(k), 1 if per_vertex else 0, int(timeout_us),
                                        ctypes.byref(rid)))
        self._dags[int(rid.value)] = dag  # keep the DAG alive while the request lives
        return int(rid.value)

    def wait(self, rid: int, timeout_ms: int = -1) -> dict:
        r = _RequestResult()
        _check(_load().kc_server_wait(self._h, int(rid), int(timeout_ms), ctypes.byref(r)))
        return {"status": int(r.status), "slot": int(r.slot), "total": int(r.total), "queue_s": r.queue_ns * 1e-9,
                "run_s": r.run_ns * 1e-9, "latency_s": r.latency_ns * 1e-9}

    def fetch_per_vertex(self, rid: int, out: torch.Tensor, stream=None) -> torch.Tensor:
        if not out.is_contiguous() or out.dtype != torch.int64:
            raise ValueError("out must be a contiguous int64 tensor")
        _check(_load().kc_server_fetch_per_vertex(self._h, int(rid), out.data_ptr(), _stream(stream)))
        return out

    def release(self, rid: int):
        _check(_load().kc_server_release(self._h, int(rid)))
        self._dags.pop(int(rid), None)

    def forget(self, rid: int):
        """Drop the DAG reference of a count request after its wait()."""
        self._dags.pop(int(rid), None)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(_load().kc_server_get_stats(self._h, ctypes.byref(st)))
        return {f: int(getattr(st, f)) for f, _ in _ServerStats._fields_}

    def close(self):
        if self._h and self._h.value:
            _load().kc_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)
            self._dags.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kc_peel(row_ptr: torch.Tensor, col: torch.Tensor, dag: Dag, k: int, out: torch.Tensor | None = None,
            stream=None, epsilon=None):
    """arb-peel (epsilon None) or arb-approx-peel (epsilon >= 0, a float or a
    Fraction, taken as a fraction with denominator <= 2^16): (result dict,
    rounds int32[n]) for the CSR the DAG was oriented from.

    result: rounds, best_rounds, best_cliques, best_vertices (the best density
    is best_cliques / best_vertices, exactly), total."""
    _require_cuda(row_ptr, "row_ptr", (torch.int64,))
    _require_cuda(col, "col", (torch.int32,))
    n = row_ptr.numel() - 1
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=row_ptr.device)
    _require_cuda(out, "out", (torch.int32,))
    g = _Csr(n, col.numel(), row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0)
    res = _PeelResult()
    if epsilon is None:
        _check(_load().kc_peel(ctypes.byref(g), dag.handle, int(k), out.data_ptr(), ctypes.byref(res),
                               _stream(stream)))
    else:
        from fractions import Fraction
        e = Fraction(epsilon).limit_denominator(1 << 16)
        if e < 0:
            raise ValueError("epsilon must be >= 0")
        _check(_load().kc_peel_approx(ctypes.byref(g), dag.handle, int(k), e.numerator, e.denominator,
                                      out.data_ptr(), ctypes.byref(res), _stream(stream)))
    return ({f: int(getattr(res, f)) for f, _ in _PeelResult._fields_}, out[:n])


def kc_count_colorful(row_ptr: torch.Tensor, col: torch.Tensor, k: int, colors: int, seed: int,
                      method: str = "degree", stream=None):
    """Colorful sparsification: (C, estimate) with C the exact k-clique count of
    the monochromatic subgraph and estimate = C * colors^(k-1)."""
    _require_cuda(row_ptr, "row_ptr", (torch.int64,))
    _require_cuda(col, "col", (torch.int32,))
    n = row_ptr.numel() - 1
    g = _Csr(n, col.numel(), row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0)
    c, est = ctypes.c_uint64(), ctypes.c_double()
    _check(_load().kc_count_colorful(ctypes.byref(g), int(k), int(colors), int(seed) & ((1 << 64) - 1),
                                     _METHODS[method], ctypes.byref(c), ctypes.byref(est), _stream(stream)))
    return int(c.value), float(est.value)


def kc_dag_get_stats(dag: Dag, stream=None) -> dict:
    st = _Stats()
    _check(_load().kc_dag_get_stats(dag.handle, ctypes.byref(st), _stream(stream)))
    return {"sum_out_sq": int(st.sum_out_sq), "sum_arc_head": int(st.sum_arc_head),
            "triangles": int(st.triangles), "max_out": int(st.max_out),
            "core_vertices": int(st.core_vertices), "build_scanned": int(st.build_scanned),
            "build_lookups": int(st.build_lookups)}


def kc_checked_sum(values: torch.Tensor, stream=None) -> int:
    """Sum of a device int64 tensor read as uint64, through the counting
    kernels' wrap-checked reduction (raises KcOverflow if it does not fit)."""
    _require_cuda(values, "values", (torch.int64,))
    t = ctypes.c_uint64()
    _check(_load().kc_checked_sum(values.data_ptr() if values.numel() else None, values.numel(), ctypes.byref(t),
                                  _stream(stream)))
    return int(t.value)


def kc_measure_word_op_rate(stream=None) -> float:
    """Measured 64-bit AND + popcount operations per second on the current device."""
    r = ctypes.c_double()
    _check(_load().kc_measure_word_op_rate(ctypes.byref(r), _stream(stream)))
    return float(r.value)


def kc_set_bulk_build(enabled: bool):
    """Block-root builds stage the members' out-lists with bulk copies (True) or read them
    with ordinary loads (False, the default); counts are identical."""
    _load().kc_set_bulk_build(1 if enabled else 0)


def kc_set_core_policy(max_vertices: int = 131072, ratio: int = 1):
    """Dense core: largest core later orientations build (0: none), and the
    lookup rule of later counts (a member's row comes from the core when its
    out-degree is at least ratio times the members after it; 0: always;
    2**32 - 1: never). Counts are identical either way."""
    _load().kc_set_core_policy(int(max_vertices), int(ratio))


def kc_debug_fail_allocations_after(count: int):
    """Tests only: the library's device allocations fail (KC_ENOMEM) after `count` more
    succeed; a negative count switches this off."""
    _load().kc_debug_fail_allocations_after(int(count))


def kc_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_load().kc_kernel_launches())


# short forms of the paper's interface (Algorithm 1: Orient, arb-count)
orient = kc_orient
count = kc_count
count_per_vertex = kc_count_per_vertex
count_per_arc = kc_count_per_arc
count_roots = kc_count_roots
count_budget = kc_count_budget
count_batched = kc_count_batched
peel = kc_peel
count_colorful = kc_count_colorful
autotune_batched = kc_autotune_batched
dag_stats = kc_dag_get_stats


def csr_to_device(g, device="cuda"):
    """(row_ptr int64, col int32) device tensors of a host CSR with .row_ptr/.col numpy arrays."""
    rp = torch.from_numpy(g.row_ptr.astype("int64", copy=False)).to(device)
    col = torch.from_numpy(g.col.view("int32") if g.col.dtype.name == "uint32" else g.col.astype("int32")).to(device)
    return rp, col


def as_uint64(t: torch.Tensor):
    """Host numpy uint64 view of an int64 tensor holding uint64 counts."""
    return t.detach().cpu().numpy().view("uint64")
