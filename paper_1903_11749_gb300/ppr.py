"""Python binding of libppr.so: argument marshalling only.

Every computation runs in the CUDA library behind include/ppr.h; this module
passes pointers and sizes through ctypes and turns status codes into
exceptions.  Host arrays are numpy arrays; device arrays are torch CUDA
tensors (their data pointers are passed with PPR_PTRS_DEVICE).  There is no
fallback: if the library is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PPR_LIBRARY_PATH selects another build of the library (the checked build)
LIB_PATH = os.environ.get("PPR_LIBRARY_PATH") or os.path.join(_HERE, "libppr.so")

PPR_OK, PPR_EINVAL, PPR_ENOMEM, PPR_ECUDA, PPR_ETIMEOUT, PPR_ERANGE, PPR_EBUSY, PPR_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
PPR_PTRS_DEVICE = 1
PPR_RENUMBER = 2
PPR_KEEP_IDS = 4
KERNEL_PERSISTENT, KERNEL_PLAIN = 0, 1
SERVE_DEVICE_LOOP, SERVE_STREAMS = 0, 1
LOOP_STOPPED, LOOP_IDLE, LOOP_SLOT_TIMEOUT, LOOP_BUSY_TIMEOUT = 1, 2, 4, 8
_NAMES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ERANGE", -6: "EBUSY", -7: "ENOTSUP"}


class PPRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class GraphInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("max_degree", C.c_int64), ("dangling", C.c_int64),
                ("wide", C.c_int32), ("instances", C.c_int32), ("device_bytes", C.c_int64),
                ("segment_nodes", C.c_int64), ("segment_entries", C.c_int64), ("renumbered", C.c_int32),
                ("reserved", C.c_int32)]


class RunArgs(C.Structure):
    _fields_ = [("alpha", C.c_double), ("R", C.c_uint32), ("seed", C.c_uint64), ("src_begin", C.c_int64),
                ("src_end", C.c_int64), ("tag", C.c_uint32), ("dangling", C.c_int32), ("segments", C.c_int32),
                ("topk", C.c_int32), ("kernel", C.c_int32), ("large_degree", C.c_int32),
                ("warps_per_block", C.c_int32), ("chunk_sources", C.c_int32), ("max_batch_sources", C.c_int64),
                ("stats", C.c_int32), ("sampler", C.c_int32), ("l2_persist", C.c_int32),
                ("refill_lanes", C.c_int32), ("stream", C.c_void_p), ("step_loads", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("chunk_sources", C.c_int32), ("large_degree", C.c_int32), ("warps_per_block", C.c_int32),
                ("ms", C.c_float), ("candidates", C.c_int32), ("sample_sources", C.c_int64),
                ("refill_lanes", C.c_int32)]


class ServeCfg(C.Structure):
    _fields_ = [("streams", C.c_int32), ("max_sources", C.c_int64), ("max_topk", C.c_int32),
                ("memory_budget", C.c_int64), ("max_pending", C.c_int64), ("chunk_sources", C.c_int32),
                ("large_degree", C.c_int32), ("warps_per_block", C.c_int32), ("sampler", C.c_int32),
                ("refill_lanes", C.c_int32), ("mode", C.c_int32), ("idle_us", C.c_int64)]


class ServeInfo(C.Structure):
    _fields_ = [("mode", C.c_int32), ("status", C.c_uint32), ("launches", C.c_int64), ("idle_exits", C.c_int64),
                ("in_flight", C.c_int64), ("completed", C.c_int64), ("running", C.c_int32),
                ("draws", C.c_uint64), ("iterations", C.c_uint64), ("claims", C.c_uint64),
                ("claim_misses", C.c_uint64), ("sleeps", C.c_uint64), ("reduced", C.c_uint64),
                ("cycles_claim", C.c_uint64), ("cycles_step", C.c_uint64), ("cycles_sleep", C.c_uint64),
                ("cycles_total", C.c_uint64), ("grid_blocks", C.c_int32)]


class QueryStats(C.Structure):
    _fields_ = [("submit_ns", C.c_int64), ("admit_ns", C.c_int64), ("done_ns", C.c_int64), ("walks", C.c_uint64),
                ("sources", C.c_int64), ("device_walk_ns", C.c_int64), ("device_reduce_ns", C.c_int64)]


class ResultInfo(C.Structure):
    _fields_ = [("sources", C.c_int64), ("R", C.c_uint32), ("topk", C.c_int32), ("nnz", C.c_int64),
                ("steps", C.c_uint64), ("walks", C.c_uint64), ("kernel_ms", C.c_float), ("sectors", C.c_uint64),
                ("run_ms", C.c_float), ("model_sectors", C.c_uint64)]


# Every symbol include/ppr.h declares, with its ctypes signature.
_SIGS = {
    "ppr_version": (C.c_int, []),
    "ppr_alpha_threshold": (C.c_uint32, [C.c_double]),
    "ppr_walks_for_accuracy": (C.c_int, [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_uint64)]),
    "ppr_last_error": (C.c_char_p, []),
    "ppr_kernel_launches": (C.c_int64, []),
    "ppr_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "ppr_destroy": (None, [C.c_void_p]),
    "ppr_device_sms": (C.c_int, [C.c_void_p]),
    "ppr_load_graph": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32,
                                 C.c_void_p, C.POINTER(C.c_void_p)]),
    "ppr_load_graph_batch": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_uint32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "ppr_graph_get_info": (C.c_int, [C.c_void_p, C.POINTER(GraphInfo)]),
    "ppr_free_graph": (None, [C.c_void_p]),
    "ppr_run_args_init": (None, [C.POINTER(RunArgs)]),
    "ppr_run": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RunArgs), C.POINTER(C.c_void_p)]),
    "ppr_wait": (C.c_int, [C.c_void_p, C.c_int64]),
    "ppr_result_get_info": (C.c_int, [C.c_void_p, C.POINTER(ResultInfo)]),
    "ppr_sparse_rows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.POINTER(C.c_int64), C.c_uint32]),
    "ppr_topk": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_uint32]),
    "ppr_dense": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32]),
    "ppr_free_result": (None, [C.c_void_p]),
    "ppr_run_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RunArgs), C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_uint32, C.c_void_p, C.c_void_p]),
    "ppr_run_list": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RunArgs), C.c_void_p, C.c_int64,
                               C.POINTER(C.c_void_p)]),
    "ppr_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(RunArgs), C.POINTER(C.c_size_t)]),
    "ppr_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RunArgs), C.c_int64, C.POINTER(Tuning)]),
    "ppr_serve_cfg_init": (None, [C.POINTER(ServeCfg)]),
    "ppr_serve_start": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(ServeCfg)]),
    "ppr_serve_stop": (C.c_int, [C.c_void_p]),
    "ppr_serve_get_info": (C.c_int, [C.c_void_p, C.POINTER(ServeInfo)]),
    "ppr_debug_serve_publish_unwritten": (C.c_int, [C.c_void_p]),
    "ppr_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_uint32, C.c_uint64, C.c_int32,
                             C.POINTER(C.c_uint64)]),
    "ppr_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(QueryStats)]),
    "ppr_debug_fail_allocs": (None, [C.c_int64]),
    "ppr_probe_philox": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p]),
    "ppr_probe_rate": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "ppr_run_to_host": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RunArgs), C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p,
                                  C.POINTER(ResultInfo)]),
    "ppr_run_into": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RunArgs), C.c_void_p, C.c_size_t, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1903_11749_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != PPR_OK:
        raise PPRError(rc, lib().ppr_last_error().decode(errors="replace"))


def kernel_launches() -> int:
    return int(lib().ppr_kernel_launches())


def alpha_threshold(alpha: float) -> int:
    return int(lib().ppr_alpha_threshold(alpha))


def debug_fail_allocs(after: int) -> None:
    """Test hook: device allocations fail with PPR_ENOMEM after `after` more (negative: off)."""
    lib().ppr_debug_fail_allocs(after)


def walks_for_accuracy(eps: float, delta: float, p_f: float) -> int:
    out = C.c_uint64()
    _check(lib().ppr_walks_for_accuracy(eps, delta, p_f, C.byref(out)))
    return out.value


def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr(), a.is_cuda
    raise TypeError(type(a))


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


class Context:
    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().ppr_create(device, C.byref(h)))
        self.h = h
        self.device = device

    @property
    def sms(self) -> int:
        return lib().ppr_device_sms(self.h)

    def close(self):
        if self.h:
            lib().ppr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- serving
    def probe_philox(self, seed: int, counter, count: int) -> np.ndarray:
        """Device Philox4x32-10 words uint32[count, 4] for counters (c0 + i, c1, c2, c3)."""
        ctr = np.ascontiguousarray(counter, dtype=np.uint32)
        out = np.empty((count, 4), dtype=np.uint32)
        _check(lib().ppr_probe_philox(self.h, seed, ctr.ctypes.data, count, out.ctypes.data))
        return out

    def probe_rate(self, kind: int, nbytes: int = 0):
        """(units per second, kernel ms): kind 0 dependent random 32-byte sector
        reads over nbytes, kind 1 Philox draws, kind 2 independent random
        32-byte sector reads over nbytes."""
        v = C.c_double()
        ms = C.c_float()
        _check(lib().ppr_probe_rate(self.h, kind, nbytes, C.byref(v), C.byref(ms)))
        return v.value, ms.value

    def serve_start(self, graph: "Graph", **cfg):
        c = ServeCfg()
        lib().ppr_serve_cfg_init(C.byref(c))
        for k_, v in cfg.items():
            setattr(c, k_, v)
        _check(lib().ppr_serve_start(self.h, graph.h, C.byref(c)))
        self._serving = graph

    def serve_stop(self):
        _check(lib().ppr_serve_stop(self.h))

    def serve_info(self) -> dict:
        i = ServeInfo()
        _check(lib().ppr_serve_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in ServeInfo._fields_}

    def debug_serve_publish_unwritten(self):
        """Test hook: publishes a ring slot the host never wrote (see include/ppr.h)."""
        _check(lib().ppr_debug_serve_publish_unwritten(self.h))
        self._serving = None

    def submit(self, sources, alpha=0.15, R=100, seed=1, topk=32) -> int:
        src = np.ascontiguousarray(sources, dtype=np.int32)
        q = C.c_uint64()
        _check(lib().ppr_submit(self.h, src.ctypes.data, len(src), alpha, R, seed, topk, C.byref(q)))
        return q.value

    def poll(self, qid: int, ns: int, topk: int, timeout_ms: int = -1):
        """(idx int32[ns, topk], cnt uint32[ns, topk], stats dict) of a finished query."""
        idx = np.zeros((ns, topk), dtype=np.int32)
        cnt = np.zeros((ns, topk), dtype=np.uint32)
        st = QueryStats()
        _check(lib().ppr_poll(self.h, qid, idx.ctypes.data, cnt.ctypes.data, timeout_ms, C.byref(st)))
        return idx, cnt, {"submit_ns": st.submit_ns, "admit_ns": st.admit_ns, "done_ns": st.done_ns,
                          "walks": st.walks, "sources": st.sources, "device_walk_ns": st.device_walk_ns,
                          "device_reduce_ns": st.device_reduce_ns}

    def load_graph(self, n, row_ptr, col, w, stream=None, m=None, renumber=None) -> "Graph":
        """renumber: None lets the library decide (by the layout's size against
        L2), True / False force PPR_RENUMBER / PPR_KEEP_IDS."""
        rp, dev = _ptr(row_ptr)
        cp, dev2 = _ptr(col)
        wp, dev3 = _ptr(w)
        if not (dev == dev2 == dev3):
            raise ValueError("row_ptr, col and w must all be host arrays or all device tensors")
        if m is None:
            m = int(row_ptr[-1]) if not dev else int(row_ptr[-1].item())
        flags = PPR_PTRS_DEVICE if dev else 0
        if renumber is not None:
            flags |= PPR_RENUMBER if renumber else PPR_KEEP_IDS
        h = C.c_void_p()
        _check(lib().ppr_load_graph(self.h, n, m, rp, cp, wp, flags, _stream_ptr(stream), C.byref(h)))
        return Graph(self, h)

    def load_graph_batch(self, node_off, row_ptr, col, w, stream=None) -> "Graph":
        node_off = np.ascontiguousarray(node_off, dtype=np.int64)
        rp, dev = _ptr(row_ptr)
        cp, _ = _ptr(col)
        wp, _ = _ptr(w)
        m = int(row_ptr[-1]) if not dev else int(row_ptr[-1].item())
        h = C.c_void_p()
        _check(lib().ppr_load_graph_batch(self.h, len(node_off) - 1, node_off.ctypes.data, m, rp, cp, wp,
                                          PPR_PTRS_DEVICE if dev else 0, _stream_ptr(stream), C.byref(h)))
        return Graph(self, h)


class Graph:
    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def info(self) -> GraphInfo:
        gi = GraphInfo()
        _check(lib().ppr_graph_get_info(self.h, C.byref(gi)))
        return gi

    def free(self):
        if self.h:
            lib().ppr_free_graph(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _args(self, alpha=0.15, R=100, seed=1, src_begin=0, src_end=None, tag=0, dangling=0, segments=False,
              topk=0, kernel=KERNEL_PERSISTENT, large_degree=0, warps_per_block=0, chunk_sources=0,
              max_batch_sources=0, stats=False, stream=None, sampler=0, l2_persist=0, refill_lanes=0, step_loads=0):
        a = RunArgs()
        lib().ppr_run_args_init(C.byref(a))
        a.alpha, a.R, a.seed = alpha, R, seed
        a.src_begin = src_begin
        a.src_end = self.info().n if src_end is None else src_end
        a.tag, a.dangling, a.segments, a.topk, a.kernel = tag, dangling, int(bool(segments)), topk, kernel
        a.large_degree, a.warps_per_block, a.chunk_sources = large_degree, warps_per_block, chunk_sources
        a.max_batch_sources = max_batch_sources
        a.stats = int(bool(stats))
        a.sampler = sampler
        a.l2_persist = l2_persist
        a.refill_lanes = refill_lanes
        a.step_loads = step_loads
        a.stream = _stream_ptr(stream)
        return a

    def run_list(self, sources, wait=True, **kw) -> "Result":
        """Walks from an explicit list of source ids; row i belongs to sources[i]."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        a = self._args(**kw)
        h = C.c_void_p()
        _check(lib().ppr_run_list(self.ctx.h, self.h, C.byref(a), src.ctypes.data, len(src), C.byref(h)))
        r = Result(self, h, len(src), kw.get("topk", 0))
        if wait:
            r.wait()
        return r

    def autotune(self, sample_sources=0, **kw) -> dict:
        a = self._args(**kw)
        t = Tuning()
        _check(lib().ppr_autotune(self.ctx.h, self.h, C.byref(a), sample_sources, C.byref(t)))
        return {"chunk_sources": t.chunk_sources, "large_degree": t.large_degree,
                "warps_per_block": t.warps_per_block, "refill_lanes": t.refill_lanes, "ms": t.ms,
                "candidates": t.candidates, "sample_sources": t.sample_sources}

    def workspace_size(self, **kw) -> int:
        a = self._args(**kw)
        n = C.c_size_t()
        _check(lib().ppr_workspace_size(self.h, C.byref(a), C.byref(n)))
        return n.value

    def run_to_host(self, row_ptr, col, cnt, topk_idx=None, topk_cnt=None, parts=0, **kw):
        """Runs a source range and writes rows (and top-k) into host arrays,
        output copies pipelined against the walks; returns (nnz, info)."""
        a = self._args(**kw)
        for arr in (row_ptr, col, cnt, topk_idx, topk_cnt):
            if arr is not None and _ptr(arr)[1]:
                raise ValueError("run_to_host writes host memory")
        ti = _ptr(topk_idx)[0] if topk_idx is not None else None
        tc = _ptr(topk_cnt)[0] if topk_cnt is not None else None
        cap = col.shape[0] if hasattr(col, "shape") else len(col)
        nnz = C.c_int64()
        info = ResultInfo()
        _check(lib().ppr_run_to_host(self.ctx.h, self.h, C.byref(a), parts, _ptr(row_ptr)[0], _ptr(col)[0],
                                     _ptr(cnt)[0], cap, C.byref(nnz), ti, tc, C.byref(info)))
        return nnz.value, info

    def run_into(self, workspace, nnz, cols, cnts, cap, topk_idx=None, topk_cnt=None, **kw):
        """Enqueues a run into caller-owned device tensors (no allocation; capturable)."""
        a = self._args(**kw)
        ti = _ptr(topk_idx)[0] if topk_idx is not None else None
        tc = _ptr(topk_cnt)[0] if topk_cnt is not None else None
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().ppr_run_into(self.ctx.h, self.h, C.byref(a), _ptr(workspace)[0], nbytes, _ptr(nnz)[0],
                                  _ptr(cols)[0], _ptr(cnts)[0], cap, ti, tc))

    def run(self, wait=True, **kw) -> "Result":
        """Walks from every source of [src_begin, src_end) (default: all); takes
        the arguments of ppr_run_args by name (include/ppr.h)."""
        a = self._args(**kw)
        h = C.c_void_p()
        _check(lib().ppr_run(self.ctx.h, self.h, C.byref(a), C.byref(h)))
        r = Result(self, h, a.src_end - a.src_begin, kw.get("topk", 0))
        if wait:
            r.wait()
        return r

    def run_noalloc(self, nnz, cols, cnts, cap, topk_idx=None, topk_cnt=None, **kw):
        """Allocation-free run into caller-owned device tensors (see ppr_run_noalloc in include/ppr.h);
        takes the arguments of run(); returns once the work is queued on `stream`."""
        a = self._args(**kw)
        ti = _ptr(topk_idx)[0] if topk_idx is not None else None
        tc = _ptr(topk_cnt)[0] if topk_cnt is not None else None
        _check(lib().ppr_run_noalloc(self.ctx.h, self.h, C.byref(a), _ptr(nnz)[0], _ptr(cols)[0], _ptr(cnts)[0],
                                     cap, ti, tc))


class Result:
    def __init__(self, graph: Graph, h, S: int, topk: int):
        self.graph = graph
        self.h = h
        self.S = S
        self.topk_k = topk

    def wait(self, timeout_ms: int = -1):
        _check(lib().ppr_wait(self.h, timeout_ms))
        return self

    def info(self) -> ResultInfo:
        ri = ResultInfo()
        _check(lib().ppr_result_get_info(self.h, C.byref(ri)))
        return ri

    def nnz(self) -> int:
        n = C.c_int64()
        _check(lib().ppr_sparse_rows(self.h, None, None, None, 0, C.byref(n), 0))
        return n.value

    def sparse_rows(self):
        """(row_ptr int64[S+1], col int32[nnz], cnt uint32[nnz]) as numpy arrays."""
        row_ptr = np.zeros(self.S + 1, dtype=np.int64)
        n = C.c_int64()
        _check(lib().ppr_sparse_rows(self.h, row_ptr.ctypes.data, None, None, 0, C.byref(n), 0))
        col = np.zeros(max(n.value, 1), dtype=np.int32)
        cnt = np.zeros(max(n.value, 1), dtype=np.uint32)
        _check(lib().ppr_sparse_rows(self.h, row_ptr.ctypes.data, col.ctypes.data, cnt.ctypes.data, len(col),
                                     C.byref(n), 0))
        return row_ptr, col[: n.value], cnt[: n.value]

    def sparse_rows_into(self, row_ptr, col, cnt) -> int:
        """Fills caller buffers (numpy host arrays or torch device tensors)."""
        rp, dev = _ptr(row_ptr)
        cp, _ = _ptr(col)
        kp, _ = _ptr(cnt)
        n = C.c_int64()
        _check(lib().ppr_sparse_rows(self.h, rp, cp, kp, int(col.shape[0]), C.byref(n), PPR_PTRS_DEVICE if dev else 0))
        return n.value

    def topk(self, k: int | None = None):
        k = self.topk_k if k is None else k
        idx = np.zeros((self.S, k), dtype=np.int32)
        cnt = np.zeros((self.S, k), dtype=np.uint32)
        _check(lib().ppr_topk(self.h, k, idx.ctypes.data, cnt.ctypes.data, 0))
        return idx, cnt

    def topk_into(self, k: int, idx, cnt):
        ip, dev = _ptr(idx)
        cp, _ = _ptr(cnt)
        _check(lib().ppr_topk(self.h, k, ip, cp, PPR_PTRS_DEVICE if dev else 0))

    def dense(self):
        n = self.graph.info().n
        out = np.zeros((self.S, n), dtype=np.uint32)
        _check(lib().ppr_dense(self.h, out.ctypes.data, 0))
        return out

    def free(self):
        if self.h:
            lib().ppr_free_result(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
