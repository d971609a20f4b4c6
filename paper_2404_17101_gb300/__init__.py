"""Python binding of the GB300 frontier-traversal library (libpasgal_gb.so).

Argument marshalling only: every step of the traversal runs in the CUDA
kernels behind the C ABI declared in include/pasgal.h.  PyTorch is used for
device memory and streams.  There is no CPU fallback: if the shared library
or a CUDA device is missing, every call raises.

    g = Graph.upload(offsets, indices, directed=False)   # numpy or torch
    dist = g.bfs(src)                       # torch.int32 view of uint32 on cuda
    fwd, bwd = g.reach_multi(sources, PG_FWD | PG_BWD)   # torch.int64 views
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpasgal_gb.so")

PG_OK, PG_ERR_INVALID_ARG, PG_ERR_INVALID_GRAPH, PG_ERR_OOM = 0, 1, 2, 3
PG_ERR_CUDA, PG_ERR_TIMEOUT, PG_ERR_UNSUPPORTED, PG_ERR_OVERFLOW = 4, 5, 6, 7
STATUS_NAMES = {0: "PG_OK", 1: "PG_ERR_INVALID_ARG", 2: "PG_ERR_INVALID_GRAPH", 3: "PG_ERR_OOM",
                4: "PG_ERR_CUDA", 5: "PG_ERR_TIMEOUT", 6: "PG_ERR_UNSUPPORTED",
                7: "PG_ERR_OVERFLOW"}
PG_DIRECTED, PG_BUILD_TRANSPOSE, PG_SKIP_VALIDATE, PG_ELL = 1, 2, 4, 8
PG_FWD, PG_BWD = 1, 2
PG_SCHED_FIXED, PG_SCHED_LEARNED, PG_SCHED_RANDOM, PG_SCHED_SCRIPT = 0, 1, 2, 3
PG_DIR_PUSH, PG_DIR_AUTO = 0, 1
PG_VGC_CTA, PG_VGC_WARP, PG_VGC_BUCKETS = 0, 1, 2
PG_NUM_ACTIONS, PG_ACTION_PULL = 8, 7
PG_MLP_NPARAMS = 1512
INF = 0xFFFFFFFF

# every symbol include/pasgal.h declares
EXPORTS = ["pg_config_default", "pg_graph_upload", "pg_graph_set_transpose", "pg_graph_free",
           "pg_graph_info", "pg_bfs", "pg_reach_multi", "pg_bfs_multi", "pg_count_reached",
           "pg_set_schedule_weights", "pg_mlp_forward", "pg_mlp_backward", "pg_mlp_adam",
           "pg_autotune", "pg_bfs_noalloc", "pg_scc", "pg_probe_barrier", "pg_graph_set_weights",
           "pg_sssp", "pg_last_error", "pg_version"]
NOALLOC_MAX_N = 1 << 20


class PgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class RoundTrace(ctypes.Structure):
    _fields_ = [("round", ctypes.c_uint32), ("action", ctypes.c_uint32),
                ("frontier", ctypes.c_uint32), ("min_level", ctypes.c_uint32),
                ("out_edges", ctypes.c_uint64), ("t_begin_ns", ctypes.c_uint64),
                ("t_end_ns", ctypes.c_uint64), ("settled", ctypes.c_uint64),
                ("features", ctypes.c_float * 5), ("reserved", ctypes.c_uint32)]


class Config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("schedule", ctypes.c_uint32),
                ("tau", ctypes.c_uint32), ("direction", ctypes.c_uint32),
                ("alpha", ctypes.c_uint32), ("beta", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("threads_per_block", ctypes.c_uint32),
                ("local_queue", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("hub_degree", ctypes.c_uint32), ("timeout_ms", ctypes.c_uint32),
                ("max_rounds", ctypes.c_uint32), ("seed", ctypes.c_uint32),
                ("script_len", ctypes.c_uint32), ("trace_cap", ctypes.c_uint32),
                ("test_stall_block", ctypes.c_uint32), ("vgc_mode", ctypes.c_uint32),
                ("cta_queue", ctypes.c_uint32), ("delta", ctypes.c_uint32),
                ("script", ctypes.c_void_p), ("trace_out", ctypes.POINTER(RoundTrace)),
                ("ref_dist", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("pull_rounds", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("expansions", ctypes.c_uint64), ("pushes", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_float), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str | None = None):
    """Load the shared library (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(p)
    vp, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    P = ctypes.POINTER
    sigs = {
        "pg_config_default": (None, [P(Config)]),
        "pg_graph_upload": (ctypes.c_int, [vp, vp, u32, u32, u32, vp, P(vp)]),
        "pg_graph_set_transpose": (ctypes.c_int, [vp, vp, vp, vp]),
        "pg_graph_free": (ctypes.c_int, [vp]),
        "pg_graph_info": (ctypes.c_int, [vp, P(u32), P(u32), P(u32)]),
        "pg_bfs": (ctypes.c_int, [vp, u32, vp, P(Config), P(Stats), vp]),
        "pg_reach_multi": (ctypes.c_int, [vp, vp, u32, u32, vp, vp, P(Config), P(Stats), vp]),
        "pg_bfs_multi": (ctypes.c_int, [vp, vp, u32, vp, P(Config), P(Stats), vp]),
        "pg_count_reached": (ctypes.c_int, [vp, vp, P(u64), P(u64), vp]),
        "pg_set_schedule_weights": (ctypes.c_int, [vp, vp, sz]),
        "pg_mlp_forward": (ctypes.c_int, [vp, vp, u32, vp, vp]),
        "pg_mlp_backward": (ctypes.c_int, [vp, vp, vp, vp, u32, vp, vp, vp]),
        "pg_mlp_adam": (ctypes.c_int, [vp, vp, vp, vp, u32, u32, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, vp]),
        "pg_autotune": (ctypes.c_int, [vp, u32, vp, u32, u32, u32, P(Config), vp]),
        "pg_bfs_noalloc": (ctypes.c_int, [vp, vp, u32, u32, u32, vp, P(Config), vp]),
        "pg_scc": (ctypes.c_int, [vp, vp, P(Config), P(Stats), P(u32), vp]),
        "pg_probe_barrier": (ctypes.c_int, [u32, u32, u32, P(ctypes.c_float), vp]),
        "pg_graph_set_weights": (ctypes.c_int, [vp, vp, vp]),
        "pg_sssp": (ctypes.c_int, [vp, u32, vp, P(Config), P(Stats), vp]),
        "pg_last_error": (ctypes.c_char_p, []),
        "pg_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != PG_OK:
        raise PgError(rc, load().pg_last_error().decode())


def default_config(**kw) -> Config:
    c = Config()
    load().pg_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _u32_array(x):
    """numpy uint32 view or CUDA tensor -> (pointer, keepalive)."""
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype not in (torch.int32, torch.uint32) or not x.is_contiguous():
            raise TypeError("expected a contiguous int32/uint32 tensor")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=np.uint32)
    return ctypes.c_void_p(a.ctypes.data), a


def _buf(t, count, what, torch_dtypes, np_dtype, device=None, cuda_only=False, writes=True):
    """Pointer to a caller-given buffer of at least `count` elements.

    The C ABI sees raw pointers and no sizes, so a short, strided or
    wrongly typed buffer would be read or written past its end by a kernel.
    Checked here, before anything is launched (ValueError): the element
    type, contiguity, size, and for a CUDA tensor the device the graph
    lives on (`device`; None skips the check).  Host buffers (numpy arrays,
    CPU tensors) are staged and copied by the library unless `cuda_only`."""
    import torch
    if isinstance(t, torch.Tensor):
        if t.dtype not in torch_dtypes:
            raise ValueError(f"{what}: dtype {t.dtype}, expected {' or '.join(map(str, torch_dtypes))}")
        if not t.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        if t.numel() < count:
            raise ValueError(f"{what}: {t.numel()} elements, fewer than the {count} needed")
        if cuda_only and not t.is_cuda:
            raise ValueError(f"{what}: must be a CUDA tensor")
        if t.is_cuda and device is not None and t.device.index != device:
            raise ValueError(f"{what}: tensor on cuda:{t.device.index}, the graph is on cuda:{device}")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray) and not cuda_only:
        if t.dtype != np_dtype:
            raise ValueError(f"{what}: dtype {t.dtype}, expected {np.dtype(np_dtype)}")
        if not t.flags.c_contiguous or (writes and not t.flags.writeable):
            raise ValueError(f"{what}: array must be C-contiguous" + (" and writeable" if writes else ""))
        if t.size < count:
            raise ValueError(f"{what}: {t.size} elements, fewer than the {count} needed")
        return ctypes.c_void_p(t.ctypes.data)
    raise ValueError(f"{what}: expected a {'CUDA tensor' if cuda_only else 'torch tensor or numpy array'}, "
                     f"got {type(t).__name__}")


def _u32_types():
    import torch
    return (torch.int32, torch.uint32)


def _u64_types():
    import torch
    return (torch.int64, torch.uint64)


def _f32_types():
    import torch
    return (torch.float32,)


class Graph:
    """A graph resident on the CUDA device that was current at upload."""

    def __init__(self, handle, n, m, directed, device=None):
        self._h = handle
        self.n, self.m, self.directed = n, m, directed
        self.device = device  # CUDA device index (None: not checked)

    def _cuda(self) -> str:
        """Where outputs the binding allocates go: the graph's device."""
        return "cuda" if self.device is None else f"cuda:{self.device}"

    @classmethod
    def upload(cls, offsets, indices, directed: bool = False, transpose: bool = True,
               validate: bool = True, ell: bool = False, stream=None) -> "Graph":
        """Copy a CSR (numpy host arrays or CUDA tensors) into library-owned memory."""
        lib = load()
        po, ko = _u32_array(offsets)
        pi, ki = _u32_array(indices)
        n = int(len(ko)) - 1
        m = int(len(ki))
        flags = (PG_DIRECTED if directed else 0) | (PG_BUILD_TRANSPOSE if (directed and transpose) else 0)
        if not validate:
            flags |= PG_SKIP_VALIDATE
        if ell:
            flags |= PG_ELL
        h = ctypes.c_void_p()
        import torch
        dev = torch.cuda.current_device()
        _check(lib.pg_graph_upload(po, pi, n, m, flags, _stream_ptr(stream), ctypes.byref(h)))
        return cls(h, n, m, directed, device=dev)

    @classmethod
    def from_graphgen(cls, g, **kw) -> "Graph":
        return cls.upload(g.offsets, g.indices, directed=g.directed, **kw)

    def free(self):
        if self._h:
            load().pg_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        n, m, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(load().pg_graph_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(f)))
        return n.value, m.value, f.value

    # ---------------------------------------------------------- traversals
    def bfs(self, src: int, out=None, cfg: Config | None = None, stats: Stats | None = None,
            stream=None):
        """Exact hop distances from src; returns a CUDA int32 tensor (uint32 bits)."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device=self._cuda())
        ptr = _buf(out, self.n, "bfs: out", _u32_types(), np.uint32, self.device)
        _check(load().pg_bfs(self._h, int(src), ptr, ctypes.byref(cfg) if cfg else None,
                             ctypes.byref(stats) if stats else None, _stream_ptr(stream)))
        return out

    def bfs_host(self, src: int, out: np.ndarray, cfg: Config | None = None, stream=None):
        """pg_bfs with a host output buffer (the library stages and copies back)."""
        if not isinstance(out, np.ndarray):
            raise ValueError("bfs_host: out must be a numpy uint32 array")
        ptr = _buf(out, self.n, "bfs_host: out", _u32_types(), np.uint32)
        _check(load().pg_bfs(self._h, int(src), ptr,
                             ctypes.byref(cfg) if cfg else None, None, _stream_ptr(stream)))
        return out

    def reach_multi(self, sources, direction: int = PG_FWD, cfg: Config | None = None,
                    stats: Stats | None = None, stream=None):
        """Per-vertex uint64 source bitmasks (int64 CUDA tensors); (fwd, bwd)."""
        import torch
        src = np.ascontiguousarray(sources, dtype=np.uint32)
        fwd = torch.empty(self.n, dtype=torch.int64, device=self._cuda()) if direction & PG_FWD else None
        bwd = torch.empty(self.n, dtype=torch.int64, device=self._cuda()) if direction & PG_BWD else None
        _check(load().pg_reach_multi(self._h, ctypes.c_void_p(src.ctypes.data), len(src), direction,
                                     ctypes.c_void_p(fwd.data_ptr() if fwd is not None else 0),
                                     ctypes.c_void_p(bwd.data_ptr() if bwd is not None else 0),
                                     ctypes.byref(cfg) if cfg else None,
                                     ctypes.byref(stats) if stats else None, _stream_ptr(stream)))
        return fwd, bwd

    def bfs_multi(self, sources, cfg: Config | None = None, stats: Stats | None = None,
                  stream=None, out=None):
        """k x n hop distances (int32 CUDA tensor, uint32 bits), source-major."""
        import torch
        src = np.ascontiguousarray(sources, dtype=np.uint32)
        if out is None:
            out = torch.empty((len(src), self.n), dtype=torch.int32, device=self._cuda())
        ptr = _buf(out, len(src) * self.n, "bfs_multi: out", _u32_types(), np.uint32, self.device,
                   cuda_only=True)
        _check(load().pg_bfs_multi(self._h, ctypes.c_void_p(src.ctypes.data), len(src), ptr,
                                   ctypes.byref(cfg) if cfg else None,
                                   ctypes.byref(stats) if stats else None, _stream_ptr(stream)))
        return out

    def scc(self, out=None, cfg: Config | None = None, stats: Stats | None = None, stream=None):
        """SCC labels (smallest vertex id of each component) as a CUDA int32
        tensor (uint32 bits), and the number of pivot iterations."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device=self._cuda())
        # a host output (numpy array) is staged and copied back by the library
        ptr = _buf(out, self.n, "scc: out", _u32_types(), np.uint32, self.device)
        it = ctypes.c_uint32()
        _check(load().pg_scc(self._h, ptr, ctypes.byref(cfg) if cfg else None,
                             ctypes.byref(stats) if stats else None, ctypes.byref(it), _stream_ptr(stream)))
        return out, it.value

    def set_weights(self, weights, stream=None):
        """Arc weights for sssp: uint32, one per arc of the forward CSR (numpy
        or CUDA tensor)."""
        p, keep = _u32_array(weights)
        n_w = keep.numel() if hasattr(keep, "numel") else len(keep)
        if n_w != self.m:
            raise ValueError(f"set_weights: {n_w} weights for {self.m} arcs")
        _check(load().pg_graph_set_weights(self._h, p, _stream_ptr(stream)))

    def sssp(self, src: int, out=None, cfg: Config | None = None, stats: Stats | None = None,
             stream=None):
        """Shortest-path distances from src (needs set_weights); returns a CUDA
        int64 tensor holding uint64 bits (0xFFFFFFFFFFFFFFFF: unreachable)."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.int64, device=self._cuda())
        ptr = _buf(out, self.n, "sssp: out", _u64_types(), np.uint64, self.device)
        _check(load().pg_sssp(self._h, int(src), ptr, ctypes.byref(cfg) if cfg else None,
                              ctypes.byref(stats) if stats else None, _stream_ptr(stream)))
        return out

    def count_reached(self, dist, stream=None):
        """(n_r, m_r) of a device distance vector: reached vertices and the
        sum of their out-degrees."""
        ptr = _buf(dist, self.n, "count_reached: dist", _u32_types(), np.uint32, self.device,
                   cuda_only=True, writes=False)
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().pg_count_reached(self._h, ptr, ctypes.byref(a),
                                       ctypes.byref(b), _stream_ptr(stream)))
        return a.value, b.value

    def set_transpose(self, t_offsets, t_indices, stream=None):
        """Replace the reversed CSR (host numpy arrays or CUDA tensors, uint32)."""
        ptrs = []
        for a, count, what in ((t_offsets, self.n + 1, "set_transpose: t_offsets"),
                               (t_indices, self.m, "set_transpose: t_indices")):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.uint32)
            ptrs.append((a, _buf(a, count, what, _u32_types(), np.uint32, self.device, writes=False)))
        _check(load().pg_graph_set_transpose(self._h, ptrs[0][1], ptrs[1][1], _stream_ptr(stream)))

    def set_schedule_weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().pg_set_schedule_weights(self._h, ctypes.c_void_p(a.ctypes.data), a.size))

    def autotune(self, sources, kind: int = 0, direction: int = PG_FWD, trials: int = 3,
                 cfg: Config | None = None, stream=None) -> Config:
        c = cfg if cfg is not None else default_config()
        src = np.ascontiguousarray(sources, dtype=np.uint32)
        _check(load().pg_autotune(self._h, kind, ctypes.c_void_p(src.ctypes.data), len(src),
                                  direction, trials, ctypes.byref(c), _stream_ptr(stream)))
        return c


def to_uint32(t) -> np.ndarray:
    """CUDA int32 tensor holding uint32 bits -> numpy uint32."""
    return t.cpu().numpy().view(np.uint32)


def to_uint64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


# ------------------------------------------------------------- MLP kernels
PG_MLP_IN = 5


def _mlp_inputs(params, X):
    """Shape, type and device checks of the network's parameters and
    feature rows (X: B x PG_MLP_IN fp32); returns (B, device index)."""
    if not (hasattr(X, "dim") and X.dim() == 2 and X.shape[1] == PG_MLP_IN):
        raise ValueError(f"X must be a B x {PG_MLP_IN} tensor")
    dev = X.device.index
    _buf(params, PG_MLP_NPARAMS, "params", _f32_types(), np.float32, dev, cuda_only=True, writes=False)
    _buf(X, X.shape[0] * PG_MLP_IN, "X", _f32_types(), np.float32, dev, cuda_only=True, writes=False)
    return int(X.shape[0]), dev


def mlp_forward(params, X, stream=None):
    import torch
    B, _ = _mlp_inputs(params, X)
    Y = torch.empty((B, PG_NUM_ACTIONS), dtype=torch.float32, device=X.device)
    _check(load().pg_mlp_forward(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                 B, ctypes.c_void_p(Y.data_ptr()), _stream_ptr(stream)))
    return Y


def mlp_backward(params, X, act, target, stream=None):
    import torch
    B, dev = _mlp_inputs(params, X)
    pa = _buf(act, B, "act", _u32_types(), np.uint32, dev, cuda_only=True, writes=False)
    pt = _buf(target, B, "target", _f32_types(), np.float32, dev, cuda_only=True, writes=False)
    grad = torch.empty(PG_MLP_NPARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(load().pg_mlp_backward(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                  pa, pt, B, ctypes.c_void_p(grad.data_ptr()),
                                  ctypes.c_void_p(loss.data_ptr()), _stream_ptr(stream)))
    return loss, grad


def mlp_adam(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step in place on params, m and v (fp32 CUDA tensors of the
    same size as grad)."""
    if not hasattr(params, "numel"):
        raise ValueError("params must be a CUDA fp32 tensor")
    count, dev = params.numel(), params.device.index
    ptrs = [_buf(x, count, name, _f32_types(), np.float32, dev, cuda_only=True)
            for x, name in ((params, "params"), (grad, "grad"), (m, "m"), (v, "v"))]
    _check(load().pg_mlp_adam(*ptrs, count, t, lr, beta1, beta2, eps, _stream_ptr(stream)))


def bfs_noalloc(offsets, indices, src: int, out, cfg: Config | None = None, stream=None):
    """pg_bfs_noalloc on caller-owned CUDA tensors (int32 views of uint32).

    For callers that cannot allocate device memory at call time: the library
    uses a fixed scratch array instead of allocating.  offsets/indices/out
    must be contiguous int32 or uint32 tensors on one CUDA device, with
    out.numel() >= n = offsets.numel() - 1 and n <= NOALLOC_MAX_N.  The C ABI
    cannot see buffer sizes, so they are checked here (ValueError) before
    anything is launched; the call runs on the tensors' device."""
    import torch
    for name, t in (("offsets", offsets), ("indices", indices), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"bfs_noalloc: {name} must be a torch tensor")
        if t.dtype not in (torch.int32, torch.uint32):
            raise ValueError(f"bfs_noalloc: {name} must be int32 or uint32, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"bfs_noalloc: {name} must be contiguous")
    n = offsets.numel() - 1
    if n < 1:
        raise ValueError("bfs_noalloc: offsets must hold n + 1 >= 2 entries")
    if out.numel() < n:
        raise ValueError(f"bfs_noalloc: out holds {out.numel()} entries, fewer than n = {n}")
    devs = {t.device for t in (offsets, indices, out)}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError(f"bfs_noalloc: offsets, indices and out must be on one CUDA device, got {devs}")
    with torch.cuda.device(out.device):
        _check(load().pg_bfs_noalloc(ctypes.c_void_p(offsets.data_ptr()),
                                     ctypes.c_void_p(indices.data_ptr()), n, indices.numel(),
                                     int(src), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.byref(cfg) if cfg else None, _stream_ptr(stream)))
    return out


def probe_barrier(rounds: int = 20000, threads_per_block: int = 0, blocks_per_sm: int = 0,
                  stream=None) -> float:
    """Microseconds per grid barrier of an empty persistent loop on the
    current device (the per-round floor of any traversal)."""
    us = ctypes.c_float()
    _check(load().pg_probe_barrier(int(rounds), int(threads_per_block), int(blocks_per_sm),
                                   ctypes.byref(us), _stream_ptr(stream)))
    return float(us.value)


def version() -> str:
    return load().pg_version().decode()


def weights_path() -> str:
    return os.path.join(_HERE, "schedule_mlp.f32")


def trained_weights():
    """The committed schedule-MLP weights (float32[1512]) or None."""
    p = weights_path()
    if not os.path.exists(p):
        return None
    w = np.fromfile(p, dtype=np.float32)
    return w if w.size == PG_MLP_NPARAMS else None
