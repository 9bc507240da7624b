"""ctypes binding of libgmt.so: the C ABI of include/gmt.h under the same names.

Argument marshalling only: every step of the planner runs in the library's CUDA
kernels.  Device arrays are passed as raw pointers (torch tensors' data_ptr());
the stream is torch's current CUDA stream unless one is given.  There is no CPU
fallback: if libgmt.so is missing or cannot be loaded, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgmt.so")

GMT_OK, GMT_NO_PATH = 0, 1
GMT_ERR_INVALID, GMT_ERR_OOM, GMT_ERR_CUDA, GMT_ERR_TIMEOUT, GMT_ERR_ITER_LIMIT, GMT_ERR_ADMISSION = -1, -2, -3, -4, -5, -6
GMT_COST_EUCLID, GMT_COST_DI, GMT_COST_DUBINS = 0, 1, 2
GMT_MAX_DIM = 10
GMT_DEBUG_UNREACHABLE_BARRIER = 0x1
GMT_DEBUG_PAIRS_ALL, GMT_DEBUG_PAIRS_CELLS, GMT_DEBUG_CELLS_LIST = 0x2, 0x4, 0x8
GMT_SAMPLER_PHILOX, GMT_SAMPLER_HALTON = 0, 1

STATUS_NAMES = {0: "GMT_OK", 1: "GMT_NO_PATH", -1: "GMT_ERR_INVALID", -2: "GMT_ERR_OOM", -3: "GMT_ERR_CUDA",
                -4: "GMT_ERR_TIMEOUT", -5: "GMT_ERR_ITER_LIMIT", -6: "GMT_ERR_ADMISSION"}


class GmtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gmt_space(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("pos_dim", C.c_int32),
                ("lo", C.c_float * GMT_MAX_DIM), ("hi", C.c_float * GMT_MAX_DIM)]


class gmt_boxes(C.Structure):
    _fields_ = [("count", C.c_int32), ("lo", C.c_void_p), ("hi", C.c_void_p)]


class gmt_goal(C.Structure):
    _fields_ = [("center", C.c_float * GMT_MAX_DIM), ("radius", C.c_float), ("pos_only", C.c_int32)]


class gmt_params(C.Structure):
    _fields_ = [("n", C.c_int32), ("r", C.c_float), ("lambda_", C.c_float), ("seed", C.c_uint64),
                ("seg_spacing", C.c_float), ("traj_points", C.c_int32), ("max_iters", C.c_int32),
                ("max_attempts", C.c_int32), ("eta", C.c_float), ("mu_free", C.c_float),
                ("spin_limit", C.c_int32), ("debug_flags", C.c_uint32), ("sampler", C.c_int32),
                ("turn_radius", C.c_float)]


class gmt_graph_view(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("pos_dim", C.c_int32), ("N", C.c_int32),
                ("x_pitch", C.c_int32), ("E", C.c_int64), ("r", C.c_float),
                ("X", C.c_void_p), ("is_goal", C.c_void_p),
                ("out_row", C.c_void_p), ("out_col", C.c_void_p), ("out_cost", C.c_void_p),
                ("in_row", C.c_void_p), ("in_col", C.c_void_p), ("in_cost", C.c_void_p),
                ("out_tau", C.c_void_p), ("in_tau", C.c_void_p), ("turn_radius", C.c_float),
                ("in_path", C.c_void_p)]


class gmt_plan_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("goal_node", C.c_int32), ("path_cost", C.c_float), ("path_len", C.c_int32),
                ("iters", C.c_int64), ("final_i", C.c_int64), ("push_edges", C.c_int64),
                ("pull_edges", C.c_int64), ("checks", C.c_int64), ("failed", C.c_int64),
                ("tree_size", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gmt_profile(C.Structure):
    _fields_ = [("sample_ms", C.c_float), ("pair_ms", C.c_float), ("transpose_ms", C.c_float),
                ("scan_ms", C.c_float), ("fill_ms", C.c_float), ("plan_ms", C.c_float),
                ("plan_blocks", C.c_int32), ("plan_threads", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gmt_query(C.Structure):
    _fields_ = [("space", gmt_space), ("boxes", gmt_boxes), ("x_init", C.c_float * GMT_MAX_DIM),
                ("goal", gmt_goal), ("params", gmt_params), ("extra", C.c_void_p), ("extra_count", C.c_int32),
                ("extra_pitch", C.c_int32)]


class gmt_model_config(C.Structure):
    _fields_ = [("grid", C.c_int32), ("hidden", C.c_int32), ("cells", C.c_int32), ("max_batch", C.c_int32),
                ("seed", C.c_uint64)]


class gmt_model_view(C.Structure):
    _fields_ = [("grid", C.c_int32), ("hidden", C.c_int32), ("cells", C.c_int32), ("in_features", C.c_int32),
                ("z_features", C.c_int32), ("n_cells", C.c_int32), ("max_batch", C.c_int32), ("step", C.c_int64),
                ("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
                ("W3", C.c_void_p), ("b3", C.c_void_p),
                ("gW1", C.c_void_p), ("gb1", C.c_void_p), ("gW2", C.c_void_p), ("gb2", C.c_void_p),
                ("gW3", C.c_void_p), ("gb3", C.c_void_p),
                ("W1_bf16", C.c_void_p), ("W2_bf16", C.c_void_p), ("W3_bf16", C.c_void_p),
                ("logits", C.c_void_p), ("loss", C.c_void_p),
                ("H1", C.c_void_p), ("H2", C.c_void_p), ("Z", C.c_void_p), ("dlog", C.c_void_p),
                ("dH2", C.c_void_p), ("dH1", C.c_void_p)]


class gmt_server_config(C.Structure):
    _fields_ = [("slots", C.c_int32), ("cluster", C.c_int32), ("threads", C.c_int32), ("max_nodes", C.c_int32),
                ("max_boxes", C.c_int32), ("memory_budget", C.c_uint64)]


class gmt_server_result(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("session", C.c_int32), ("status", C.c_int32), ("goal_node", C.c_int32),
                ("path_cost", C.c_float), ("iters", C.c_int64), ("checks", C.c_int64),
                ("checks_computed", C.c_int64), ("edges_checked", C.c_int64), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every symbol include/gmt.h declares, with its ctypes signature.
_P, _I32, _I64, _F32, _F64, _U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_uint64
SIGNATURES = {
    "gmt_build_graph": (_I32, [C.POINTER(gmt_space), C.POINTER(gmt_boxes), _P, C.POINTER(gmt_goal),
                               C.POINTER(gmt_params), C.POINTER(C.c_void_p), _P]),
    "gmt_graph_get_view": (_I32, [_P, C.POINTER(gmt_graph_view)]),
    "gmt_graph_free": (None, [_P]),
    "gmt_graph_set_launch": (_I32, [_P, _I32, _I32, _I32]),
    "gmt_plan": (_I32, [_P, C.POINTER(gmt_boxes), C.POINTER(gmt_params), _P, _P, _P, C.POINTER(gmt_plan_info), _P]),
    "gmt_plan_static": (_I32, [C.POINTER(gmt_space), C.POINTER(gmt_graph_view), C.POINTER(gmt_boxes),
                               C.POINTER(gmt_params), _P, _P, _P, C.POINTER(gmt_plan_info), _P]),
    "gmt_graph_set_profiling": (_I32, [_P, _I32]),
    "gmt_graph_get_profile": (_I32, [_P, C.POINTER(gmt_profile)]),
    "gmt_plan_batch": (_I32, [_I32, C.POINTER(gmt_query), C.POINTER(C.c_void_p), _P, _P, C.POINTER(gmt_plan_info),
                              _P]),
    "gmt_batch_get_view": (_I32, [_P, _I32, C.POINTER(gmt_graph_view), C.POINTER(C.c_void_p)]),
    "gmt_batch_set_mode": (_I32, [_P, _I32]),
    "gmt_batch_set_launch": (_I32, [_P, _I32, _I32]),
    "gmt_batch_get_launch": (_I32, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
    "gmt_batch_last_plan_ms": (_I32, [_P, C.POINTER(_F32)]),
    "gmt_batch_autotune": (_I32, [_P, _P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_F32)]),
    "gmt_batch_free": (None, [_P]),
    "gmt_gemm_bf16": (_I32, [_I32, _I32, _I32, _P, _P, _I32, _P, _P, _P, _I32, _P, _P, _P]),
    "gmt_build_graph_ex": (_I32, [C.POINTER(gmt_space), C.POINTER(gmt_boxes), _P, C.POINTER(gmt_goal),
                                  C.POINTER(gmt_params), _P, _I32, _I32, C.POINTER(C.c_void_p), _P]),
    "gmt_build_graph_async": (_I32, [C.POINTER(gmt_space), C.POINTER(gmt_boxes), _P, C.POINTER(gmt_goal),
                                     C.POINTER(gmt_params), C.POINTER(C.c_void_p), _P]),
    "gmt_model_create": (_I32, [C.POINTER(gmt_model_config), C.POINTER(C.c_void_p)]),
    "gmt_model_free": (None, [_P]),
    "gmt_model_get_view": (_I32, [_P, C.POINTER(gmt_model_view)]),
    "gmt_voxelize": (_I32, [_I32, C.POINTER(gmt_boxes), _I32, _P, _P]),
    "gmt_model_forward": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "gmt_model_backward": (_I32, [_P, _I32, _P, _P, _P, C.POINTER(_F32), _P]),
    "gmt_model_train_step": (_I32, [_P, _I32, _P, _P, _P, _F32, _F32, C.POINTER(_F32), _P]),
    "gmt_model_save": (_I32, [_P, C.c_char_p]),
    "gmt_model_load": (_I32, [_P, C.c_char_p]),
    "gmt_path_histogram": (_I32, [_P, _I32, _P, _I32, _I32, _F32, _F32, _P, _P]),
    "gmt_propose": (_I32, [_P, C.POINTER(gmt_space), C.POINTER(gmt_boxes), _P, _P, _I32, _U64, _P, _I32, _P]),
    "gmt_propose_batch": (_I32, [_P, _I32, C.POINTER(gmt_space), C.POINTER(gmt_boxes), _P, _I32, _P, _P, _I32,
                                 _P]),
    "gmt_server_create": (_I32, [C.POINTER(gmt_server_config), C.POINTER(C.c_void_p)]),
    "gmt_server_free": (None, [_P]),
    "gmt_server_open_session": (_I32, [_P, C.POINTER(gmt_space), _P, C.POINTER(gmt_goal), C.POINTER(gmt_params), _I32,
                                       _P, _P, C.POINTER(_I32)]),
    "gmt_server_submit": (_I32, [_P, _I32, _U64, _P, _P, _P, _P]),
    "gmt_server_poll": (_I32, [_P, C.POINTER(gmt_server_result), _I32, C.POINTER(_I32), _I32]),
    "gmt_server_close_session": (_I32, [_P, _I32]),
    "gmt_server_move_start": (_I32, [_P, _I32, _P]),
    "gmt_server_session_view": (_I32, [_P, _I32, C.POINTER(gmt_graph_view)]),
    "gmt_connection_radius": (_F64, [_I32, _I32, _F64, _F64]),
    "gmt_connection_radius_halton": (_F64, [_I32, _I32, _F64, _F64]),
    "gmt_last_error": (C.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1705_02403_gb300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int, allow=(GMT_OK,)):
    if status not in allow:
        raise GmtError(status, lib.gmt_last_error().decode())
    return status


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------- C ABI names
def gmt_last_error() -> str:
    return lib.gmt_last_error().decode()


def gmt_connection_radius(n: int, d: int, eta: float = 0.0, mu_free: float = 1.0) -> float:
    return lib.gmt_connection_radius(n, d, eta, mu_free)


def gmt_connection_radius_halton(n: int, d: int, eta: float = 0.0, mu_free: float = 1.0) -> float:
    return lib.gmt_connection_radius_halton(n, d, eta, mu_free)


class Graph:
    """Owner of a gmt_graph handle (freed with gmt_graph_free)."""

    def __init__(self):
        self.handle = C.c_void_p(None)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib.gmt_graph_free(self.handle)
            self.handle = C.c_void_p(None)


def gmt_build_graph(space: gmt_space, boxes: gmt_boxes, x_init, goal: gmt_goal, params: gmt_params,
                    graph: Graph | None = None, stream=None) -> Graph:
    """x_init: host sequence of floats (state dimension)."""
    g = graph if graph is not None else Graph()
    xi = (C.c_float * GMT_MAX_DIM)(*[float(v) for v in x_init])
    _check(lib.gmt_build_graph(C.byref(space), C.byref(boxes), C.cast(xi, C.c_void_p), C.byref(goal),
                               C.byref(params), C.byref(g.handle), _stream(stream)))
    return g


def gmt_build_graph_async(space: gmt_space, boxes: gmt_boxes, x_init, goal: gmt_goal, params: gmt_params,
                          graph: Graph | None = None, stream=None) -> Graph:
    """gmt_build_graph without the host synchronisation (confirmed by the next
    gmt_plan or view on the handle); `boxes`' arrays must stay valid until then."""
    g = graph if graph is not None else Graph()
    xi = (C.c_float * GMT_MAX_DIM)(*[float(v) for v in x_init])
    _check(lib.gmt_build_graph_async(C.byref(space), C.byref(boxes), C.cast(xi, C.c_void_p), C.byref(goal),
                                     C.byref(params), C.byref(g.handle), _stream(stream)))
    return g


def gmt_graph_get_view(graph: Graph) -> gmt_graph_view:
    v = gmt_graph_view()
    _check(lib.gmt_graph_get_view(graph.handle, C.byref(v)))
    return v


def gmt_graph_set_launch(graph: Graph, blocks: int, threads: int, cluster: int = 0) -> None:
    _check(lib.gmt_graph_set_launch(graph.handle, blocks, threads, cluster))


def gmt_plan_static(space: gmt_space, view: gmt_graph_view, boxes: gmt_boxes, params: gmt_params,
                    parent_ptr: int, cost_ptr: int, path_ptr: int | None = None, stream=None,
                    allow_errors=False) -> gmt_plan_info:
    """Allocation-free plan on caller-described device arrays (see gmt.h)."""
    info = gmt_plan_info()
    st = lib.gmt_plan_static(C.byref(space), C.byref(view), C.byref(boxes), C.byref(params), C.c_void_p(parent_ptr),
                             C.c_void_p(cost_ptr), C.c_void_p(path_ptr or 0), C.byref(info), _stream(stream))
    if not allow_errors:
        _check(st, allow=(GMT_OK, GMT_NO_PATH))
    info.rc = st
    return info


def gmt_graph_set_profiling(graph: Graph, enable: bool) -> None:
    _check(lib.gmt_graph_set_profiling(graph.handle, int(enable)))


def gmt_graph_get_profile(graph: Graph) -> dict:
    p = gmt_profile()
    _check(lib.gmt_graph_get_profile(graph.handle, C.byref(p)))
    return p.as_dict()


def gmt_graph_free(graph: Graph) -> None:
    if graph.handle.value:
        lib.gmt_graph_free(graph.handle)
        graph.handle = C.c_void_p(None)


def gmt_plan(graph: Graph, boxes: gmt_boxes, params: gmt_params, parent_ptr: int, cost_ptr: int,
             path_ptr: int | None = None, stream=None, allow_errors=False) -> gmt_plan_info:
    info = gmt_plan_info()
    st = lib.gmt_plan(graph.handle, C.byref(boxes), C.byref(params), C.c_void_p(parent_ptr), C.c_void_p(cost_ptr),
                      C.c_void_p(path_ptr or 0), C.byref(info), _stream(stream))
    if not allow_errors:
        _check(st, allow=(GMT_OK, GMT_NO_PATH))
    return info


class Batch:
    """Owner of a gmt_batch handle (freed with gmt_batch_free)."""

    def __init__(self):
        self.handle = C.c_void_p(None)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib.gmt_batch_free(self.handle)
            self.handle = C.c_void_p(None)


def gmt_plan_batch(queries, batch: Batch, parent_ptr: int, cost_ptr: int, stream=None, allow_errors=False,
                   raw=False):
    """queries: a ctypes array of gmt_query.  Returns the list of info dicts
    (raw=True: the ctypes gmt_plan_info array, for infos_as_dicts later)."""
    q = len(queries)
    infos = (gmt_plan_info * q)()
    st = lib.gmt_plan_batch(q, queries, C.byref(batch.handle), C.c_void_p(parent_ptr), C.c_void_p(cost_ptr), infos,
                            _stream(stream))
    if not allow_errors:
        _check(st)
    return infos if raw else infos_as_dicts(infos)


def infos_as_dicts(infos):
    return [i.as_dict() for i in infos]


def gmt_batch_get_view(batch: Batch, k: int):
    v = gmt_graph_view()
    path = C.c_void_p()
    _check(lib.gmt_batch_get_view(batch.handle, k, C.byref(v), C.byref(path)))
    return v, path.value


BATCH_AUTO, BATCH_TEAMS, BATCH_LOCKSTEP, BATCH_POOL = 0, 1, 2, 3


def gmt_batch_set_mode(batch: Batch, mode: int) -> None:
    _check(lib.gmt_batch_set_mode(batch.handle, mode))


def gmt_batch_set_launch(batch: Batch, cluster: int, threads: int) -> None:
    _check(lib.gmt_batch_set_launch(batch.handle, cluster, threads))


def gmt_batch_get_launch(batch: Batch):
    """(mode, cluster, threads) of the next plan stage."""
    m, c, t = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.gmt_batch_get_launch(batch.handle, C.byref(m), C.byref(c), C.byref(t)))
    return m.value, c.value, t.value


def gmt_batch_last_plan_ms(batch: Batch) -> float:
    """Device time of the last call's plan stage (ms)."""
    ms = C.c_float()
    _check(lib.gmt_batch_last_plan_ms(batch.handle, C.byref(ms)))
    return ms.value


def gmt_batch_autotune(batch: Batch, stream=None):
    c, t, ms = C.c_int32(), C.c_int32(), C.c_float()
    _check(lib.gmt_batch_autotune(batch.handle, _stream(stream), C.byref(c), C.byref(t), C.byref(ms)))
    return c.value, t.value, ms.value


def gmt_gemm_bf16(A, B, epilogue=0, bias=None, splits=1, stream=None):
    """C = A . B^T on the tensor cores (A [M,K], B [N,K] torch bf16 CUDA tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    dev = A.device
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    C = torch.empty(M, N, dtype=torch.float32, device=dev) if epilogue != 1 else None
    Cb = torch.empty(M, N, dtype=torch.bfloat16, device=dev) if epilogue == 1 else None
    ws = torch.empty(splits * M * N, dtype=torch.float32, device=dev) if splits > 1 else None
    _check(lib.gmt_gemm_bf16(M, N, K, A.data_ptr(), B.data_ptr(), epilogue,
                             bias.data_ptr() if bias is not None else None,
                             C.data_ptr() if C is not None else None, Cb.data_ptr() if Cb is not None else None,
                             splits, ws.data_ptr() if ws is not None else None, err.data_ptr(), _stream(stream)))
    return (C if epilogue != 1 else Cb), err


class Model:
    """Owner of a gmt_model handle."""

    def __init__(self, grid=32, hidden=512, cells=16, max_batch=256, seed=1):
        cfg = gmt_model_config(grid, hidden, cells, max_batch, seed)
        self.handle = C.c_void_p(None)
        _check(lib.gmt_model_create(C.byref(cfg), C.byref(self.handle)))

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib.gmt_model_free(self.handle)
            self.handle = C.c_void_p(None)

    def view(self) -> gmt_model_view:
        v = gmt_model_view()
        _check(lib.gmt_model_get_view(self.handle, C.byref(v)))
        return v

    def forward(self, B, voxels_ptr, sg_ptr, logits_ptr=None, stream=None):
        _check(lib.gmt_model_forward(self.handle, B, C.c_void_p(voxels_ptr), C.c_void_p(sg_ptr),
                                     C.c_void_p(logits_ptr or 0), _stream(stream)))

    def backward(self, B, voxels_ptr, sg_ptr, target_ptr, stream=None):
        loss = C.c_float()
        _check(lib.gmt_model_backward(self.handle, B, C.c_void_p(voxels_ptr), C.c_void_p(sg_ptr),
                                      C.c_void_p(target_ptr), C.byref(loss), _stream(stream)))
        return loss.value

    def train_step(self, B, voxels_ptr, sg_ptr, target_ptr, lr, weight_decay=0.0, stream=None):
        loss = C.c_float()
        _check(lib.gmt_model_train_step(self.handle, B, C.c_void_p(voxels_ptr), C.c_void_p(sg_ptr),
                                        C.c_void_p(target_ptr), lr, weight_decay, C.byref(loss), _stream(stream)))
        return loss.value

    def save(self, path):
        _check(lib.gmt_model_save(self.handle, path.encode()))

    def load(self, path):
        _check(lib.gmt_model_load(self.handle, path.encode()))


def gmt_voxelize(boxes_list, grid, voxels_ptr, stream=None):
    arr = (gmt_boxes * len(boxes_list))(*boxes_list)
    _check(lib.gmt_voxelize(len(boxes_list), arr, grid, C.c_void_p(voxels_ptr), _stream(stream)))


def gmt_path_histogram(X_ptr, pitch, path_ptr, length, cells, spacing, eps, hist_ptr, stream=None):
    _check(lib.gmt_path_histogram(C.c_void_p(X_ptr), pitch, C.c_void_p(path_ptr), length, cells, spacing, eps,
                                  C.c_void_p(hist_ptr), _stream(stream)))


def gmt_propose(model: Model, space: gmt_space, boxes: gmt_boxes, start, goal, count, seed, samples_ptr, pitch,
                stream=None):
    s3 = (C.c_float * 3)(*[float(v) for v in start[:3]])
    g3 = (C.c_float * 3)(*[float(v) for v in goal[:3]])
    _check(lib.gmt_propose(model.handle, C.byref(space), C.byref(boxes), C.cast(s3, C.c_void_p),
                           C.cast(g3, C.c_void_p), count, seed, C.c_void_p(samples_ptr), pitch, _stream(stream)))


class ProposeBatchArgs:
    """The HOST arrays of a gmt_propose_batch call, marshalled once (reusable
    across calls on the same problems)."""

    def __init__(self, spaces, boxes, start_goal, seeds):
        B = len(spaces)
        self.B = B
        self.sp = (gmt_space * B)(*spaces)
        self.bx = (gmt_boxes * B)(*boxes)
        self.sg = (C.c_float * (6 * B))(*[float(v) for row in start_goal for v in row[:6]])
        self.sd = (C.c_uint64 * B)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in seeds])


def gmt_propose_batch(model: Model, spaces, boxes, start_goal, count, seeds, samples_ptr, pitch, stream=None,
                      args: ProposeBatchArgs | None = None):
    """spaces, boxes: sequences of B structs; start_goal: [B][6] floats; seeds:
    B integers; samples: DEVICE [B][3][pitch].  args: the same inputs
    marshalled once (then spaces .. seeds are ignored)."""
    a = args if args is not None else ProposeBatchArgs(spaces, boxes, start_goal, seeds)
    _check(lib.gmt_propose_batch(model.handle, a.B, a.sp, a.bx, C.cast(a.sg, C.c_void_p), count,
                                 C.cast(a.sd, C.c_void_p), C.c_void_p(samples_ptr), pitch, _stream(stream)))


def gmt_build_graph_ex(space, boxes, x_init, goal, params, extra_ptr, extra_count, extra_pitch,
                       graph: Graph | None = None, stream=None) -> Graph:
    g = graph if graph is not None else Graph()
    xi = (C.c_float * GMT_MAX_DIM)(*[float(v) for v in x_init])
    _check(lib.gmt_build_graph_ex(C.byref(space), C.byref(boxes), C.cast(xi, C.c_void_p), C.byref(goal),
                                  C.byref(params), C.c_void_p(extra_ptr or 0), extra_count, extra_pitch,
                                  C.byref(g.handle), _stream(stream)))
    return g


class Server:
    """Owner of a gmt_server handle."""

    def __init__(self, slots=16, cluster=4, threads=0, max_nodes=8193, max_boxes=64, memory_budget=0):
        cfg = gmt_server_config(slots, cluster, threads, max_nodes, max_boxes, memory_budget)
        self.handle = C.c_void_p(None)
        _check(lib.gmt_server_create(C.byref(cfg), C.byref(self.handle)))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib.gmt_server_free(self.handle)
            self.handle = C.c_void_p(None)

    __del__ = close

    def open_session(self, space, x_init, goal, params, box_lo, box_hi, allow_errors=False):
        import numpy as np
        lo = np.ascontiguousarray(box_lo, np.float32)
        hi = np.ascontiguousarray(box_hi, np.float32)
        xi = (C.c_float * GMT_MAX_DIM)(*[float(v) for v in x_init])
        sid = C.c_int32()
        st = lib.gmt_server_open_session(self.handle, C.byref(space), C.cast(xi, C.c_void_p), C.byref(goal),
                                         C.byref(params), lo.shape[0], lo.ctypes.data_as(C.c_void_p),
                                         hi.ctypes.data_as(C.c_void_p), C.byref(sid))
        if allow_errors and st != GMT_OK:
            return None, st
        _check(st)
        return sid.value, st

    def submit(self, session, request_id, box_lo, box_hi, parent_ptr=None, cost_ptr=None):
        import numpy as np
        lo = np.ascontiguousarray(box_lo, np.float32)
        hi = np.ascontiguousarray(box_hi, np.float32)
        _check(lib.gmt_server_submit(self.handle, session, request_id, lo.ctypes.data_as(C.c_void_p),
                                     hi.ctypes.data_as(C.c_void_p), C.c_void_p(parent_ptr or 0),
                                     C.c_void_p(cost_ptr or 0)))

    def poll(self, max_results=1024, wait_ms=0):
        out = (gmt_server_result * max_results)()
        n = C.c_int32()
        _check(lib.gmt_server_poll(self.handle, out, max_results, C.byref(n), wait_ms))
        return [out[k].as_dict() for k in range(n.value)]

    def close_session(self, session):
        _check(lib.gmt_server_close_session(self.handle, session))

    def move_start(self, session, x_init):
        xi = (C.c_float * GMT_MAX_DIM)(*[float(v) for v in x_init])
        _check(lib.gmt_server_move_start(self.handle, session, C.cast(xi, C.c_void_p)))

    def session_view(self, session):
        v = gmt_graph_view()
        _check(lib.gmt_server_session_view(self.handle, session, C.byref(v)))
        return v
