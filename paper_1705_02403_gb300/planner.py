"""Thin Python layer over the C ABI: builds the ABI structs from a Problem,
keeps device buffers in torch tensors, and wraps the library's device arrays
as torch tensors without copying.  Every computation runs in libgmt.so."""
from __future__ import annotations

import numpy as np
import torch

from . import _native as N
from .envgen import Problem


class _CudaArray:
    """__cuda_array_interface__ exporter for a device pointer owned elsewhere."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}
        self._owner = owner


def wrap_device(ptr: int, shape, dtype: str, owner, device=None) -> torch.Tensor:
    """Zero-copy torch view of device memory owned by `owner` (kept alive)."""
    typestr = {"f4": "<f4", "i4": "<i4", "i2": "<i2", "u1": "|u1"}[dtype]
    if int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype={"f4": torch.float32, "i4": torch.int32, "i2": torch.int16,
                                         "u1": torch.uint8}[dtype], device=device or "cuda")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr, owner), device=device or "cuda")


def space_struct(pb: Problem) -> N.gmt_space:
    s = N.gmt_space()
    s.kind, s.dim, s.pos_dim = pb.kind, pb.d, pb.dp
    for a in range(pb.d):
        s.lo[a], s.hi[a] = float(pb.lo[a]), float(pb.hi[a])
    return s


def goal_struct(pb: Problem) -> N.gmt_goal:
    g = N.gmt_goal()
    for a in range(pb.d):
        g.center[a] = float(pb.goal_center[a])
    g.radius = float(pb.goal_radius)
    g.pos_only = int(pb.goal_pos_only)
    return g


def params_struct(pb: Problem, **over) -> N.gmt_params:
    p = N.gmt_params()
    p.n, p.r, p.lambda_, p.seed = pb.n, float(pb.r), float(pb.lam), int(pb.seed)
    p.seg_spacing, p.traj_points = float(pb.seg_spacing), int(pb.traj_points)
    p.max_iters, p.max_attempts = 0, 0
    p.eta, p.mu_free = float(pb.eta), float(pb.mu_free)
    p.spin_limit, p.debug_flags = 0, 0
    p.sampler = int(pb.sampler)
    p.turn_radius = float(getattr(pb, "rho", 0.0))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def boxes_on_device(pb: Problem, device="cuda"):
    lo = torch.as_tensor(np.ascontiguousarray(pb.box_lo, np.float32).reshape(-1, pb.dp), device=device)
    hi = torch.as_tensor(np.ascontiguousarray(pb.box_hi, np.float32).reshape(-1, pb.dp), device=device)
    b = N.gmt_boxes()
    b.count = int(lo.shape[0])
    b.lo = lo.data_ptr() if b.count else None
    b.hi = hi.data_ptr() if b.count else None
    return b, (lo, hi)


class GraphView:
    """torch views (no copies) of a built graph's device arrays."""

    def __init__(self, graph: N.Graph):
        v = N.gmt_graph_get_view(graph)
        self.raw = v
        self.N, self.E, self.dim, self.pitch, self.r = v.N, v.E, v.dim, v.x_pitch, v.r
        self.X = wrap_device(v.X, (v.dim, v.x_pitch), "f4", graph)[:, :v.N]
        self.is_goal = wrap_device(v.is_goal, (v.N,), "u1", graph)
        self.out_row = wrap_device(v.out_row, (v.N + 1,), "i4", graph)
        self.out_col = wrap_device(v.out_col, (v.E,), "i4", graph)
        self.out_cost = wrap_device(v.out_cost, (v.E,), "f4", graph)
        self.in_row = wrap_device(v.in_row, (v.N + 1,), "i4", graph)
        self.in_col = wrap_device(v.in_col, (v.E,), "i4", graph)
        self.in_cost = wrap_device(v.in_cost, (v.E,), "f4", graph)


class Planner:
    """One planning problem: gmt_build_graph then gmt_plan on the same stream."""

    def __init__(self, pb: Problem, device="cuda"):
        self.pb = pb
        self.device = device
        self.space, self.goal = space_struct(pb), goal_struct(pb)
        self.params = params_struct(pb)
        self.boxes, self._box_tensors = boxes_on_device(pb, device)
        self.graph = N.Graph()
        self.parent = torch.empty(pb.N, dtype=torch.int32, device=device)
        self.cost = torch.empty(pb.N, dtype=torch.float32, device=device)
        self.path = torch.empty(pb.N, dtype=torch.int32, device=device)

    def build(self, stream=None, debug_flags=0, asynchronous=False):
        """gmt_build_graph; asynchronous=True queues the build without a host
        wait (gmt_build_graph_async; confirmed by the next plan or view)."""
        params = params_struct(self.pb, debug_flags=debug_flags) if debug_flags else self.params
        fn = N.gmt_build_graph_async if asynchronous else N.gmt_build_graph
        fn(self.space, self.boxes, [float(v) for v in self.pb.x_init], self.goal, params, self.graph, stream)
        return self

    def view(self) -> GraphView:
        return GraphView(self.graph)

    def set_launch(self, blocks: int, threads: int, cluster: int = 0):
        N.gmt_graph_set_launch(self.graph, blocks, threads, cluster)

    def plan(self, stream=None, allow_errors=False, **param_over) -> dict:
        params = params_struct(self.pb, **param_over) if param_over else self.params
        info = N.gmt_plan(self.graph, self.boxes, params, self.parent.data_ptr(), self.cost.data_ptr(),
                          self.path.data_ptr(), stream, allow_errors=allow_errors)
        return info.as_dict()


class BatchPlanner:
    """A batch of problems planned with gmt_plan_batch (one handle, reusable).
    extra: optional DEVICE tensor [q, d, pitch] of samples appended to every
    query (its first extra_count columns; e.g. gmt_propose_batch's output)."""

    def __init__(self, problems, device="cuda", extra=None, extra_count=0):
        self.problems = list(problems)
        self.extra = extra
        self.device = device
        self._keep = []
        self.queries = (N.gmt_query * len(self.problems))()
        for k, pb in enumerate(self.problems):
            qd = self.queries[k]
            qd.space = space_struct(pb)
            b, tens = boxes_on_device(pb, device)
            self._keep.append(tens)
            qd.boxes = b
            for a in range(pb.d):
                qd.x_init[a] = float(pb.x_init[a])
            qd.goal = goal_struct(pb)
            qd.params = params_struct(pb)
            if extra is not None and extra_count > 0:
                assert extra.is_contiguous() and extra.dtype == torch.float32 and extra.shape[0] == len(self.problems)
                qd.extra = extra[k].data_ptr()
                qd.extra_count = extra_count
                qd.extra_pitch = extra.shape[2]
        self.extra_count = extra_count if extra is not None else 0
        self.offsets = np.concatenate(
            [[0], np.cumsum([pb.N + self.extra_count for pb in self.problems])]).astype(np.int64)
        total = int(self.offsets[-1])
        self.parent = torch.empty(total, dtype=torch.int32, device=device)
        self.cost = torch.empty(total, dtype=torch.float32, device=device)
        self.batch = N.Batch()

    def plan(self, stream=None, allow_errors=False, raw=False):
        """Info dicts, or (raw=True) the ctypes info array (N.infos_as_dicts)."""
        return N.gmt_plan_batch(self.queries, self.batch, self.parent.data_ptr(), self.cost.data_ptr(), stream,
                                allow_errors, raw)

    def result(self, k):
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        return self.parent[a:b], self.cost[a:b]

    def view(self, k):
        v, path_ptr = N.gmt_batch_get_view(self.batch, k)
        out = {"N": v.N, "E": v.E, "r": v.r,
               "X": wrap_device(v.X, (v.dim, v.x_pitch), "f4", self.batch)[:, :v.N],
               "is_goal": wrap_device(v.is_goal, (v.N,), "u1", self.batch),
               "out_row": wrap_device(v.out_row, (v.N + 1,), "i4", self.batch),
               "out_col": wrap_device(v.out_col, (v.E,), "i4", self.batch),
               "out_cost": wrap_device(v.out_cost, (v.E,), "f4", self.batch),
               "in_row": wrap_device(v.in_row, (v.N + 1,), "i4", self.batch),
               "in_col": wrap_device(v.in_col, (v.E,), "i4", self.batch),
               "in_cost": wrap_device(v.in_cost, (v.E,), "f4", self.batch),
               "path": wrap_device(path_ptr, (v.N,), "i4", self.batch)}
        return out
