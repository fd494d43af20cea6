"""Thin ctypes binding of libcomo3r.so (the C ABI in include/como3r.h).

Argument marshalling only: every step of the refinement runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the shared library
is missing the import of this module raises, so there is no silent fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcomo3r.so")

OK = 0
WARN_SOLVE_FAILED = 1
WARN_SKIPPED = 2
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_UNSUPPORTED = -4
F16, F32, F64 = 0, 1, 2
PLAIN_FP64, MIXED = 0, 1
VJP_UNROLLED, VJP_ENVELOPE = 0, 1
EDGE_RECORD = 64
STAT_NAMES = ["graphs", "keyframes", "edges", "items", "columns", "blocks", "fill", "updates", "levels",
              "valid", "chunk", "block", "grid", "smem_solve", "nd_graphs", "k1_stalls", "solve_ctas", "solve_flops",
              "solve_groups"]

STAGE_NAMES = ["edge_prep", "residual_reduce", "edge_reduce", "assemble", "factor_solve", "retract", "iteration"]

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


class GraphDesc(ctypes.Structure):
    _fields_ = [
        ("num_graphs", ctypes.c_int32),
        ("kf_offset", _i32p), ("height", _i32p), ("width", _i32p), ("agent_of", _i32p),
        ("points_conf", ctypes.c_void_p), ("dtype", ctypes.c_int32),
        ("edge_offset", _i32p), ("edge_i", _i32p), ("edge_j", _i32p),
        ("match_idx", ctypes.c_void_p), ("anchor", _i32p),
        ("sigma_ray", ctypes.c_double), ("sigma_dist", ctypes.c_double), ("huber_k", ctypes.c_double),
        ("lam", ctypes.c_double), ("eps0", ctypes.c_double),
        ("max_attempts", ctypes.c_int32), ("mode", ctypes.c_int32), ("copy_inputs", ctypes.c_int32),
    ]


class GraphInfo(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_double), ("attempts", ctypes.c_int32), ("solved", ctypes.c_int32),
                ("valid_matches", ctypes.c_int64), ("skipped_matches", ctypes.c_int64)]


class DepthDesc(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_void_p), ("c_min", ctypes.c_double), ("min_pixels", ctypes.c_int32),
                ("sigma_point", ctypes.c_double), ("lambda_smooth", ctypes.c_double),
                ("lambda_prior", ctypes.c_double), ("lambda_lm", ctypes.c_double), ("eta_max", ctypes.c_double)]


DEPTH_DEFAULTS = dict(c_min=1.5, min_pixels=16, sigma_point=0.05, lambda_smooth=1.0, lambda_prior=1.0,
                      lambda_lm=0.05, eta_max=0.5)


class MatchDesc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("frame_points", ctypes.c_void_p),
                ("query_points", ctypes.c_void_p), ("num_queries", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("init", ctypes.c_void_p), ("max_steps", ctypes.c_int32), ("max_angle", ctypes.c_double)]


class GaugeDesc(ctypes.Structure):
    _fields_ = [
        ("num_candidates", ctypes.c_int32), ("num_kf", ctypes.c_int32), ("pix_off", ctypes.POINTER(ctypes.c_int64)),
        ("points_conf", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("kf_i", ctypes.POINTER(ctypes.c_int32)),
        ("kf_j", ctypes.POINTER(ctypes.c_int32)), ("match_ij", ctypes.c_void_p), ("match_ji", ctypes.c_void_p),
        ("poses", ctypes.c_void_p), ("q_min", ctypes.c_double), ("nu_min", ctypes.c_double),
        ("nc_min", ctypes.c_int32), ("mode", ctypes.c_int32),
    ]


class GaugeResult(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double * 8), ("nu_i", ctypes.c_double), ("nu_j", ctypes.c_double),
                ("n_i", ctypes.c_int64), ("n_j", ctypes.c_int64), ("valid_i", ctypes.c_int64),
                ("valid_j", ctypes.c_int64), ("admitted", ctypes.c_int32), ("fallback", ctypes.c_int32)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libcomo3r.so not built ({path}); run `python -m paper_2605_30488_b300.build`")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.como3r_graph_create.argtypes = [ctypes.POINTER(GraphDesc), vp, ctypes.POINTER(vp)]
    lib.como3r_graph_destroy.argtypes = [vp]
    lib.como3r_graph_destroy.restype = None
    lib.como3r_gn_step.argtypes = [vp, vp, vp, vp, ctypes.POINTER(GraphInfo)]
    lib.como3r_solve.argtypes = [vp, vp, ctypes.c_int32, _f64p, ctypes.POINTER(GraphInfo)]
    lib.como3r_linearize.argtypes = [vp, vp, vp, _f64p]
    lib.como3r_solve_timestamps.argtypes = [vp, _i64p, _i64p]
    lib.como3r_last_step.argtypes = [vp, vp]
    lib.como3r_sim3_retract.argtypes = [vp, vp, ctypes.c_int32, vp]
    lib.como3r_update_inputs.argtypes = [vp, vp, vp]
    lib.como3r_time_stages.argtypes = [vp, vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    lib.como3r_last_launch_count.argtypes = [vp]
    lib.como3r_last_launch_count.restype = ctypes.c_int64
    lib.como3r_graph_stats.argtypes = [vp, _i64p]
    lib.como3r_plan_stats.argtypes = [ctypes.POINTER(GraphDesc), _i64p]
    lib.como3r_linearize_noalloc.argtypes = [ctypes.POINTER(GraphDesc), vp, vp, vp]
    lib.como3r_vjp.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp, vp, vp, _f64p]
    lib.como3r_time_vjp.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    lib.como3r_points_from_logdepth.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    lib.como3r_rays_from_points.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp, vp, vp]
    lib.como3r_gauge_sync.argtypes = [ctypes.POINTER(GaugeDesc), vp, ctypes.POINTER(GaugeResult),
                                      ctypes.POINTER(ctypes.c_float)]
    lib.como3r_gauge_transport.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_int32, vp]
    lib.como3r_depth_setup.argtypes = [vp, ctypes.POINTER(DepthDesc), _i64p]
    lib.como3r_depth_refine.argtypes = [vp, vp, vp, ctypes.c_int32, _f64p, vp, ctypes.POINTER(ctypes.c_float)]
    lib.como3r_project_match.argtypes = [ctypes.POINTER(MatchDesc), vp, vp, vp]
    lib.como3r_fuse.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, _f64p, vp]
    lib.como3r_fuse_packed.argtypes = [vp, vp, _i64p, _f64p, ctypes.c_int32, ctypes.c_int32, vp]
    lib.como3r_status_str.argtypes = [ctypes.c_int]
    lib.como3r_status_str.restype = ctypes.c_char_p
    lib.como3r_last_error.argtypes = []
    lib.como3r_last_error.restype = ctypes.c_char_p
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class Como3rError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().como3r_last_error().decode() or lib().como3r_status_str(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def _check(code: int, where: str) -> int:
    if code < 0:
        raise Como3rError(code, where)
    return code


def _ptr(a):
    """Raw address of a torch tensor or a numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _dtype_code(np_dtype) -> int:
    return {np.dtype(np.float16): F16, np.dtype(np.float32): F32, np.dtype(np.float64): F64}[np.dtype(np_dtype)]


def _torch_stream(stream):
    if stream is not None:  # a raw cudaStream_t handle or a torch.cuda.Stream
        return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _build_desc(prob, points_ptr, midx_ptr, mode: int, copy_inputs: bool, keep: list) -> GraphDesc:
    arrs = dict(kf_offset=_i32(prob.kf_offset), height=_i32(prob.height), width=_i32(prob.width),
                agent_of=_i32(prob.agent_of), edge_offset=_i32(prob.edge_offset), edge_i=_i32(prob.edge_i),
                edge_j=_i32(prob.edge_j), anchor=_i32(prob.anchor))
    keep.append(arrs)
    d = GraphDesc()
    d.num_graphs = len(arrs["kf_offset"]) - 1
    for k in ("kf_offset", "height", "width", "agent_of", "edge_offset", "edge_i", "edge_j", "anchor"):
        setattr(d, k, arrs[k].ctypes.data_as(_i32p))
    d.points_conf = points_ptr
    d.dtype = _dtype_code(prob.points.dtype)
    d.match_idx = midx_ptr
    d.sigma_ray, d.sigma_dist, d.huber_k = prob.sigma_ray, prob.sigma_dist, prob.huber_k
    d.lam, d.eps0, d.max_attempts = prob.lam, prob.eps0, prob.max_attempts
    d.mode = mode
    d.copy_inputs = 1 if copy_inputs else 0
    return d


def plan_stats(prob) -> dict:
    """Host-only plan of a problem (ordering, factor pattern); no GPU needed."""
    keep = []
    pts = np.zeros(4, dtype=prob.points.dtype)  # non-NULL placeholder; never dereferenced
    d = _build_desc(prob, _ptr(pts), _ptr(np.zeros(1, np.int32)), MIXED, False, keep)
    out = (ctypes.c_int64 * len(STAT_NAMES))()
    _check(lib().como3r_plan_stats(ctypes.byref(d), out), "plan_stats")
    return dict(zip(STAT_NAMES, list(out)))


class Graph:
    """One handle of como3r_graph_create over a problem's arrays (synth.Problem-like).

    `points` / `match_idx` default to device copies of the problem's arrays held by this
    object (borrowed by the library); with copy_inputs=True the library copies them (host
    or device sources) into its own buffers.
    """

    def __init__(self, prob, mode: int = MIXED, points=None, match_idx=None, copy_inputs: bool = False,
                 stream=None, device: str = "cuda"):
        import torch
        self.prob = prob
        self.N = prob.num_kf
        self.G = prob.num_graphs
        self.E = prob.num_edges
        self._keep = []
        if points is None:
            points = torch.from_numpy(np.ascontiguousarray(prob.points))
            points = points.pin_memory() if copy_inputs else points.to(device)
        if match_idx is None:
            match_idx = torch.from_numpy(np.ascontiguousarray(prob.match_idx.astype(np.int32)))
            match_idx = match_idx.pin_memory() if copy_inputs else match_idx.to(device)
        self.points, self.match_idx = points, match_idx
        self.copy_inputs = bool(copy_inputs)
        self._stream = _torch_stream(stream)
        d = _build_desc(prob, _ptr(points), _ptr(match_idx), mode, copy_inputs, self._keep)
        h = ctypes.c_void_p()
        _check(lib().como3r_graph_create(ctypes.byref(d), self._stream, ctypes.byref(h)), "graph_create")
        self.handle = h

    # -- lifetime
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().como3r_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def gn_step(self, poses, H_out=None, g_out=None):
        info = (GraphInfo * self.G)()
        st = _check(lib().como3r_gn_step(self.handle, _ptr(poses), _ptr(H_out), _ptr(g_out), info), "gn_step")
        return st, [_info_dict(x) for x in info]

    def solve(self, poses, iters: int, trace: bool = True):
        info = (GraphInfo * self.G)()
        tr = np.zeros((iters + 1) * self.G) if trace else None
        st = _check(lib().como3r_solve(self.handle, _ptr(poses), int(iters),
                                       tr.ctypes.data_as(_f64p) if trace else None, info), "solve")
        return st, (tr.reshape(iters + 1, self.G) if trace else None), [_info_dict(x) for x in info]

    def depth_setup(self, labels, **params) -> int:
        """como3r_depth_setup: snapshot the current pointmaps, build the segments from the
        per-pixel labels (host or device int32, concatenated like the pixels); returns M."""
        pr = dict(DEPTH_DEFAULTS)
        pr.update(params)
        if not hasattr(labels, "data_ptr"):
            labels = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
        self._depth_labels = labels
        d = DepthDesc(labels=_ptr(labels), c_min=float(pr["c_min"]), min_pixels=int(pr["min_pixels"]),
                      sigma_point=float(pr["sigma_point"]), lambda_smooth=float(pr["lambda_smooth"]),
                      lambda_prior=float(pr["lambda_prior"]), lambda_lm=float(pr["lambda_lm"]),
                      eta_max=float(pr["eta_max"]))
        M = np.zeros(1, dtype=np.int64)
        _check(lib().como3r_depth_setup(self.handle, ctypes.byref(d), M.ctypes.data_as(_i64p)), "depth_setup")
        return int(M[0])

    def depth_refine(self, poses, eta, iters: int, points_out=None, timing: bool = False):
        """como3r_depth_refine: `iters` Jacobi steps from eta (host float64 array or CUDA
        tensor, updated in place); returns (eta, cost trace [iters + 1]) and the mean
        per-match pass time in ms when `timing`."""
        tr = np.zeros(iters + 1)
        ms = ctypes.c_float(0.0)
        _check(lib().como3r_depth_refine(self.handle, _ptr(poses), _ptr(eta), int(iters),
                                         tr.ctypes.data_as(_f64p), _ptr(points_out),
                                         ctypes.byref(ms) if timing else None), "depth_refine")
        return (eta, tr, float(ms.value)) if timing else (eta, tr)

    def timestamps(self):
        """como3r_solve_timestamps: (start_ns, done_ns[G]) of the last gn_step / solve."""
        t0 = np.zeros(1, dtype=np.int64)
        done = np.zeros(self.G, dtype=np.int64)
        _check(lib().como3r_solve_timestamps(self.handle, t0.ctypes.data_as(_i64p), done.ctypes.data_as(_i64p)),
               "solve_timestamps")
        return int(t0[0]), done

    def last_step(self, tau_out=None):
        """como3r_last_step: the step tau [N, 7] of the last iteration (host float64)."""
        tau = tau_out if tau_out is not None else np.zeros((self.prob.num_kf, 7))
        _check(lib().como3r_last_step(self.handle, _ptr(tau)), "last_step")
        return tau

    def linearize(self, poses, edge_out=None):
        cost = np.zeros(self.G)
        st = _check(lib().como3r_linearize(self.handle, _ptr(poses), _ptr(edge_out), cost.ctypes.data_as(_f64p)),
                    "linearize")
        return st, cost

    def update_inputs(self, points=None, match_idx=None):
        _check(lib().como3r_update_inputs(self.handle, _ptr(points), _ptr(match_idx)), "update_inputs")

    def time_stages(self, poses, reps: int = 10) -> dict:
        """Mean per-kernel durations (ms) from CUDA events on the library's stream."""
        ms = (ctypes.c_float * 7)()
        _check(lib().como3r_time_stages(self.handle, _ptr(poses), int(reps), ms), "time_stages")
        return dict(zip(STAGE_NAMES, [float(x) for x in ms]))

    def vjp(self, poses_init, iters: int, mode: int = VJP_UNROLLED, upstream: float = 1.0, grad_logdepth=None,
            grad_conf=None, poses_out=None):
        """como3r_vjp: (status, grad_logdepth, grad_conf, loss per graph); the gradients are
        float32 CUDA tensors over the packed pixels (allocated here unless given)."""
        import torch
        P = int(self.prob.points.shape[0])
        dev = self.points.device if self.points.is_cuda else torch.device("cuda")
        gl = grad_logdepth if grad_logdepth is not None else torch.empty(P, dtype=torch.float32, device=dev)
        gc = grad_conf if grad_conf is not None else torch.empty(P, dtype=torch.float32, device=dev)
        loss = np.zeros(self.G)
        st = _check(lib().como3r_vjp(self.handle, _ptr(poses_init), int(iters), int(mode), float(upstream), _ptr(gl),
                                     _ptr(gc), _ptr(poses_out), loss.ctypes.data_as(_f64p)), "vjp")
        return st, gl, gc, loss

    def time_vjp(self, poses_init, iters: int, reps: int = 3) -> dict:
        """Mean durations (ms) of the parts of an unrolled como3r_vjp (CUDA events)."""
        ms = (ctypes.c_float * 4)()
        _check(lib().como3r_time_vjp(self.handle, _ptr(poses_init), int(iters), int(reps), ms), "time_vjp")
        return dict(zip(["forward", "envelope", "backward", "adjoint_match"], [float(x) for x in ms]))

    def last_launch_count(self) -> int:
        return int(lib().como3r_last_launch_count(self.handle))

    def stats(self) -> dict:
        out = (ctypes.c_int64 * len(STAT_NAMES))()
        _check(lib().como3r_graph_stats(self.handle, out), "graph_stats")
        return dict(zip(STAT_NAMES, list(out)))


def _info_dict(x: GraphInfo) -> dict:
    return dict(cost=x.cost, attempts=x.attempts, solved=bool(x.solved), valid_matches=x.valid_matches,
                skipped_matches=x.skipped_matches)


def sim3_retract(tau, poses, stream=None) -> None:
    """poses[k] <- Exp(tau[k]) poses[k] on the device (tau [n, 7], poses [n, 8], float64 CUDA tensors)."""
    n = int(poses.shape[0])
    _check(lib().como3r_sim3_retract(_ptr(tau), _ptr(poses), n, _torch_stream(stream)), "sim3_retract")


def linearize_noalloc(prob, poses, edge_out, mode: int = MIXED, points=None, match_idx=None, stream=None) -> int:
    """como3r_linearize_noalloc: per-edge records into `edge_out` without any allocation
    by the library (inputs must already be device tensors; see include/como3r.h)."""
    keep = []
    d = _build_desc(prob, _ptr(points), _ptr(match_idx), mode, False, keep)
    return _check(lib().como3r_linearize_noalloc(ctypes.byref(d), _ptr(poses), _ptr(edge_out), _torch_stream(stream)),
                  "linearize_noalloc")


def points_from_logdepth(rays, logdepth, conf, points_out, stream=None) -> None:
    """points_out[p] = (exp(logdepth[p]) * rays[p], conf[p]) in points_out's storage type
    (float16 / float32 / float64 CUDA tensor [n, 4]); rays [n, 3], logdepth / conf [n] float32."""
    import torch
    code = {torch.float16: F16, torch.float32: F32, torch.float64: F64}[points_out.dtype]
    n = int(points_out.shape[0])
    _check(lib().como3r_points_from_logdepth(_ptr(rays), _ptr(logdepth), _ptr(conf), n, code, _ptr(points_out),
                                             _torch_stream(stream)), "points_from_logdepth")


def rays_from_points(points, stream=None):
    """(rays [n, 3], logdepth [n], conf [n]) float32 CUDA tensors split from packed points."""
    import torch
    code = {torch.float16: F16, torch.float32: F32, torch.float64: F64}[points.dtype]
    n = int(points.shape[0])
    rays = torch.empty((n, 3), dtype=torch.float32, device=points.device)
    ld = torch.empty(n, dtype=torch.float32, device=points.device)
    cf = torch.empty(n, dtype=torch.float32, device=points.device)
    _check(lib().como3r_rays_from_points(_ptr(points), n, code, _ptr(rays), _ptr(ld), _ptr(cf), _torch_stream(stream)),
           "rays_from_points")
    return rays, ld, cf


def _make_cost_function():
    import torch

    class Como3rCost(torch.autograd.Function):
        """L(logdepth, conf) = refined cost after `iters` GN iterations from poses_init
        (sum over graphs), with a backward pass through como3r_vjp.

        forward(logdepth [P] f32, conf [P] f32, graph, rays [P, 3] f32, poses_init [N, 8]
        f64 CUDA, iters, mode) packs the pointmaps into the buffer the graph borrows
        (graph.points), runs the iterations and returns L as a float64 scalar tensor."""

        @staticmethod
        def forward(ctx, logdepth, conf, graph, rays, poses_init, iters, mode=VJP_UNROLLED):
            points_from_logdepth(rays, logdepth.detach().contiguous(), conf.detach().contiguous(), graph.points)
            work = poses_init.detach().clone()
            _, trace, _ = graph.solve(work, int(iters), trace=True)
            ctx.graph, ctx.iters, ctx.mode = graph, int(iters), int(mode)
            ctx.save_for_backward(poses_init)
            return torch.tensor(float(trace[-1].sum()), dtype=torch.float64, device=logdepth.device)

        @staticmethod
        def backward(ctx, grad_out):
            (poses_init,) = ctx.saved_tensors
            _, gl, gc, _ = ctx.graph.vjp(poses_init, ctx.iters, ctx.mode, upstream=float(grad_out))
            return gl, gc, None, None, None, None, None

    return Como3rCost


_cost_fn = None


def refined_cost(logdepth, conf, graph: "Graph", rays, poses_init, iters: int, mode: int = VJP_UNROLLED):
    """Differentiable refined cost (torch.autograd): see Como3rCost."""
    global _cost_fn
    if _cost_fn is None:
        _cost_fn = _make_cost_function()
    return _cost_fn.apply(logdepth, conf, graph, rays, poses_init, iters, mode)


def exported_symbols(header: str) -> Sequence[str]:
    """Names of the functions a header declares (used by the ABI-load test)."""
    import re
    txt = open(header).read()
    return re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(como3r_[a-z_0-9]+)\s*\(", txt, flags=re.M)


def gauge_sync(points, dtype: int, pix_off, kf_i, kf_j, match_ij, match_ji, poses, q_min: float = 1.5,
               nu_min: float = 0.1, nc_min: int = 64, mode: int = MIXED, stream=None, timing: bool = False):
    """como3r_gauge_sync over candidates (kf_i[c], kf_j[c]) (Sec. III-B/III-C).

    points, match_ij, match_ji: CUDA tensors (packed pixels; per-candidate match rows
    concatenated); pix_off: int64 [num_kf + 1]; poses: [num_kf][8] (host or device).
    Returns a list of dicts (T as a (t, q, s) array, nu_i, nu_j, n_i, n_j, valid_i, valid_j,
    admitted, fallback), plus the kernel time in ms when `timing`."""
    pix_off = np.ascontiguousarray(np.asarray(pix_off, dtype=np.int64))
    kf_i = np.ascontiguousarray(np.asarray(kf_i, dtype=np.int32))
    kf_j = np.ascontiguousarray(np.asarray(kf_j, dtype=np.int32))
    C = int(kf_i.size)
    d = GaugeDesc(num_candidates=C, num_kf=int(pix_off.size - 1),
                  pix_off=pix_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), points_conf=_ptr(points),
                  dtype=int(dtype), kf_i=kf_i.ctypes.data_as(_i32p), kf_j=kf_j.ctypes.data_as(_i32p),
                  match_ij=_ptr(match_ij), match_ji=_ptr(match_ji), poses=_ptr(poses), q_min=float(q_min),
                  nu_min=float(nu_min), nc_min=int(nc_min), mode=int(mode))
    out = (GaugeResult * max(C, 1))()
    ms = ctypes.c_float(0.0)
    _check(lib().como3r_gauge_sync(ctypes.byref(d), _torch_stream(stream), out,
                                   ctypes.byref(ms) if timing else None), "gauge_sync")
    res = [dict(T=np.array(list(r.T)), nu_i=r.nu_i, nu_j=r.nu_j, n_i=int(r.n_i), n_j=int(r.n_j),
                valid_i=int(r.valid_i), valid_j=int(r.valid_j), admitted=bool(r.admitted), fallback=int(r.fallback))
           for r in out[:C]]
    return (res, float(ms.value)) if timing else res


def gauge_transport(poses, which, T, stream=None):
    """como3r_gauge_transport: poses[k] <- T[which[k]] poses[k] for which[k] >= 0 (CUDA tensors)."""
    _check(lib().como3r_gauge_transport(_ptr(poses), int(poses.shape[0]), _ptr(which), _ptr(T), int(T.shape[0]),
                                        _torch_stream(stream)), "gauge_transport")


def terminal_refine(graph: "Graph", poses, labels, rounds: int = 3, depth_iters: int = 10, pose_iters: int = 50,
                    **params):
    """Terminal schedule (Sec. III-E): `rounds` times, up to `depth_iters` Jacobi structure
    steps at fixed poses (como3r_depth_refine, eta carried over), then a pose pass of
    `pose_iters` Gauss-Newton iterations (como3r_solve) on the refined pointmaps.  The
    segments are built from the graph's pointmaps at the call (the pristine snapshot).
    Returns (poses [N][8] as a numpy array, eta [M])."""
    import torch
    M = graph.depth_setup(labels, **params)
    eta = np.zeros(M)
    work = torch.tensor(np.asarray(poses, dtype=np.float64), device="cuda")
    buf = torch.empty(graph.points.shape, dtype=graph.points.dtype, device="cuda")
    for _ in range(rounds):
        eta, _ = graph.depth_refine(work, eta, depth_iters, points_out=buf)
        if graph.copy_inputs:
            graph.update_inputs(points=buf)
        else:
            graph.points.copy_(buf)
        graph.solve(work, pose_iters, trace=False)
    return work.cpu().numpy(), eta


def project_match(frame_points, H: int, W: int, query_points, dtype: int = F32, init=None, max_steps: int = 64,
                  max_angle: float = 0.01, stream=None, with_dist: bool = False):
    """como3r_project_match on CUDA tensors; returns int32 matches (and FP32 distances)."""
    import torch
    Q = int(query_points.shape[0])
    match = torch.empty(Q, dtype=torch.int32, device=query_points.device)
    dist = torch.empty(Q, dtype=torch.float32, device=query_points.device) if with_dist else None
    d = MatchDesc(H=int(H), W=int(W), frame_points=_ptr(frame_points), query_points=_ptr(query_points),
                  num_queries=Q, dtype=int(dtype), init=_ptr(init), max_steps=int(max_steps),
                  max_angle=float(max_angle))
    _check(lib().como3r_project_match(ctypes.byref(d), _ptr(match), _ptr(dist), _torch_stream(stream)),
           "project_match")
    return (match, dist) if with_dist else match


def fuse_packed(canon, pred, pix_off, T_kf, dtype: int = F32, stream=None):
    """como3r_fuse_packed: every keyframe q (rows pix_off[q] .. pix_off[q+1]-1 of the packed
    canon / pred CUDA tensors) fused in place with its own pose T_kf[q] (one launch per 128)."""
    off = np.ascontiguousarray(np.asarray(pix_off, dtype=np.int64))
    T = np.ascontiguousarray(np.asarray(T_kf, dtype=np.float64).reshape(-1, 8))
    if T.shape[0] != off.shape[0] - 1:
        raise ValueError("T_kf needs one pose per keyframe of pix_off")
    _check(lib().como3r_fuse_packed(_ptr(canon), _ptr(pred), off.ctypes.data_as(_i64p), T.ctypes.data_as(_f64p),
                                    int(T.shape[0]), int(dtype), _torch_stream(stream)), "fuse_packed")
    return canon


def fuse(canon, pred, T_kf, dtype: int = F32, stream=None):
    """como3r_fuse: canon <- confidence-weighted running average with T_kf pred (in place)."""
    T = np.ascontiguousarray(np.asarray(T_kf, dtype=np.float64))
    _check(lib().como3r_fuse(_ptr(canon), _ptr(pred), int(canon.shape[0]), int(dtype), T.ctypes.data_as(_f64p),
                             _torch_stream(stream)), "fuse")
    return canon

