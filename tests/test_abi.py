"""CPU checks of the boundary: the library loads, exports every declared symbol, and its
host planner validates descriptions and plans the factorisation without a GPU."""
import ctypes
import copy
import os

import numpy as np
import pytest

from synth import make_problem, make_workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def C():
    from paper_2605_30488_b300 import build
    build.build()
    from paper_2605_30488_b300 import como3r
    return como3r


def test_every_declared_symbol_is_exported(C):
    names = C.exported_symbols(os.path.join(ROOT, "include", "como3r.h"))
    assert "como3r_graph_create" in names and "como3r_solve" in names
    lib = ctypes.CDLL(C.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_plan_of_small_problem(C):
    p = make_workload("two_agent_6kf_64x48")
    s = C.plan_stats(p)
    assert s["keyframes"] == 12 and s["edges"] == 14 and s["columns"] == 11
    assert s["blocks"] >= 11 + 13  # diagonals + at least the non-anchor edges' pairs
    assert s["items"] == 14 * -(-3072 // s["chunk"])  # ceil(3072 px / chunk) items per edge


def test_plan_depth_is_logarithmic_on_a_long_chain(C):
    # a 200-keyframe chain with (k, k+1) and (k, k+3) edges; the planner never reads pixels
    n = 200
    class T:  # minimal problem-like object
        pass
    t = T()
    t.kf_offset = np.array([0, n]); t.height = np.array([2]); t.width = np.array([2])
    t.agent_of = np.zeros(n, np.int32); t.edge_offset = np.array([0, 2 * n - 4])
    ei = [k for k in range(n - 1)] + [k for k in range(n - 3)]
    ej = [k + 1 for k in range(n - 1)] + [k + 3 for k in range(n - 3)]
    t.edge_i = np.array(ei); t.edge_j = np.array(ej); t.edge_offset = np.array([0, len(ei)])
    t.anchor = np.array([0]); t.points = np.zeros((4 * n, 4), np.float32); t.match_idx = np.zeros(1, np.int32)
    t.sigma_ray, t.sigma_dist, t.huber_k, t.lam, t.eps0, t.max_attempts = 0.003, 10.0, 1.345, 0.0, 1e-6, 6
    s = C.plan_stats(t)
    assert s["columns"] == n - 1
    assert s["levels"] <= 40, s   # a minimum-degree order would give ~n levels


@pytest.mark.parametrize("mutate,msg", [
    (lambda p: setattr(p, "edge_j", np.where(np.arange(len(p.edge_j)) == 0, p.edge_i, p.edge_j)), "i == j"),
    (lambda p: setattr(p, "edge_j", np.where(np.arange(len(p.edge_j)) == 1, 999, p.edge_j)), "outside"),
    (lambda p: setattr(p, "sigma_ray", -1.0), "sigma"),
    (lambda p: setattr(p, "max_attempts", 0), "max_attempts"),
    (lambda p: setattr(p, "anchor", np.array([99])), "anchor"),
])
def test_invalid_descriptions_rejected(C, mutate, msg):
    p = copy.deepcopy(make_workload("two_agent_6kf_64x48"))
    mutate(p)
    with pytest.raises(C.Como3rError) as ei:
        C.plan_stats(p)
    assert ei.value.code == C.ERR_INVALID_ARG
    assert msg in str(ei.value)


def test_fuse_packed_arguments_checked_on_the_host(C):
    """como3r_fuse_packed rejects bad offsets, NULL buffers and FP16 storage before touching
    the GPU, and an empty batch is a no-op (every case here returns before any CUDA call)."""
    lib = ctypes.CDLL(C.LIB_PATH)
    f = lib.como3r_fuse_packed
    vp, i64p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    f.argtypes = [vp, vp, i64p, f64p, ctypes.c_int32, ctypes.c_int32, vp]
    f.restype = ctypes.c_int
    pose = np.zeros((2, 8))
    pose[:, 6] = pose[:, 7] = 1.0
    buf = np.zeros(64, dtype=np.float32)  # stands in for device buffers; never dereferenced here

    def call(off, n, dtype=C.F32, data=True):
        o = np.ascontiguousarray(np.asarray(off, dtype=np.int64))
        p = buf.ctypes.data if data else None
        return f(p, p, o.ctypes.data_as(i64p), pose.ctypes.data_as(f64p), n, dtype, None)

    assert call([0, 0, 0], 2) == C.OK              # nothing to fuse
    assert call([0], 0) == C.OK                    # no keyframes
    assert call([0, 4], -1) == C.ERR_INVALID_ARG   # negative count
    assert call([1, 4], 1) == C.ERR_INVALID_ARG    # offsets must start at 0
    assert call([0, 4, 2], 2) == C.ERR_INVALID_ARG  # and not decrease
    assert call([0, 4], 1, data=False) == C.ERR_INVALID_ARG
    assert call([0, 4], 1, dtype=C.F16) == C.ERR_UNSUPPORTED
    assert f(buf.ctypes.data, buf.ctypes.data, None, pose.ctypes.data_as(f64p), 1, C.F32, None) == C.ERR_INVALID_ARG


def test_fuse_packed_checks_every_quaternion_before_any_launch(C):
    """A zero quaternion in a later batch of 128 keyframes is rejected before the first batch
    is launched, so a rejected call leaves canon untouched (the buffers below are host
    memory that no CUDA call may touch: the call must return before any)."""
    lib = ctypes.CDLL(C.LIB_PATH)
    f = lib.como3r_fuse_packed
    vp, i64p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    f.argtypes = [vp, vp, i64p, f64p, ctypes.c_int32, ctypes.c_int32, vp]
    f.restype = ctypes.c_int
    n = 300
    pose = np.zeros((n, 8))
    pose[:, 6] = pose[:, 7] = 1.0
    pose[200, 3:7] = 0.0  # keyframe 200 lies in the second launch batch
    off = np.arange(n + 1, dtype=np.int64) * 4
    buf = np.zeros(4 * 4 * n, dtype=np.float32)
    assert f(buf.ctypes.data, buf.ctypes.data, off.ctypes.data_as(i64p), pose.ctypes.data_as(f64p), n, C.F32,
             None) == C.ERR_INVALID_ARG
    assert "quaternion" in lib_last_error(C)
    assert not buf.any()


def lib_last_error(C):
    return C.lib().como3r_last_error().decode()
