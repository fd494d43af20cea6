"""The allocation-free linearisation entry point, compared with the handle-based one.

como3r_linearize_noalloc serves callers that cannot allocate device memory when they
need a linearisation (during CUDA-graph capture, in real-time loops, under a framework
that owns the memory budget); it keeps all intermediates in one static device array
that every call reuses.  This file is collected last on purpose.  Each case calls the
entry point twice in a row through the C ABI, so a second call must not be disturbed by
what the first left in the shared array, and compares both with como3r_linearize within
the tolerances of the parity tests (FP64 form 1e-9, mixed form 1e-5 relative).
"""
import numpy as np
import pytest

from synth import make_problem, make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30488_b300 import build
    build.build()
    from paper_2605_30488_b300 import como3r
    return como3r


def _cases():
    tiny = make_workload("two_agent_6kf_64x48", seed=0)
    mid = make_problem(5, agents=2, n_kf=8, H=120, W=160, f=125.0, noise=0.01, conf="lognormal",
                       outlier=0.15, skip_max=4, n_inter=4, exact=False, dtype=np.float32, name="mid")
    return [(tiny, "plain", 1e-9), (mid, "mixed", 1e-5), (tiny, "mixed", 1e-5)]


def test_noalloc_matches_handle_linearize_on_two_calls(C):
    import torch
    for prob, mode_name, tol in _cases():
        mode = C.PLAIN_FP64 if mode_name == "plain" else C.MIXED
        poses = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
        pts = torch.from_numpy(np.ascontiguousarray(prob.points)).cuda()
        idx = torch.from_numpy(np.ascontiguousarray(prob.match_idx)).cuda()
        ref = torch.zeros((prob.num_edges, C.EDGE_RECORD), dtype=torch.float64, device="cuda")
        with C.Graph(prob, mode=mode, points=pts, match_idx=idx) as g:
            g.linearize(poses, ref)
        ref = ref.cpu().numpy()
        for call in range(2):
            out = torch.full((prob.num_edges, C.EDGE_RECORD), np.nan, dtype=torch.float64, device="cuda")
            st = C.linearize_noalloc(prob, poses, out, mode, points=pts, match_idx=idx)
            torch.cuda.synchronize()
            assert st == C.OK
            got = out.cpu().numpy()
            for e in range(prob.num_edges):
                Hr, Hg = ref[e, :49], got[e, :49]
                assert np.linalg.norm(Hg - Hr) <= tol * np.linalg.norm(Hr), (mode_name, call, e)
                gscale = max(np.linalg.norm(ref[e, 49:56]), 1e-3 * np.sqrt(np.abs(Hr[::8]).max()))
                assert np.linalg.norm(got[e, 49:56] - ref[e, 49:56]) <= max(tol, 1e-9) * 10 * gscale
                assert abs(got[e, 56] - ref[e, 56]) <= tol * max(ref[e, 56], 1e-300)
                assert got[e, 57] == ref[e, 57] and got[e, 58] == ref[e, 58]


def test_noalloc_rejects_too_many_edges(C):
    import copy
    import torch
    prob = copy.deepcopy(make_workload("two_agent_6kf_64x48", seed=0))
    reps = 2049  # one edge more than COMO3R_NOALLOC_MAX_EDGES
    prob.edge_i = np.resize(prob.edge_i, reps)
    prob.edge_j = np.resize(prob.edge_j, reps)
    prob.edge_offset = np.array([0, reps], np.int32)
    pts = torch.from_numpy(np.ascontiguousarray(prob.points)).cuda()
    idx = torch.zeros(reps * 3072, dtype=torch.int32, device="cuda")
    poses = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
    out = torch.zeros((reps, C.EDGE_RECORD), dtype=torch.float64, device="cuda")
    with pytest.raises(C.Como3rError) as ei:
        C.linearize_noalloc(prob, poses, out, C.MIXED, points=pts, match_idx=idx)
    assert ei.value.code == C.ERR_INVALID_ARG
