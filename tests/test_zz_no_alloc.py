"""The allocation-free linearisation entry point, against the oracle and the handle-based one.

como3r_linearize_noalloc serves callers that cannot allocate device memory when they
need a linearisation (real-time loops that must not wait on the allocator, frameworks
that own the whole memory budget); it keeps all intermediates in one static device array
that every call reuses.  This file is collected last on purpose.  Each case calls the
entry point twice in a row through the C ABI and checks both calls' per-edge records
against the FP64 oracle's H_rel, g_rel, cost and counts (FP64 form 1e-9, mixed form
1e-5 relative, the parity tests' tolerances) and against como3r_linearize.  The cases run
in the order large mixed problem, then small FP64 problem, so the small call finds the
shared array filled by a larger one and must not be disturbed by what is left there.
"""
import numpy as np
import pytest

from oracle import como3r_oracle as O
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


def _mid():
    return make_problem(5, agents=2, n_kf=8, H=120, W=160, f=125.0, noise=0.01, conf="lognormal",
                        outlier=0.15, skip_max=4, n_inter=4, exact=False, dtype=np.float32, name="mid")


def _check_records(got, recs, tol, what):
    """Per-edge records [E, 64] against the oracle's linearize_edge results."""
    for e, r in enumerate(recs):
        Hg = got[e, :49].reshape(7, 7)
        assert np.linalg.norm(Hg - r["H_rel"]) <= tol * np.linalg.norm(r["H_rel"]), (what, e)
        gscale = max(np.linalg.norm(r["g_rel"]), 1e-3 * np.sqrt(np.abs(np.diag(r["H_rel"])).max()))
        assert np.linalg.norm(got[e, 49:56] - r["g_rel"]) <= (tol if tol < 1e-6 else 1e-4) * gscale, (what, e)
        assert abs(got[e, 56] - r["cost"]) <= tol * max(r["cost"], 1e-300), (what, e)
        assert got[e, 57] == r["n_valid"] and got[e, 58] == r["n_skipped"], (what, e)


def test_noalloc_matches_oracle_and_handle_on_two_calls(C):
    import torch
    tiny = make_workload("two_agent_6kf_64x48", seed=0)
    mid = _mid()
    # large first: the small FP64 calls then run on a shared array a larger mixed call filled
    for prob, mode_name, tol in [(mid, "mixed", 1e-5), (tiny, "plain", 1e-9), (tiny, "mixed", 1e-5),
                                 (mid, "plain", 1e-9), (tiny, "plain", 1e-9)]:
        mode = C.PLAIN_FP64 if mode_name == "plain" else C.MIXED
        poses = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
        pts = torch.from_numpy(np.ascontiguousarray(prob.points)).cuda()
        idx = torch.from_numpy(np.ascontiguousarray(prob.match_idx)).cuda()
        _, _, _, recs = O.build_system(prob, prob.poses_init, 0)
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
            _check_records(got, recs, tol, (prob.name, mode_name, call))
            # and the handle-based call on the same inputs, at the same tolerance
            for e in range(prob.num_edges):
                Hr, Hg = ref[e, :49], got[e, :49]
                assert np.linalg.norm(Hg - Hr) <= tol * np.linalg.norm(Hr), (prob.name, mode_name, call, e)
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
    assert "COMO3R_NOALLOC_MAX_EDGES" in str(ei.value)
