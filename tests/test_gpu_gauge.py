"""Cross-agent candidate verification and gauge synchronisation on the GPU
(como3r_gauge_sync / como3r_gauge_transport, Sec. III-B/III-C) against the oracle.

Integer results (valid and high-confidence match counts, hence nu, the admission decision
and the fallback choice) must be equal; T* within 1e-5 (rotation angle, relative scale,
translation relative to the larger of |t| and 1) in the mixed form and 1e-9 in the FP64
form.  Candidates are the inter-agent pairs of shared-canvas teams listed in both
directions."""
import numpy as np
import pytest

from oracle import como3r_oracle as O
from tests.gpu_helpers import pose_err

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


def team(seed, dtype=np.float32, **kw):
    from synth import make_cloud_problem
    spec = dict(agents=3, n_kf=8, H=48, W=64, period=30, shift=6, n_inter=4, reverse_inter=True, noise=0.01,
                outlier=0.1)
    spec.update(kw)
    return make_cloud_problem(seed, [spec], dtype=dtype)


def candidates(p):
    """(kf_i, kf_j, fwd rows, bwd rows) of the inter-agent pairs listed in both directions."""
    E = p.num_edges
    px = p.pixels_of().astype(np.int64)
    slots = np.concatenate([[0], np.cumsum(px[p.edge_i.astype(np.int64)])])
    def paired(n):
        return all((p.edge_i[E - 2 * n + k], p.edge_j[E - 2 * n + k]) == (p.edge_j[E - n + k], p.edge_i[E - n + k])
                   for k in range(n))
    n = next(n for n in range(E // 2, 0, -1) if paired(n))
    fw = list(range(E - 2 * n, E - n))
    bw = list(range(E - n, E))
    for a, b in zip(fw, bw):
        assert (p.edge_i[a], p.edge_j[a]) == (p.edge_j[b], p.edge_i[b])
    kf_i = p.edge_i[fw].astype(np.int32)
    kf_j = p.edge_j[fw].astype(np.int32)
    rows_f = [p.match_idx[slots[e]:slots[e + 1]] for e in fw]
    rows_b = [p.match_idx[slots[e]:slots[e + 1]] for e in bw]
    return kf_i, kf_j, rows_f, rows_b


def run(C, p, poses, q_min=1.5, nu_min=0.1, nc_min=64, mode=None, rows=None):
    import torch
    kf_i, kf_j, rows_f, rows_b = rows or candidates(p)
    dtype = {np.float16: C.F16, np.float32: C.F32, np.float64: C.F64}[p.points.dtype.type]
    pts = torch.from_numpy(np.ascontiguousarray(p.points)).cuda()
    mij = torch.from_numpy(np.concatenate(rows_f).astype(np.int32)).cuda()
    mji = torch.from_numpy(np.concatenate(rows_b).astype(np.int32)).cuda()
    pix_off = np.concatenate([[0], np.cumsum(p.pixels_of())]).astype(np.int64)
    return C.gauge_sync(pts, dtype, pix_off, kf_i, kf_j, mij, mji, np.ascontiguousarray(poses), q_min=q_min,
                        nu_min=nu_min, nc_min=nc_min, mode=C.MIXED if mode is None else mode)


def oracle(p, poses, q_min=1.5, nu_min=0.1, nc_min=64, rows=None):
    kf_i, kf_j, rows_f, rows_b = rows or candidates(p)
    px = p.pixels_of().astype(np.int64)
    off = np.concatenate([[0], np.cumsum(px)])
    out = []
    for i, j, f, b in zip(kf_i, kf_j, rows_f, rows_b):
        Pi = p.points[off[i]:off[i + 1]].astype(np.float64)
        Pj = p.points[off[j]:off[j + 1]].astype(np.float64)
        out.append(O.gauge_candidate(O.pose_to_matrix(poses[i]), O.pose_to_matrix(poses[j]), Pi, Pj, f, b,
                                     q_min=q_min, nu_min=nu_min, nc_min=nc_min))
    return out


def check(got, want, tol):
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert (g["n_i"], g["n_j"]) == (w["n_i"], w["n_j"])
        assert g["nu_i"] == w["nu_i"] and g["nu_j"] == w["nu_j"]
        assert g["admitted"] == w["admitted"]
        assert (g["fallback"] > 0) == w["fallback"]
        wt = O.matrix_to_pose(w["T"])
        err = O.pose_errors(g["T"][None, :], wt[None, :], ref_scale=1.0)
        assert max(err.values()) <= tol, (err, g, w)


@pytest.mark.parametrize("dtype", [np.float16, np.float32, np.float64])
def test_gauge_sync_matches_oracle(C, dtype):
    p = team(41, dtype=dtype)
    seen = []
    for q_min in (1.5, 3.0, 8.0):  # 8.0: few matches pass, so rejected candidates and fallbacks occur
        want = oracle(p, p.poses_init, q_min=q_min)
        check(run(C, p, p.poses_init, q_min=q_min), want, 1e-5)
        check(run(C, p, p.poses_init, q_min=q_min, mode=C.PLAIN_FP64), want, 1e-9)
        seen += [(w["admitted"], w["fallback"]) for w in want]
    assert (True, False) in seen and (False, True) in seen


def test_gauge_sync_recovers_extra_similarity_and_transport_restores(C):
    import torch
    p = team(42, dtype=np.float64, noise=0.0, outlier=0.0)  # exact to FP64: the 1e-9 check needs it
    rng = np.random.default_rng(3)
    G = O.exp_sim3(np.concatenate([rng.normal(size=3) * 2, rng.normal(size=3) * 0.6, [0.3]]))
    poses = p.poses_gt.copy()
    moving = p.agent_of == 2
    for k in np.nonzero(moving)[0]:
        poses[k] = O.matrix_to_pose(G @ O.pose_to_matrix(poses[k]))
    kf_i, kf_j, rf, rb = candidates(p)
    sel = [c for c in range(len(kf_i)) if p.agent_of[kf_j[c]] == 2 and p.agent_of[kf_i[c]] != 2]
    assert sel
    rows = (kf_i[sel], kf_j[sel], [rf[c] for c in sel], [rb[c] for c in sel])
    for mode, tol in ((C.MIXED, 1e-5), (C.PLAIN_FP64, 1e-9)):
        res = run(C, p, poses, q_min=0.0, rows=rows, mode=mode)
        Ginv = O.matrix_to_pose(O.sim3_inverse(G))
        for r in res:
            assert r["fallback"] == 0
            assert max(O.pose_errors(r["T"][None], Ginv[None], ref_scale=1.0).values()) <= tol
        Td = torch.tensor(np.stack([res[0]["T"]]), dtype=torch.float64, device="cuda")
        which = torch.tensor(np.where(moving, 0, -1), dtype=torch.int32, device="cuda")
        pd = torch.tensor(poses, dtype=torch.float64, device="cuda")
        C.gauge_transport(pd, which, Td)
        torch.cuda.synchronize()
        assert max(pose_err(pd.cpu().numpy(), p.poses_gt).values()) <= 10 * tol


def test_gauge_sync_fallback_boundary_and_errors(C):
    import torch
    p = team(43)
    # too few correspondences: the endpoint transform, T* T_j = T_i
    res = run(C, p, p.poses_init, nc_min=10 ** 9)
    kf_i, kf_j, rf, rb = candidates(p)
    for r, i, j in zip(res, kf_i, kf_j):
        assert r["fallback"] == 1
        T = O.pose_to_matrix(r["T"])
        np.testing.assert_allclose(T @ O.pose_to_matrix(p.poses_init[j]), O.pose_to_matrix(p.poses_init[i]),
                                   atol=1e-12)
    # c_m c_n exactly q_min^2 where the FP32-rounded product falls below it: counted
    q = 1.0 + 2.0 ** -12
    pts = p.points.copy()
    pts[:, 3] = np.float32(q)
    pb = type(p)(**{**p.__dict__, "points": pts})
    got = run(C, pb, p.poses_init, q_min=q)
    want = oracle(pb, p.poses_init, q_min=q)
    assert all(w["n_i"] == w_["valid_i"] for w, w_ in zip(want, got))  # every finite valid match passes
    check(got, want, 1e-5)
    # no candidates; a match index out of range is an error
    pix_off = np.concatenate([[0], np.cumsum(p.pixels_of())]).astype(np.int64)
    empty = torch.zeros(1, dtype=torch.int32, device="cuda")
    pts_d = torch.from_numpy(p.points).cuda()
    assert C.gauge_sync(pts_d, C.F32, pix_off, [], [], empty, empty, p.poses_init) == []
    bad = [r.copy() for r in rf]
    bad[0][5] = 10 ** 6
    with pytest.raises(C.Como3rError):
        run(C, p, p.poses_init, rows=(kf_i, kf_j, bad, rb))


def test_gauge_sync_full_size_sampled(C):
    """60 candidates at 512x384 (4 agents x 40 keyframes, FP32, generated in device
    memory); three sampled candidates against the oracle, all counts consistent."""
    import torch
    from synth import graph_subproblem, make_cloud_batch_gpu
    spec = [dict(agents=4, n_kf=40, H=384, W=512, period=40, shift=51, n_inter=60, reverse_inter=True,
                 noise=0.01, outlier=0.15)]
    prob, pts, midx = make_cloud_batch_gpu(7, spec, device="cuda")
    E, P = prob.num_edges, 384 * 512
    fw, bw = list(range(E - 120, E - 60)), list(range(E - 60, E))
    assert all((prob.edge_i[a], prob.edge_j[a]) == (prob.edge_j[b], prob.edge_i[b]) for a, b in zip(fw, bw))
    mij = torch.cat([midx[e * P:(e + 1) * P] for e in fw])
    mji = torch.cat([midx[e * P:(e + 1) * P] for e in bw])
    pix_off = np.arange(prob.num_kf + 1, dtype=np.int64) * P
    res = C.gauge_sync(pts, C.F32, pix_off, prob.edge_i[fw], prob.edge_j[fw], mij, mji, prob.poses_init)
    assert len(res) == 60 and all(r["valid_i"] > 0 for r in res)
    sub = graph_subproblem(prob, pts, midx, 0)
    for c in (0, 29, 59):
        e_f, e_b = fw[c], bw[c]
        rows = (np.array([prob.edge_i[e_f]]), np.array([prob.edge_j[e_f]]), [sub.match_idx[e_f * P:(e_f + 1) * P]],
                [sub.match_idx[e_b * P:(e_b + 1) * P]])
        check([res[c]], oracle(sub, prob.poses_init, rows=rows), 1e-5)
