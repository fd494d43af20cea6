"""Segment-level structure refinement on the GPU (como3r_depth_setup / como3r_depth_refine,
Sec. III-E) against the oracle: the segment count, eta after the Jacobi steps and the
objective trace within 1e-5 (mixed: FP32 per-match arithmetic, FP64 sums and steps) and
1e-9 (plain FP64); the refined pointmaps; the clip and fixed-segment rules; one step of
the 2 x 40 workload at 512 x 384 with 200 segments per keyframe; and the terminal
alternation of depth steps with pose passes."""
import dataclasses

import numpy as np
import pytest

from oracle import como3r_oracle as O
from synth.segments import perturb_segment_ranges, problem_labels

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


def case(seed=61, dtype=np.float32, sigma=0.05, noise=0.01, outlier=0.1, n_seg=12, **kw):
    from synth import make_cloud_problem
    spec = dict(agents=2, n_kf=5, H=32, W=40, period=30, shift=5, n_inter=2, noise=noise, outlier=outlier)
    spec.update(kw)
    p = make_cloud_problem(seed, [spec], dtype=dtype)
    lab = problem_labels(p, n_seg=n_seg, seed=seed)
    pix_off = np.concatenate([[0], np.cumsum(p.pixels_of())])
    pts = perturb_segment_ranges(p.points, lab, pix_off, sigma, seed=seed)
    return dataclasses.replace(p, points=pts), lab


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("mode", ["mixed", "plain"])
@pytest.mark.parametrize("chunk", ["1024", "2048"])
def test_depth_refine_matches_oracle(C, mode, chunk, monkeypatch):
    """Work items of 1024 pixels have the residual kernel's valid-match lists, which the
    match pass walks; items of 2048 pixels have none, and it reads the index rows."""
    import torch
    monkeypatch.setenv("COMO3R_K1_CHUNK", chunk)
    dtype = np.float32 if mode == "mixed" else np.float64
    p, lab = case(dtype=dtype)
    m = C.MIXED if mode == "mixed" else C.PLAIN_FP64
    tol = 1e-5 if mode == "mixed" else 1e-9
    seg = O.depth_segments(p, lab)
    eta_o, tr_o = O.depth_refine(p, p.poses_init, np.zeros(seg["M"]), 10, seg)
    with C.Graph(p, mode=m) as g:
        M = g.depth_setup(lab)
        assert M == seg["M"]
        eta = np.zeros(M)
        out = torch.empty_like(g.points)
        eta, tr = g.depth_refine(p.poses_init, eta, 10, points_out=out)
    assert np.abs(eta - eta_o).max() <= tol, np.abs(eta - eta_o).max()
    assert rel(tr, tr_o) <= tol
    assert tr[-1] < tr[0]
    # refined pointmaps: X(eta) for segment pixels, the snapshot elsewhere
    e = seg["eff"]
    d = np.exp(seg["logd"] + np.where(e >= 0, eta_o[np.maximum(e, 0)], 0.0))
    want = np.where((e >= 0)[:, None], d[:, None] * seg["psi"], p.points[:, :3].astype(np.float64))
    got = out.cpu().numpy().astype(np.float64)
    assert rel(got[:, :3], want) <= (2e-6 if mode == "mixed" else 1e-12)
    np.testing.assert_array_equal(got[:, 3], p.points[:, 3])


def test_depth_clip_fixed_and_storage_types(C):
    import torch
    for dtype in (np.float16, np.float32):
        p, lab = case(dtype=dtype, sigma=0.0)
        seg = O.depth_segments(p, lab)
        k = 6
        pix_off = np.concatenate([[0], np.cumsum(p.pixels_of())])
        s0 = int(seg["base"][k]) + 3
        pts = p.points.copy()
        sel = seg["eff"][pix_off[k]:pix_off[k + 1]] == s0
        pts[pix_off[k]:pix_off[k + 1]][sel, :3] = (pts[pix_off[k]:pix_off[k + 1]][sel, :3].astype(np.float64)
                                                  * np.exp(2.0)).astype(dtype)
        pb = dataclasses.replace(p, points=pts)
        segb = O.depth_segments(pb, lab)
        eta_o, tr_o = O.depth_refine(pb, pb.poses_init, np.zeros(segb["M"]), 3, segb)
        with C.Graph(pb, mode=C.MIXED) as g:
            M = g.depth_setup(lab)
            eta = torch.zeros(M, dtype=torch.float64, device="cuda")
            g.depth_refine(pb.poses_init, eta, 1)
            e1 = eta.cpu().numpy()
            g.depth_refine(pb.poses_init, eta, 2)
            e3 = eta.cpu().numpy()
        assert abs(e1[s0] + 0.5) < 1e-12
        assert np.all(e3[segb["fixed"]] == 0) and np.all(e3[~segb["active"]] == 0)
        assert np.abs(e3 - eta_o).max() <= 1e-5


def test_depth_one_step_bench_workload(C):
    """One Jacobi step of the 2 x 40 workload (512 x 384, FP32) with 200 segments per
    keyframe and per-segment range errors: eta and the objective against the oracle."""
    from synth import make_workload
    p0 = make_workload("two_agent_40kf_512x384", seed=0)
    lab = problem_labels(p0, n_seg=200, seed=1)
    pix_off = np.concatenate([[0], np.cumsum(p0.pixels_of())])
    p = dataclasses.replace(p0, points=perturb_segment_ranges(p0.points, lab, pix_off, 0.05, seed=1))
    seg = O.depth_segments(p, lab)
    eta_o, tr_o = O.depth_refine(p, p.poses_init, np.zeros(seg["M"]), 1, seg)
    with C.Graph(p, mode=C.MIXED) as g:
        M = g.depth_setup(lab)
        eta, tr = g.depth_refine(p.poses_init, np.zeros(M), 1)
    assert M == seg["M"] and M > 80 * 150
    assert np.abs(eta - eta_o).max() <= 1e-5
    assert rel(tr, tr_o) <= 1e-5


def test_terminal_alternation_matches_oracle(C):
    """Rounds of (depth steps at fixed poses, then a pose pass on the refined pointmaps):
    the GPU driver against the same alternation run by the oracle."""
    import torch
    p, lab = case(seed=62, dtype=np.float64, noise=0.0, outlier=0.0, sigma=0.05)
    rounds, d_it, p_it = 3, 4, 3
    seg = O.depth_segments(p, lab)
    poses_o = p.poses_init.copy()
    eta_o = np.zeros(seg["M"])
    for _ in range(rounds):
        eta_o, _ = O.depth_refine(p, poses_o, eta_o, d_it, seg)
        e = seg["eff"]
        d = np.exp(seg["logd"] + np.where(e >= 0, eta_o[np.maximum(e, 0)], 0.0))
        pts = p.points.copy()
        pts[:, :3] = np.where((e >= 0)[:, None], d[:, None] * seg["psi"], p.points[:, :3])
        poses_o, _ = O.gn_solve(dataclasses.replace(p, points=pts), poses_o, p_it)
    with C.Graph(p, mode=C.PLAIN_FP64, copy_inputs=True,
                 points=torch.from_numpy(p.points).pin_memory(),
                 match_idx=torch.from_numpy(p.match_idx).pin_memory()) as g:
        poses, eta = C.terminal_refine(g, p.poses_init, lab, rounds=rounds, depth_iters=d_it, pose_iters=p_it)
    assert np.abs(eta - eta_o).max() <= 1e-9
    assert max(O.pose_errors(poses, poses_o).values()) <= 1e-9
