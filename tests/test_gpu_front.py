"""Front-end kernels on the GPU (como3r_project_match, como3r_fuse; Sec. III-A) against the
oracle: the projective matches and their FP32 distances bit for bit (integer decisions
taken in the same precision on both sides), fusion within FP32 / FP64 rounding."""
import numpy as np
import pytest

from oracle import como3r_oracle as O

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


def pair_from(p, e=0, poses=None):
    """Frame = edge e's gathered keyframe j, queries = keyframe i's points in j's camera."""
    arrs = O.problem_arrays(p)
    i, j = int(p.edge_i[e]), int(p.edge_j[e])
    poses = p.poses_init if poses is None else poses
    Pi = p.points[arrs["pix_off"][i]:arrs["pix_off"][i + 1]]
    Pj = p.points[arrs["pix_off"][j]:arrs["pix_off"][j + 1]]
    Tji = O.sim3_inverse(O.pose_to_matrix(poses[j])) @ O.pose_to_matrix(poses[i])
    q = np.concatenate([O.transform(Tji, Pi[:, :3].astype(np.float64)), Pi[:, 3:4].astype(np.float64)], axis=1)
    return Pj, q.astype(p.points.dtype)


def run_both(C, frame, H, W, query, dtype, init, steps=64, angle=0.01):
    import torch
    m, d = C.project_match(torch.from_numpy(np.ascontiguousarray(frame)).cuda(), H, W,
                           torch.from_numpy(np.ascontiguousarray(query)).cuda(), dtype=dtype,
                           init=torch.from_numpy(init.astype(np.int32)).cuda(), max_steps=steps, max_angle=angle,
                           with_dist=True)
    mo, do = O.project_match(frame, H, W, query, init, max_steps=steps, max_angle=angle)
    return m.cpu().numpy(), d.cpu().numpy(), mo, do


@pytest.mark.parametrize("dtype", [np.float16, np.float32, np.float64])
def test_project_match_bitexact(C, dtype):
    from synth import make_cloud_problem
    p = make_cloud_problem(81, [dict(agents=1, n_kf=4, H=48, W=64, period=30, shift=6, n_inter=0, noise=0.01,
                                     outlier=0.1)], dtype=dtype)
    code = {np.float16: C.F16, np.float32: C.F32, np.float64: C.F64}[dtype]
    frame, q = pair_from(p, 0)
    q[7, 0] = np.nan          # a non-finite query
    frame[100, :3] = 0.0      # a frame pixel with no ray
    rng = np.random.default_rng(1)
    for init in (np.arange(48 * 64), rng.integers(0, 48 * 64, size=48 * 64)):
        # pixels are ~2.8 deg apart at this size: half a pixel is ~0.025 rad
        m, d, mo, do = run_both(C, frame, 48, 64, q, code, init, angle=0.05)
        np.testing.assert_array_equal(m, mo)
        np.testing.assert_array_equal(d, do)
    assert m[7] == -1 and (m >= 0).mean() > 0.5 and not np.any(m == 100)


def test_project_match_full_size(C):
    """A 512x384 pair with dense predicted pointmaps (FP32; queries through the perturbed
    initial poses): all 196,608 queries bit for bit."""
    from synth import make_cloud_problem
    p = make_cloud_problem(82, [dict(agents=1, n_kf=3, H=384, W=512, period=40, shift=51, n_inter=0, noise=0.01,
                                     outlier=0.0)], dtype=np.float32)
    frame, q = pair_from(p, 0)
    m, d, mo, do = run_both(C, frame, 384, 512, q, C.F32, np.arange(384 * 512))
    np.testing.assert_array_equal(m, mo)
    np.testing.assert_array_equal(d, do)
    assert (m >= 0).mean() > 0.3


def test_fuse_matches_oracle(C):
    import torch
    rng = np.random.default_rng(2)
    n = 100003
    X = rng.normal(size=(n, 3)) + np.array([0, 0, 5.0])
    canon = np.concatenate([X, rng.uniform(1, 5, (n, 1))], 1)
    pred = np.concatenate([rng.normal(size=(n, 3)), rng.uniform(0.5, 3, (n, 1))], 1)
    T = O.exp_sim3(np.concatenate([rng.normal(size=3), rng.normal(size=3) * 0.4, [0.2]]))
    want = O.fuse(canon, pred, T)
    for dt, code, tol in ((np.float32, C.F32, 2e-6), (np.float64, C.F64, 1e-13)):
        c = torch.from_numpy(canon.astype(dt)).cuda()
        C.fuse(c, torch.from_numpy(pred.astype(dt)).cuda(), O.matrix_to_pose(T), dtype=code)
        got = c.cpu().numpy().astype(np.float64)
        ref = O.fuse(canon.astype(dt).astype(np.float64), pred.astype(dt).astype(np.float64), T)
        assert np.abs(got - ref).max() / np.abs(ref).max() <= tol
    with pytest.raises(C.Como3rError):
        C.fuse(torch.zeros((4, 4), dtype=torch.float16, device="cuda"),
               torch.zeros((4, 4), dtype=torch.float16, device="cuda"), O.matrix_to_pose(T), dtype=C.F16)


def test_fuse_packed_matches_single_calls(C):
    """Many keyframes in one call (each with its own T_kf, uneven sizes, an empty one, more
    keyframes than one launch takes): bit for bit the per-keyframe como3r_fuse, and the
    oracle's fusion within FP32 / FP64 rounding."""
    import torch
    rng = np.random.default_rng(3)
    for n in (5, 130):
        sizes = rng.integers(0, 3000, size=n)
        sizes[1] = 0
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        P = int(off[-1])
        X = rng.normal(size=(P, 3)) + np.array([0, 0, 5.0])
        canon = np.concatenate([X, rng.uniform(1, 5, (P, 1))], 1)
        pred = np.concatenate([rng.normal(size=(P, 3)), rng.uniform(0.5, 3, (P, 1))], 1)
        Ts = [O.exp_sim3(np.concatenate([rng.normal(size=3), rng.normal(size=3) * 0.4, [0.1 * rng.normal()]]))
              for _ in range(n)]
        poses = np.stack([O.matrix_to_pose(T) for T in Ts])
        for dt, code, tol in ((np.float32, C.F32, 2e-6), (np.float64, C.F64, 1e-13)):
            c0 = torch.from_numpy(canon.astype(dt)).cuda()
            pr = torch.from_numpy(pred.astype(dt)).cuda()
            packed = c0.clone()
            C.fuse_packed(packed, pr, off, poses, dtype=code)
            single = c0.clone()
            for q in range(n):
                a, b = int(off[q]), int(off[q + 1])
                if b > a:
                    C.fuse(single[a:b], pr[a:b], poses[q], dtype=code)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(packed.cpu().numpy(), single.cpu().numpy())
            got = packed.cpu().numpy().astype(np.float64)
            for q in (0, 2, n - 1):
                a, b = int(off[q]), int(off[q + 1])
                if b == a:
                    continue
                ref = O.fuse(canon[a:b].astype(dt).astype(np.float64), pred[a:b].astype(dt).astype(np.float64),
                             Ts[q])
                assert np.abs(got[a:b] - ref).max() / np.abs(ref).max() <= tol
    z = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(C.Como3rError):
        C.fuse_packed(z, z, [0, 2, 1], np.tile(O.matrix_to_pose(np.eye(4)), (2, 1)))  # decreasing offsets
    bad = np.tile(O.matrix_to_pose(np.eye(4)), (1, 1))
    bad[0, 3:7] = 0.0
    with pytest.raises(C.Como3rError):
        C.fuse_packed(z, z, [0, 4], bad)  # zero quaternion
    with pytest.raises(C.Como3rError):
        C.fuse_packed(torch.zeros((4, 4), dtype=torch.float16, device="cuda"),
                      torch.zeros((4, 4), dtype=torch.float16, device="cuda"), [0, 4],
                      np.tile(O.matrix_to_pose(np.eye(4)), (1, 1)), dtype=C.F16)
