"""GPU parity of the adjoint (como3r_vjp): gradient of the refined cost with respect to
per-pixel log-range and confidence, against the FP64 oracle's complex-step derivative.

The oracle differentiates its own step-by-step Gauss-Newton iterations (IRLS weights,
damped Cholesky, matrix-exponential retraction) by the complex step, so it shares no
derivation with the hand-written reverse pass.  Comparisons: the directional derivative
along dense random directions (all pixels at once) and single-pixel derivatives.
Tolerances: the all-FP64 form differs from the oracle only by its FP32 output rounding
(2^-24 relative per element), so 1e-6 relative; the mixed form evaluates every match in
FP32 (hardware reciprocal and square-root approximations, ~2 ulp) and accumulates pixel
gradients with FP32 atomics, which agree with the oracle to ~1e-6 relative on these
problems, so 1e-5 relative.
"""
import dataclasses

import numpy as np
import pytest

from oracle import como3r_oracle as O
from synth import make_problem, make_workload

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-5}  # by mode: PLAIN_FP64, MIXED


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30488_b300 import build
    build.build()
    from paper_2605_30488_b300 import como3r
    return como3r


@pytest.fixture(scope="module")
def small():
    """2 agents x 3 keyframes at 32x24 (FP64 storage), 5 edges, perturbed initial poses."""
    return make_problem(3, agents=2, n_kf=3, H=24, W=32, f=25.0, n_inter=1, iters=3)


def gpu_grads(C, prob, mode, iters, vjp_mode, upstream=1.0):
    import torch
    g = C.Graph(prob, mode=mode)
    poses = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
    out = torch.empty_like(poses)
    st, gl, gc, loss = g.vjp(poses, iters, vjp_mode, upstream=upstream, poses_out=out)
    res = gl.double().cpu().numpy(), gc.double().cpu().numpy(), loss, out.cpu().numpy(), g.last_launch_count()
    g.close()
    return res


def touched_pixels(prob):
    pix = []
    for e in range(prob.num_edges):
        idx = prob.match_idx[prob.idx_offset()[e]:prob.idx_offset()[e + 1]]
        m = np.nonzero(idx >= 0)[0]
        pix.append(prob.pix_offset()[prob.edge_i[e]] + m)
        pix.append(prob.pix_offset()[prob.edge_j[e]] + idx[m])
    return np.unique(np.concatenate(pix))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("vjp_mode,iters", [(1, 2), (0, 1), (0, 3)])
def test_vjp_directional_matches_complex_step(C, small, mode, vjp_mode, iters):
    gl, gc, loss, _, _ = gpu_grads(C, small, mode, iters, vjp_mode)
    rng = np.random.default_rng(100 + iters)
    envelope = vjp_mode == C.VJP_ENVELOPE
    for _ in range(2):
        vl, vc = rng.normal(size=gl.size), rng.normal(size=gl.size)
        ref = O.refined_cost_derivative(small, small.poses_init, iters, vl, vc, envelope=envelope)
        got = float(gl @ vl + gc @ vc)
        # error bound from per-element relative errors (the sum may cancel)
        mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
        assert abs(got - ref) <= TOL[mode] * mag, (got, ref, mag)
    # the loss is the refined cost itself
    L = float(O.refined_cost(small, small.poses_init, iters).real)
    assert abs(loss.sum() - L) <= (1e-9 if mode == 0 else 1e-5) * abs(L)


@pytest.mark.parametrize("mode", [0, 1])
def test_vjp_single_pixels_match_complex_step(C, small, mode):
    iters = 2
    gl, gc, _, _, _ = gpu_grads(C, small, mode, iters, C.VJP_UNROLLED)
    pix = touched_pixels(small)
    scale_l, scale_c = np.abs(gl).max(), np.abs(gc).max()
    # a pixel's derivative can be a small difference of large per-match terms, and the FP32
    # evaluation of the mixed form rounds at the scale of the problem's gradients: its
    # per-pixel errors are bounded relative to the largest gradient (FP64: to 0.1 % of it)
    floor = 1e-3 if mode == 0 else 1.0
    for p in pix[np.linspace(0, len(pix) - 1, 6).astype(int)]:
        v = np.zeros(gl.size)
        v[p] = 1.0
        rl = O.refined_cost_derivative(small, small.poses_init, iters, v, None)
        rc = O.refined_cost_derivative(small, small.poses_init, iters, None, v)
        assert abs(gl[p] - rl) <= TOL[mode] * max(abs(rl), floor * scale_l), (p, gl[p], rl)
        assert abs(gc[p] - rc) <= TOL[mode] * max(abs(rc), floor * scale_c), (p, gc[p], rc)


def test_vjp_untouched_pixels_have_zero_gradient(C, small):
    gl, gc, _, _, _ = gpu_grads(C, small, 0, 2, C.VJP_UNROLLED)
    untouched = np.setdiff1d(np.arange(gl.size), touched_pixels(small))
    assert np.all(gl[untouched] == 0.0) and np.all(gc[untouched] == 0.0)


def test_vjp_is_linear_in_upstream_and_returns_final_poses(C, small, monkeypatch):
    # two graphs: the residual kernel's autotuned schedule pinned, so that they round alike
    monkeypatch.setenv("COMO3R_K1_CFG", "1")
    monkeypatch.setenv("COMO3R_K1_CHUNK", "1024")
    monkeypatch.setenv("COMO3R_K1_WEIGHTS", "1,1")
    gl1, gc1, loss1, poses1, launches = gpu_grads(C, small, 0, 2, C.VJP_UNROLLED, upstream=1.0)
    gl3, gc3, loss3, poses3, _ = gpu_grads(C, small, 0, 2, C.VJP_UNROLLED, upstream=-3.0)
    np.testing.assert_allclose(gl3, -3.0 * gl1, rtol=1e-6, atol=1e-12 * np.abs(gl1).max())
    np.testing.assert_allclose(gc3, -3.0 * gc1, rtol=1e-6, atol=1e-12 * np.abs(gc1).max())
    np.testing.assert_array_equal(poses1, poses3)
    ref, _ = O.gn_solve(small, small.poses_init, 2)
    err = O.pose_errors(poses1, ref)
    assert max(err.values()) <= 1e-9
    assert launches > 0


def test_vjp_envelope_at_zero_iterations_equals_unrolled(C, small):
    # (pixel gradients are atomically accumulated, so equal up to summation order)
    a = gpu_grads(C, small, 0, 0, C.VJP_UNROLLED)
    b = gpu_grads(C, small, 0, 0, C.VJP_ENVELOPE)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-6, atol=1e-12 * np.abs(a[0]).max())
    np.testing.assert_allclose(a[1], b[1], rtol=1e-6, atol=1e-12 * np.abs(a[1]).max())


def test_autograd_function_round_trip(C, small):
    """Como3rCost: forward from (log-range, confidence) reproduces the oracle's refined
    cost, backward equals como3r_vjp, and the packing kernels invert each other."""
    import torch
    g = C.Graph(small, mode=C.PLAIN_FP64)
    rays, ld, cf = C.rays_from_points(g.points)
    # round trip of the packed points (FP32 parameters, FP64 storage)
    back = torch.empty_like(g.points)
    C.points_from_logdepth(rays, ld, cf, back)
    # (FP32 log-range and unit ray: a few FP32 roundings of the range)
    np.testing.assert_allclose(back.cpu().numpy(), small.points, rtol=1e-6, atol=1e-12)
    ld = ld.clone().requires_grad_(True)
    cf = cf.clone().requires_grad_(True)
    poses = torch.tensor(small.poses_init, dtype=torch.float64, device="cuda")
    L = C.refined_cost(ld, cf, g, rays, poses, 2)
    (2.0 * L).backward()
    # the graph now holds the FP32-parameterised points; the oracle sees the same values
    stored = g.points.cpu().numpy()
    ref = O.refined_cost(dataclasses.replace(small, points=stored), small.poses_init, 2)
    assert abs(float(L.detach()) - float(ref.real)) <= 1e-9 * abs(float(ref.real))
    _, gl, gc, _ = g.vjp(poses, 2, C.VJP_UNROLLED, upstream=2.0)
    for a, b in ((ld.grad, gl), (cf.grad, gc)):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-12 * np.abs(b).max())
    g.close()


def test_vjp_rejects_bad_arguments(C, small):
    import torch
    g = C.Graph(small, mode=C.PLAIN_FP64)
    poses = torch.tensor(small.poses_init, dtype=torch.float64, device="cuda")
    with pytest.raises(C.Como3rError):
        g.vjp(poses, -1)
    with pytest.raises(C.Como3rError):
        g.vjp(poses, 1, mode=7)
    host = torch.zeros(len(small.points), dtype=torch.float32)
    with pytest.raises(C.Como3rError):
        g.vjp(poses, 1, grad_logdepth=host, grad_conf=host)
    g.close()


@pytest.fixture(scope="module")
def mid():
    """2 agents x 8 keyframes at 160x120, FP32 storage: several work items per edge with a
    ragged last one."""
    return make_problem(5, agents=2, n_kf=8, H=120, W=160, f=125.0, noise=0.01, conf="lognormal",
                        outlier=0.15, skip_max=4, n_inter=4, exact=False, dtype=np.float32, name="mid")


@pytest.mark.parametrize("mode", [0, 1])
def test_vjp_multi_item_edges_match_complex_step(C, mid, mode):
    gl, gc, _, _, _ = gpu_grads(C, mid, mode, 2, C.VJP_UNROLLED)
    rng = np.random.default_rng(7)
    vl, vc = rng.normal(size=gl.size), rng.normal(size=gl.size)
    ref = O.refined_cost_derivative(mid, mid.poses_init, 2, vl, vc)
    mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
    assert abs(float(gl @ vl + gc @ vc) - ref) <= TOL[mode] * mag


@pytest.fixture(scope="module")
def adjoint_workload():
    """The adjoint workload: 4 agents x 30 keyframes, 512x384 FP32 pointmaps, 8 iterations."""
    return make_workload("four_agent_30kf_512x384", seed=0)


def test_vjp_full_size_envelope_matches_finite_difference(C, adjoint_workload):
    """At T^K (K = 8) the partial derivative of E along dense random directions equals a
    central difference of the FP64 GPU cost evaluated at fixed poses (step 1e-5; the cost is
    ~1e9, so single-pixel differences would sit below its FP64 rounding noise)."""
    import torch
    prob = dataclasses.replace(adjoint_workload, points=adjoint_workload.points.astype(np.float64))
    g = C.Graph(prob, mode=C.PLAIN_FP64)
    poses = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
    TK = torch.empty_like(poses)
    _, gl, gc, _ = g.vjp(poses, prob.iters, C.VJP_ENVELOPE, poses_out=TK)
    gl, gc = gl.double().cpu().numpy(), gc.double().cpu().numpy()
    base = g.points.clone()
    rng = np.random.default_rng(3)
    for which in ("log", "conf"):
        v = rng.normal(size=len(prob.points))
        vt = torch.tensor(v, device="cuda")

        def cost(t):
            g.points.copy_(base)
            if which == "log":
                g.points[:, :3] = base[:, :3] * torch.exp(t * vt)[:, None]
            else:
                g.points[:, 3] = base[:, 3] + t * vt
            return g.linearize(TK)[1].sum()

        h = 1e-5
        fd = (cost(h) - cost(-h)) / (2 * h)
        got = float((gl if which == "log" else gc) @ v)
        assert abs(got - fd) <= 1e-4 * abs(fd), (which, got, fd)
    g.points.copy_(base)
    g.close()


def test_vjp_full_size_mixed_matches_fp64(C, adjoint_workload):
    """Mixed against all-FP64 gradients on the same FP32 pointmaps: the envelope after 8
    iterations, and the unrolled derivative through one iteration (through 8 non-converged
    IRLS iterations the unrolled derivative is too ill-conditioned for FP32 trajectories)."""
    rng = np.random.default_rng(4)
    v = rng.normal(size=len(adjoint_workload.points))
    for vjp_mode, iters, tol in ((C.VJP_ENVELOPE, adjoint_workload.iters, 1e-4), (C.VJP_UNROLLED, 1, 1e-5)):
        a = gpu_grads(C, adjoint_workload, C.MIXED, iters, vjp_mode)
        b = gpu_grads(C, adjoint_workload, C.PLAIN_FP64, iters, vjp_mode)
        for k in (0, 1):
            mag = float(np.abs(b[k] * v).sum())
            assert abs(float(a[k] @ v - b[k] @ v)) <= tol * mag, (vjp_mode, iters, k)


@pytest.mark.parametrize("setting", [("COMO3R_SOLVE_CLUSTER", "4"), ("COMO3R_SOLVE_GRID", "1"),
                                     ("COMO3R_SUBSTITUTE_SMEM", "1"), ("COMO3R_SUBSTITUTE_SMEM", "0")])
def test_vjp_with_each_kept_factor(C, mid, monkeypatch, setting):
    """The adjoint systems solved with the factor kept by the multi-SM (cluster) and the
    grid-wide factorisations, and by the substitution with the factor read through the L2
    (its plan and vector in shared memory) or with everything in global memory (the default
    stages the factor into shared memory)."""
    monkeypatch.setenv(*setting)
    gl, gc, _, _, _ = gpu_grads(C, mid, 0, 2, C.VJP_UNROLLED)
    rng = np.random.default_rng(7)
    vl, vc = rng.normal(size=gl.size), rng.normal(size=gl.size)
    ref = O.refined_cost_derivative(mid, mid.poses_init, 2, vl, vc)
    mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
    assert abs(float(gl @ vl + gc @ vc) - ref) <= TOL[0] * mag


@pytest.mark.parametrize("groups", ["0", "2"])
def test_vjp_batch_of_graphs_matches_complex_step(C, groups, monkeypatch):
    """Three graphs of different sizes in one handle: every graph's adjoint systems are
    solved with its own kept factor (kept by one CTA per graph, or by the CTA-group solve
    with two graphs on clusters)."""
    monkeypatch.setenv("COMO3R_SOLVE_GROUPS", groups)
    specs = [dict(n_kf=3), dict(n_kf=4), dict(n_kf=2)]
    prob = make_problem(11, H=24, W=32, f=25.0, n_inter=1, iters=3, graph_specs=specs)
    gl, gc, _, _, _ = gpu_grads(C, prob, 0, 3, C.VJP_UNROLLED)
    rng = np.random.default_rng(3)
    vl, vc = rng.normal(size=gl.size), rng.normal(size=gl.size)
    ref = O.refined_cost_derivative(prob, prob.poses_init, 3, vl, vc)
    mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
    assert abs(float(gl @ vl + gc @ vc) - ref) <= TOL[0] * mag
