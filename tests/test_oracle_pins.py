"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: hand-derived values
of Eq. (jacobian) / Eq. (residual), central finite differences, Lie-group identities,
the Sim(3) gauge symmetry of Eq. (global), noise-free recovery, closed-form Umeyama
(Eq. umeyama) against brute force, the escalation schedule of Sec. III-D, and the
cross-agent gate and gauge synchronisation of Sec. III-B/III-C against constructed cases
(a known extra similarity, the endpoint fallback, counted supports, equivariance).
"""
import math
import os

import numpy as np
import pytest

from oracle import como3r_oracle as O
from synth import make_problem, make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_sim3(rng, rot=1.0, trans=2.0, logs=0.5):
    tau = np.concatenate([rng.normal(size=3) * trans, rng.normal(size=3) * rot, [rng.normal() * logs]])
    return O.exp_sim3(tau)


# ------------------------------------------------------------------ golden fixtures
def load_jacobian_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "jacobian_rel.txt")) if l.strip() and not l.startswith("#")]
    cases = []
    for k in range(0, len(rows), 5):
        x = np.array([float(v) for v in rows[k]])
        J = np.array([[float(v) for v in r] for r in rows[k + 1:k + 5]])
        cases.append((x, J))
    return cases


def test_jacobian_matches_hand_derivation():
    """Eq. (jacobian): the 4x7 block written out by hand for two points."""
    for x, J in load_jacobian_golden():
        got = O.jacobian_rel(x[None, :])[0]
        np.testing.assert_allclose(got, J, rtol=0, atol=1e-15)


def test_residual_matches_hand_values():
    """Eq. (residual) on hand-picked poses and points."""
    for line in open(os.path.join(GOLDEN, "residual.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        pose, xj, xi, e = [np.array([float(v) for v in part.split()]) for part in line.split("|")]
        s, q, t = pose[0], pose[1:5], pose[5:8]
        T = O.pose_to_matrix(np.concatenate([t, q, [s]]))
        got, _ = O.residual(T, xi[None, :], xj[None, :])
        np.testing.assert_allclose(got[0], e, rtol=0, atol=1e-13)


# ------------------------------------------------------------------ Lie group identities
def test_exp_special_cases():
    rng = np.random.default_rng(1)
    v = rng.normal(size=3)
    np.testing.assert_allclose(O.exp_sim3(np.r_[v, 0, 0, 0, 0]), np.block([[np.eye(3), v[:, None]], [np.zeros((1, 3)), 1]]), atol=1e-15)
    z = 0.37
    np.testing.assert_allclose(O.exp_sim3(np.r_[0, 0, 0, 0, 0, 0, z])[:3, :3], math.exp(z) * np.eye(3), rtol=1e-15)
    w = rng.normal(size=3)
    th = np.linalg.norm(w)
    K = O.skew(w / th)
    Rrod = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K  # Rodrigues
    np.testing.assert_allclose(O.exp_sim3(np.r_[0, 0, 0, w, 0])[:3, :3], Rrod, atol=1e-14)
    tau = rng.normal(size=7)
    np.testing.assert_allclose(O.exp_sim3(tau) @ O.exp_sim3(-tau), np.eye(4), atol=1e-13)
    h = 1e-6
    dE = (O.exp_sim3(tau * (1 + h)) - O.exp_sim3(tau * (1 - h))) / (2 * h)
    np.testing.assert_allclose(dE, O.hat(tau) @ O.exp_sim3(tau), rtol=1e-6, atol=1e-8)


def test_adjoint_conjugation():
    """Ad_T tau satisfies Exp(Ad_T tau) = T Exp(tau) T^{-1}."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        T = rand_sim3(rng)
        tau = rng.normal(size=7) * 0.3
        lhs = O.exp_sim3(O.adjoint(T) @ tau)
        rhs = T @ O.exp_sim3(tau) @ np.linalg.inv(T)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-11)


def test_edge_chain_rule_signs():
    """T_ij under left perturbations of T_i and T_j moves by -Ad / +Ad of T_i^{-1} (Sec. III-D)."""
    rng = np.random.default_rng(3)
    Ti, Tj = rand_sim3(rng), rand_sim3(rng)
    Tij = np.linalg.inv(Ti) @ Tj
    Ad = O.adjoint(np.linalg.inv(Ti))
    h = 1e-6
    for k in range(7):
        d = np.zeros(7); d[k] = h
        for which, sign in (("i", -1.0), ("j", 1.0)):
            def rel(dd):
                A = O.exp_sim3(dd) @ Ti if which == "i" else Ti
                B = O.exp_sim3(dd) @ Tj if which == "j" else Tj
                return O.log_sim3(np.linalg.inv(A) @ B @ np.linalg.inv(Tij))
            fd = (rel(d) - rel(-d)) / (2 * h)
            np.testing.assert_allclose(fd, sign * Ad[:, k], rtol=1e-5, atol=1e-6)


# ------------------------------------------------------------------ Jacobians by FD
def test_edge_jacobians_central_fd():
    """J_i = -J Ad, J_j = J Ad agree with central FD of e to 1e-6 relative (Eq. jacobian)."""
    rng = np.random.default_rng(4)
    Ti, Tj = rand_sim3(rng, trans=1.0), rand_sim3(rng, trans=1.0)
    Xj = rng.normal(size=(50, 3)) + np.array([0, 0, 5.0])
    Xi = O.transform(np.linalg.inv(Ti) @ Tj, Xj) * (1 + 0.01 * rng.normal(size=(50, 1)))
    e0, x = O.residual(np.linalg.inv(Ti) @ Tj, Xi, Xj)
    J = O.jacobian_rel(x)
    Ad = O.adjoint(np.linalg.inv(Ti))
    Ji, Jj = -J @ Ad, J @ Ad
    h = 1e-6
    for k in range(7):
        d = np.zeros(7); d[k] = h
        for Jan, which in ((Ji, "i"), (Jj, "j")):
            def ev(dd):
                A = O.exp_sim3(dd) @ Ti if which == "i" else Ti
                B = O.exp_sim3(dd) @ Tj if which == "j" else Tj
                return O.residual(np.linalg.inv(A) @ B, Xi, Xj)[0]
            fd = (ev(d) - ev(-d)) / (2 * h)
            scale = np.abs(Jan[:, :, k]).max()
            assert np.abs(fd - Jan[:, :, k]).max() <= 1e-6 * scale


# ------------------------------------------------------------------ Huber
def test_huber_derivative_and_continuity():
    k = 1.345
    r = np.linspace(-5, 5, 1001)
    h = 1e-6
    fd = (O.huber_rho(r + h, k) - O.huber_rho(r - h, k)) / (2 * h)
    np.testing.assert_allclose(fd, O.huber_weight(r, k) * r, atol=1e-8)
    for s in (1, -1):  # C1 at the breakpoint
        a, b = s * (k - 1e-9), s * (k + 1e-9)
        assert abs(O.huber_rho(np.array([a]), k) - O.huber_rho(np.array([b]), k))[0] < 1e-8
        assert abs(O.huber_weight(np.array([a]), k)[0] - O.huber_weight(np.array([b]), k)[0]) < 1e-8
    assert O.huber_weight(np.array([0.0]), k)[0] == 1.0


# ------------------------------------------------------------------ system-level pins
@pytest.fixture(scope="module")
def tiny():
    return make_workload("two_agent_6kf_64x48", seed=0)


@pytest.fixture(scope="module")
def tiny_exact():
    return make_problem(3, noise=0.0, outlier=0.0, exact=True, name="noise-free")


def perturb_one(poses, k, tau):
    out = poses.copy()
    out[k] = O.matrix_to_pose(O.exp_sim3(tau) @ O.pose_to_matrix(poses[k]))
    return out


def test_gradient_is_derivative_of_cost(tiny):
    """g = sum J^T W e is dE/dtau for left perturbations (pins sign, W and whitening)."""
    poses = tiny.poses_init
    H, g, E, _ = O.build_system(tiny, poses, 0)
    rng = np.random.default_rng(5)
    h = 1e-6
    for k in rng.choice(tiny.num_kf, size=4, replace=False):
        for c in range(7):
            d = np.zeros(7); d[c] = h
            fd = (O.total_cost(tiny, perturb_one(poses, k, d))[0] - O.total_cost(tiny, perturb_one(poses, k, -d))[0]) / (2 * h)
            assert abs(fd - g[7 * k + c]) <= 1e-5 * max(1.0, abs(g).max() * 1e-2)


def test_hessian_exact_at_zero_residual(tiny_exact):
    """With all residuals zero the GN matrix is the exact Hessian: H = d g / d tau."""
    poses = tiny_exact.poses_gt
    H, g, E, _ = O.build_system(tiny_exact, poses, 0)
    assert E < 1e-18
    h = 1e-6
    for k in (1, 7):
        for c in range(7):
            d = np.zeros(7); d[c] = h
            gp = O.build_system(tiny_exact, perturb_one(poses, k, d), 0)[1]
            gm = O.build_system(tiny_exact, perturb_one(poses, k, -d), 0)[1]
            col = (gp - gm) / (2 * h)
            np.testing.assert_allclose(col, H[:, 7 * k + c], rtol=0, atol=2e-5 * np.abs(H).max())


def test_gauge_invariance(tiny):
    """E(G T) = E(T); H annihilates a common left perturbation; sum_i g_i = 0 (Eq. global)."""
    poses = tiny.poses_init
    H, g, E, _ = O.build_system(tiny, poses, 0)
    rng = np.random.default_rng(6)
    G = rand_sim3(rng)
    moved = np.array([O.matrix_to_pose(G @ O.pose_to_matrix(p)) for p in poses])
    E2 = O.total_cost(tiny, moved)[0]
    assert abs(E2 - E) <= 1e-9 * E
    delta = rng.normal(size=7)
    common = np.tile(delta, tiny.num_kf)
    assert np.abs(H @ common).max() <= 1e-9 * np.abs(H).max() * np.abs(delta).max()
    np.testing.assert_allclose(g.reshape(-1, 7).sum(0), 0.0, atol=1e-9 * np.abs(g).max())


def test_edge_block_structure(tiny):
    """Each edge adds H_ii = H_jj = -H_ij and g_i = -g_j (two diagonal + one off-diagonal block)."""
    _, _, _, recs = O.build_system(tiny, tiny.poses_init, 0)
    for r in recs:
        s = np.abs(r["H_ii"]).max()
        np.testing.assert_allclose(r["H_ii"], r["H_jj"], atol=1e-10 * s)
        np.testing.assert_allclose(r["H_ij"], -r["H_ii"], atol=1e-10 * s)
        np.testing.assert_allclose(r["g_i"], -r["g_j"], atol=1e-10 * max(1.0, np.abs(r["g_i"]).max()))
        Ad = r["Ad"]
        np.testing.assert_allclose(r["H_jj"], Ad.T @ r["H_rel"] @ Ad, atol=1e-9 * s)


def test_confidence_and_sigma_scaling(tiny_exact):
    """Quadratic regime: E scales with q (c -> 4c gives x4) and with 1/sigma^2 per block."""
    poses = tiny_exact.poses_init.copy()
    # tiny perturbation keeps every |r| below kappa
    poses = np.array([O.matrix_to_pose(O.exp_sim3(np.r_[1e-6, 0, 0, 0, 1e-7, 0, 1e-7]) @ O.pose_to_matrix(p)) if k else p
                      for k, p in enumerate(tiny_exact.poses_gt)])
    E = O.total_cost(tiny_exact, poses)[0]
    p4 = make_problem(3, noise=0.0, outlier=0.0, exact=True)
    p4.points = p4.points.copy(); p4.points[:, 3] *= 4.0
    E4 = O.total_cost(p4, poses)[0]
    assert abs(E4 / E - 4.0) < 1e-9
    pd = make_problem(3, noise=0.0, outlier=0.0, exact=True)
    pd.sigma_dist = 1e9  # range block off: only the ray block remains
    pr = make_problem(3, noise=0.0, outlier=0.0, exact=True)
    pr.sigma_ray = 1e9
    Er, Ed = O.total_cost(pd, poses)[0], O.total_cost(pr, poses)[0]
    assert abs((Er + Ed) / E - 1.0) < 1e-9
    pd.sigma_ray = tiny_exact.sigma_ray / 2
    assert abs(O.total_cost(pd, poses)[0] / Er - 4.0) < 1e-9


def test_noise_free_recovery(tiny_exact):
    """Exact correspondences, no noise: GN returns to the ground truth (anchor fixes the gauge)."""
    poses, trace = O.gn_solve(tiny_exact, tiny_exact.poses_init, 10)
    err = O.pose_errors(poses, tiny_exact.poses_gt)
    assert err["rot"] < 1e-10 and err["trans"] < 1e-10 and err["scale"] < 1e-10, err
    assert trace[-1, 0] < 1e-16 and trace[0, 0] > 1.0


def test_two_view_equals_umeyama():
    """One edge, noise-free: the GN pose of j equals Umeyama on the matched points."""
    p = make_problem(11, agents=1, n_kf=2, noise=0.0, outlier=0.0, n_inter=0, exact=True)
    poses, _ = O.gn_solve(p, p.poses_init, 10)
    arrs = O.problem_arrays(p)
    i, j, m, n, Pi, Pj = O.edge_matches(p, arrs, 0)
    x = O.transform(O.pose_to_matrix(p.poses_gt[0]), Pi[:, :3])
    s, R, t = O.umeyama(x, Pj[:, :3])
    T = np.eye(4); T[:3, :3] = s * R; T[:3, 3] = t
    np.testing.assert_allclose(O.pose_to_matrix(poses[1]), T, atol=1e-10)
    np.testing.assert_allclose(T, O.pose_to_matrix(p.poses_gt[1]), atol=1e-10)


# ------------------------------------------------------------------ Umeyama vs brute force
def _brute_force_alignment(x, y):
    """Best (s, R, t) by a rotation grid (<= 1 deg) plus local GN refinement; s, t closed form per R."""
    xc, yc = x - x.mean(0), y - y.mean(0)

    def cost_R(R):
        Ry = yc @ R.T
        s = max((xc * Ry).sum() / (yc * yc).sum(), 0.0)
        return ((xc - s * Ry) ** 2).sum(), s

    best = (np.inf, None)
    axes = []
    for a in np.linspace(0, math.pi, 13):
        for b in np.linspace(0, 2 * math.pi, 25, endpoint=False):
            axes.append([math.sin(a) * math.cos(b), math.sin(a) * math.sin(b), math.cos(a)])
    for ax in axes:
        for ang in np.linspace(0, math.pi, 19):
            R = O.exp_sim3(np.r_[0, 0, 0, np.array(ax) * ang, 0])[:3, :3]
            c, _ = cost_R(R)
            if c < best[0]:
                best = (c, R)
    R = best[1]
    for _ in range(200):  # refine with small rotations (finite-difference Newton on so(3))
        c0, _ = cost_R(R)
        h = 1e-5
        g = np.zeros(3); Hm = np.zeros((3, 3))
        for a in range(3):
            ea = np.zeros(3); ea[a] = h
            cp, cm = cost_R(O.exp_sim3(np.r_[0, 0, 0, ea, 0])[:3, :3] @ R)[0], cost_R(O.exp_sim3(np.r_[0, 0, 0, -ea, 0])[:3, :3] @ R)[0]
            g[a] = (cp - cm) / (2 * h)
            Hm[a, a] = (cp - 2 * c0 + cm) / h ** 2
            for b in range(a):
                eb = np.zeros(3); eb[b] = h
                cpp = cost_R(O.exp_sim3(np.r_[0, 0, 0, ea + eb, 0])[:3, :3] @ R)[0]
                cmm = cost_R(O.exp_sim3(np.r_[0, 0, 0, -ea - eb, 0])[:3, :3] @ R)[0]
                cpm = cost_R(O.exp_sim3(np.r_[0, 0, 0, ea - eb, 0])[:3, :3] @ R)[0]
                cmp_ = cost_R(O.exp_sim3(np.r_[0, 0, 0, -ea + eb, 0])[:3, :3] @ R)[0]
                Hm[a, b] = Hm[b, a] = (cpp - cpm - cmp_ + cmm) / (4 * h * h)
        step = -np.linalg.solve(Hm + 1e-12 * np.eye(3), g)
        if np.linalg.norm(step) > 0.05:
            step *= 0.05 / np.linalg.norm(step)
        Rn = O.exp_sim3(np.r_[0, 0, 0, step, 0])[:3, :3] @ R
        if cost_R(Rn)[0] <= c0:
            R = Rn
        if np.linalg.norm(step) < 1e-12:
            break
    c, s = cost_R(R)
    return c, s, R


@pytest.mark.parametrize("npts,seed", [(3, 0), (4, 1), (5, 2), (8, 3), (6, 4)])
def test_umeyama_matches_brute_force(npts, seed):
    rng = np.random.default_rng(seed)
    y = rng.normal(size=(npts, 3))
    T = rand_sim3(rng)
    x = O.transform(T, y) + 0.05 * rng.normal(size=(npts, 3))
    s, R, t = O.umeyama(x, y)
    c_closed = ((x - (s * y @ R.T + t)) ** 2).sum()
    c_bf, s_bf, R_bf = _brute_force_alignment(x, y)
    assert c_closed <= c_bf + 1e-12
    assert abs(c_closed - c_bf) <= 1e-9 * max(1.0, c_bf)
    np.testing.assert_allclose(R, R_bf, atol=1e-5)
    assert abs(np.linalg.det(R) - 1) < 1e-12


def test_umeyama_reflection_case():
    """Points related by a reflection: det(U V^T) = -1 and S flips the last singular direction."""
    rng = np.random.default_rng(9)
    y = rng.normal(size=(6, 3))
    x = y * np.array([1.0, 1.0, -1.0])
    A = (x - x.mean(0)).T @ (y - y.mean(0))
    U, _, Vt = np.linalg.svd(A)
    assert np.linalg.det(U @ Vt) < 0
    s, R, t = O.umeyama(x, y)
    assert abs(np.linalg.det(R) - 1) < 1e-12
    c_closed = ((x - (s * y @ R.T + t)) ** 2).sum()
    c_bf, _, _ = _brute_force_alignment(x, y)
    assert abs(c_closed - c_bf) <= 1e-8 * max(1.0, c_bf)


# ------------------------------------------------------------------ escalation (Sec. III-D)
def test_cholesky_matches_library_and_detects_indefinite():
    rng = np.random.default_rng(10)
    B = rng.normal(size=(30, 30))
    A = B @ B.T + 30 * np.eye(30)
    np.testing.assert_allclose(O.cholesky(A), np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    A[5, 5] = -1.0
    assert O.cholesky(A) is None


def test_escalation_schedule():
    """An eigenvalue of -0.5 fails at eps = 1e-6, 1e-4, 1e-2 and succeeds at eps = 1 (attempt 4)."""
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.normal(size=(14, 14)))
    lam = np.r_[-0.5, np.linspace(1, 3, 13)]
    H = Q @ np.diag(lam) @ Q.T
    Hfull = np.zeros((21, 21)); Hfull[7:, 7:] = H   # keyframe 0 is the anchor
    g = np.r_[np.zeros(7), rng.normal(size=14)]
    tau, attempts, ok = O.damped_solve(Hfull, g, 0, 0.0, 1e-6, 6)
    assert ok and attempts == 4
    np.testing.assert_allclose((H + 1.0 * np.eye(14)) @ tau[1:].ravel(), -g[7:], atol=1e-10)
    assert np.all(tau[0] == 0)
    Hbad = np.zeros((21, 21)); Hbad[7:, 7:] = Q @ np.diag(np.r_[-1e6, lam[1:]]) @ Q.T
    tau, attempts, ok = O.damped_solve(Hbad, g, 0, 0.0, 1e-6, 6)
    assert not ok and attempts == 6 and np.all(tau == 0)


def test_degenerate_matches_are_skipped():
    rng = np.random.default_rng(12)
    Pi = np.c_[rng.normal(size=(10, 3)) + [0, 0, 4], np.ones(10)]
    Pj = Pi.copy()
    Pi[3, :3] = 0.0           # zero-range streamed point
    Pj[5, :3] = np.nan        # non-finite gathered point
    rec = O.linearize_edge(np.eye(4), np.eye(4), Pi, Pj, make_problem.__defaults__ and dict(
        sigma_ray=0.003, sigma_dist=10.0, huber_k=1.345, lam=0.0, eps0=1e-6, max_attempts=6))
    assert rec["n_skipped"] == 2 and rec["n_valid"] == 10 and rec["cost"] < 1e-20


def test_unlinked_component_keeps_its_own_reference():
    """Without inter-agent edges agent 1 forms its own component: its lowest keyframe is held
    fixed (Sec. III-C reading) and its other poses are recovered exactly relative to it."""
    p = make_problem(3, noise=0.0, outlier=0.0, exact=True, n_inter=0, name="split")
    assert O.component_anchors(p, 0) == [0, 6]
    poses, _ = O.gn_solve(p, p.poses_init, 10)
    G = O.pose_to_matrix(p.poses_init[6]) @ np.linalg.inv(O.pose_to_matrix(p.poses_gt[6]))
    want = np.array([O.matrix_to_pose(G @ O.pose_to_matrix(q)) for q in p.poses_gt[6:]])
    err = O.pose_errors(poses[6:], want)
    assert max(err.values()) < 1e-9, err
    assert max(O.pose_errors(poses[:6], p.poses_gt[:6]).values()) < 1e-9


# --------------------------------------- refined cost vs depth and confidence (Sec. III-E)
@pytest.fixture(scope="module")
def small_adj():
    """Two agents x 3 keyframes, 32x24 pointmaps, 5 edges, perturbed initial poses."""
    return make_problem(3, agents=2, n_kf=3, H=24, W=32, f=25.0, n_inter=1, iters=3)


@pytest.mark.parametrize("iters", [0, 2])
def test_refined_cost_complex_step_matches_central_difference(small_adj, iters):
    """The complex-step derivative of the unrolled refined cost equals a central finite
    difference of the real-valued computation along a dense random direction."""
    p = small_adj
    rng = np.random.default_rng(11)
    vl, vc = rng.normal(size=len(p.points)), rng.normal(size=len(p.points))
    cs = O.refined_cost_derivative(p, p.poses_init, iters, vl, vc)
    h = 1e-6
    fd = (O.refined_cost(p, p.poses_init, iters, h * vl, h * vc)
          - O.refined_cost(p, p.poses_init, iters, -h * vl, -h * vc)) / (2 * h)
    assert abs(cs - fd) <= 1e-5 * abs(cs)


def test_refined_cost_single_pixel_derivatives(small_adj):
    """Per-pixel derivatives (one log-range, one confidence) match central differences."""
    p = small_adj
    P = len(p.points)
    touched = np.unique(np.concatenate([p.pix_offset()[p.edge_i[e]] + np.nonzero(
        p.match_idx[p.idx_offset()[e]:p.idx_offset()[e + 1]] >= 0)[0] for e in range(p.num_edges)]))
    for pix in touched[[5, len(touched) // 2]]:
        for which in ("log", "conf"):
            v = np.zeros(P)
            v[pix] = 1.0
            args = (v, None) if which == "log" else (None, v)
            cs = O.refined_cost_derivative(p, p.poses_init, 1, *args)
            # the cost after an iteration carries ~1e-13 relative rounding noise, so the step
            # balances it against truncation
            h = 1e-4 if which == "log" else 1e-3
            sh = lambda s: (s * v, None) if which == "log" else (None, s * v)
            fd = (O.refined_cost(p, p.poses_init, 1, *sh(h)) - O.refined_cost(p, p.poses_init, 1, *sh(-h))) / (2 * h)
            L = O.refined_cost(p, p.poses_init, 1)
            assert abs(cs - fd) <= 1e-4 * abs(cs) + 2e-13 * abs(L) / h, (pix, which, cs, fd)


def test_envelope_derivative_uniform_confidence_scaling(small_adj):
    """Scaling every confidence by (1 + t) scales q by (1 + t) and every whitened residual
    by sqrt(1 + t), so at fixed poses dE/dt = sum rho'(r) r / 2 = sum w r^2 / 2."""
    p = small_adj
    c = p.points[:, 3].astype(np.float64)
    env = O.refined_cost_derivative(p, p.poses_init, 2, None, c, envelope=True)
    arrs = O.problem_arrays(p)
    T = O.gn_trajectory(p, p.poses_init, 2, arrs)
    expect = 0.0
    for e in range(p.num_edges):
        i, j, m, n, Pi, Pj = O.edge_matches(p, arrs, e)
        ee, _ = O.residual(np.linalg.inv(T[i]) @ T[j], Pi[:, :3], Pj[:, :3])
        r = O.whiten(ee, np.sqrt(Pi[:, 3] * Pj[:, 3]), p.sigma_ray, p.sigma_dist)
        expect += 0.5 * float((O.huber_weight(r, p.huber_k) * r * r).sum())
    assert abs(env - expect) <= 1e-12 * abs(expect)


def test_unrolled_derivative_approaches_envelope(small_adj):
    """At convergence g(T^K) -> 0, so dL/dtheta -> the partial derivative at fixed poses;
    after one iteration the two still differ."""
    p = small_adj
    rng = np.random.default_rng(5)
    vl, vc = rng.normal(size=len(p.points)), rng.normal(size=len(p.points))
    gap = lambda K: abs(O.refined_cost_derivative(p, p.poses_init, K, vl, vc)
                        - O.refined_cost_derivative(p, p.poses_init, K, vl, vc, envelope=True))
    env12 = abs(O.refined_cost_derivative(p, p.poses_init, 12, vl, vc, envelope=True))
    assert gap(12) <= 1e-3 * env12
    assert gap(1) >= 0.05 * env12


# -------------------------------------- cross-agent gate and gauge synchronisation
def _candidate(prob, e_fwd, e_bwd):
    """Keyframes, pointmaps and the two match directions of one cross-agent candidate."""
    px = prob.pixels_of().astype(np.int64)
    off = np.concatenate([[0], np.cumsum(px)])
    slots = np.concatenate([[0], np.cumsum(px[prob.edge_i.astype(np.int64)])])
    i, j = int(prob.edge_i[e_fwd]), int(prob.edge_j[e_fwd])
    assert (int(prob.edge_i[e_bwd]), int(prob.edge_j[e_bwd])) == (j, i)
    Pi = prob.points[off[i]:off[i + 1]].astype(np.float64)
    Pj = prob.points[off[j]:off[j + 1]].astype(np.float64)
    return i, j, Pi, Pj, prob.match_idx[slots[e_fwd]:slots[e_fwd + 1]], prob.match_idx[slots[e_bwd]:slots[e_bwd + 1]]


def _team(seed=31, **kw):
    from synth import make_cloud_problem
    spec = dict(agents=2, n_kf=6, H=24, W=32, period=30, shift=4, n_inter=2, reverse_inter=True)
    spec.update(kw)
    return make_cloud_problem(seed, [spec], dtype=np.float64)


def test_gauge_sync_recovers_the_moving_components_gauge():
    """Sec. III-C: if agent 1's poses carry an extra similarity G, the aligned T* is G^{-1}
    (exact correspondences), and transporting agent 1 by T* restores the ground truth."""
    p = _team()
    rng = np.random.default_rng(4)
    G = rand_sim3(rng, rot=0.7, trans=3.0, logs=0.4)
    moving = [k for k in range(p.num_kf) if p.agent_of[k] == 1]
    poses = p.poses_gt.copy()
    for k in moving:
        poses[k] = O.matrix_to_pose(G @ O.pose_to_matrix(poses[k]))
    E = p.num_edges
    i, j, Pi, Pj, fwd, bwd = _candidate(p, E - 4, E - 2)
    r = O.gauge_candidate(O.pose_to_matrix(poses[i]), O.pose_to_matrix(poses[j]), Pi, Pj, fwd, bwd, q_min=0.0)
    assert not r["fallback"] and r["n_c"] >= 64 and r["admitted"]
    np.testing.assert_allclose(r["T"], O.sim3_inverse(G), atol=1e-12)
    assert r["rms"] < 1e-12
    back = O.gauge_transport(poses, r["T"], moving)
    assert max(O.pose_errors(back, p.poses_gt).values()) < 1e-12


def test_gauge_sync_endpoint_fallback_below_nc_min():
    """Fewer than N_c^min high-confidence matches: T* = T_i T_j^{-1}, which puts j's pose
    exactly onto i's (the moving endpoint snaps onto the anchor)."""
    p = _team()
    E = p.num_edges
    i, j, Pi, Pj, fwd, bwd = _candidate(p, E - 4, E - 2)
    keep = np.nonzero(fwd >= 0)[0][:10]
    Pi = Pi.copy()
    Pi[:, 3] = 0.5
    Pi[keep, 3] = 10.0  # with c_j in (e^-1, ...) only these pass q_min = 1.5 (c_i c_j >= 2.25)
    Pj = Pj.copy()
    Pj[:, 3] = 1.0
    Ti, Tj = O.pose_to_matrix(p.poses_init[i]), O.pose_to_matrix(p.poses_init[j])
    r = O.gauge_candidate(Ti, Tj, Pi, Pj, fwd, bwd, q_min=1.5, nc_min=64)
    assert r["n_c"] == 10 and r["fallback"]
    np.testing.assert_allclose(r["T"] @ Tj, Ti, atol=1e-12)


def test_support_gate_counts_and_threshold():
    """Sec. III-B: nu = fraction of a view's pixels with a valid match whose
    q = sqrt(c_m c_n) reaches q_min (equality counts); the edge is admitted only when
    both directions reach nu_min; non-finite points are not counted."""
    p = _team()
    E = p.num_edges
    i, j, Pi, Pj, fwd, bwd = _candidate(p, E - 4, E - 2)
    Pi, Pj = Pi.copy(), Pj.copy()
    Pi[:, 3] = 1.0
    Pj[:, 3] = 1.0
    vf = np.nonzero(fwd >= 0)[0]
    pick = vf[:100]
    Pi[pick, 3] = 2.25  # with c_j = 1: q = 1.5 exactly, in both directions of a partner pair
    partners = fwd[pick]
    assert np.array_equal(bwd[partners], pick)  # the canvas matches are mutual on the overlap
    bwd = bwd.copy()
    bwd[partners[:63]] = -1  # 63 of the partners lose their backward match
    Pi[vf[100], 3] = 2.25
    Pi[vf[100], 0] = np.nan  # not finite: counted in neither direction
    r = O.gauge_candidate(np.eye(4), np.eye(4), Pi, Pj, fwd, bwd, q_min=1.5, nu_min=0.1)
    assert r["n_i"] == 100 and r["nu_i"] == 100 / Pi.shape[0]
    assert r["n_j"] == 37 and r["nu_j"] == 37 / Pj.shape[0]
    assert not r["admitted"]
    r2 = O.gauge_candidate(np.eye(4), np.eye(4), Pi, Pj, fwd, bwd, q_min=1.0, nu_min=0.1)
    nb = int((bwd >= 0).sum())
    assert r2["n_i"] == len(vf) - 1 and r2["n_j"] == nb - 1
    assert r2["admitted"] == (min((len(vf) - 1) / Pi.shape[0], (nb - 1) / Pj.shape[0]) >= 0.1)


def test_gauge_sync_is_equivariant_under_a_common_similarity():
    """A common similarity H applied to all poses conjugates T*: T*' = H T* H^{-1}."""
    p = _team(seed=32, noise=0.01, outlier=0.1)
    E = p.num_edges
    i, j, Pi, Pj, fwd, bwd = _candidate(p, E - 3, E - 1)
    H = rand_sim3(np.random.default_rng(5))
    Ti, Tj = O.pose_to_matrix(p.poses_init[i]), O.pose_to_matrix(p.poses_init[j])
    r = O.gauge_candidate(Ti, Tj, Pi, Pj, fwd, bwd, q_min=1.0)
    r2 = O.gauge_candidate(H @ Ti, H @ Tj, Pi, Pj, fwd, bwd, q_min=1.0)
    assert not r["fallback"]
    np.testing.assert_allclose(r2["T"], H @ r["T"] @ O.sim3_inverse(H), rtol=1e-9, atol=1e-9)


# ------------------------------------ segment-level structure refinement (Sec. III-E)
def _depth_case(seed=51, sigma=0.05, outlier=0.0, noise=0.0):
    from synth import make_cloud_problem
    from synth.segments import perturb_segment_ranges, problem_labels
    p = make_cloud_problem(seed, [dict(agents=2, n_kf=4, H=24, W=32, period=30, shift=4, n_inter=2,
                                       noise=noise, outlier=outlier)], dtype=np.float64)
    lab = problem_labels(p, n_seg=12, seed=seed)
    pix_off = np.concatenate([[0], np.cumsum(p.pixels_of())])
    anchors = set(O.component_anchors(p, 0))
    pts = perturb_segment_ranges(p.points, lab, pix_off, sigma, seed=seed)
    for k in anchors:  # the fixed keyframes keep their true ranges
        pts[pix_off[k]:pix_off[k + 1]] = p.points[pix_off[k]:pix_off[k + 1]]
    pts[:, 3] = np.maximum(pts[:, 3], 1.6)  # every pixel passes c_min
    import dataclasses
    return dataclasses.replace(p, points=pts), lab, p


def test_depth_gradient_is_the_full_gradient():
    """The Jacobi solver keeps the full gradient: g = dE'/d eta (complex step, exact to
    rounding), with Huber-downweighted outliers present."""
    p, lab, _ = _depth_case(outlier=0.1, noise=0.01)
    seg = O.depth_segments(p, lab)
    rng = np.random.default_rng(0)
    eta = rng.normal(size=seg["M"]) * 0.05
    _, g, _ = O.depth_terms(p, p.poses_gt, eta, seg)
    h = 1e-30
    for s in rng.choice(np.nonzero(seg["active"])[0], size=8, replace=False):
        e = eta.astype(complex)
        e[s] += 1j * h
        Ec, _, _ = O.depth_terms(p, p.poses_gt, e, seg)
        assert abs(np.imag(Ec) / h - g[s]) <= 1e-9 * max(1.0, abs(g[s])), s


def test_depth_jacobi_diagonal_is_the_exact_hessian_diagonal_at_zero_residual():
    """At consistent geometry (true ranges and poses) every data residual is 0, so the
    Gauss-Newton diagonal equals d^2 E'/d eta_s^2 (central difference of the gradient)."""
    _, lab, p = _depth_case()
    seg = O.depth_segments(p, lab)
    eta = np.zeros(seg["M"])
    _, g0, H = O.depth_terms(p, p.poses_gt, eta, seg)
    h = 1e-5
    for s in np.nonzero(seg["active"])[0][::7]:
        e1, e2 = eta.copy(), eta.copy()
        e1[s] += h
        e2[s] -= h
        d2 = (O.depth_terms(p, p.poses_gt, e1, seg)[1][s] - O.depth_terms(p, p.poses_gt, e2, seg)[1][s]) / (2 * h)
        assert abs(d2 - H[s]) <= 1e-6 * H[s], s


def test_depth_boundary_delta_of_a_constructed_step():
    """Two segments side by side whose log-ranges differ by a constant: Delta = -step."""
    _, lab, p = _depth_case()
    pts = p.points.copy()
    H, W = int(p.height[0]), int(p.width[0])
    lab2 = np.full(lab.shape, -1, dtype=np.int32)
    P = H * W
    cols = np.arange(P) % W
    lab2[:P] = np.where(cols < W // 2, 0, 1)
    d = np.where(cols < W // 2, np.exp(0.2), np.exp(0.2 + 0.37))
    ray = pts[:P, :3] / np.linalg.norm(pts[:P, :3], axis=1, keepdims=True)
    pts[:P, :3] = ray * d[:, None]
    pts[:, 3] = 2.0
    import dataclasses
    seg = O.depth_segments(dataclasses.replace(p, points=pts), lab2)
    assert len(seg["pairs"]) == 1
    a, b, delta = seg["pairs"][0]
    assert (a, b) == (0, 1) and abs(delta + 0.37) < 1e-12


def test_depth_refinement_recovers_injected_segment_scales():
    """Per-segment range errors exp(delta_g) on consistent data: iterated to convergence
    the Jacobi steps reach a stationary point of E' (g = 0) that undoes the errors
    (eta_g ~ -delta_g, up to the prior's pull), and E' falls."""
    from synth.segments import problem_labels
    p, lab, p0 = _depth_case(sigma=0.05)
    seg = O.depth_segments(p, lab)
    eta, trace = O.depth_refine(p, p.poses_gt, np.zeros(seg["M"]), 200, seg)
    _, g, H = O.depth_terms(p, p.poses_gt, eta, seg)
    assert np.abs(g[seg["active"]]).max() <= 1e-8 * np.abs(H).max()
    assert trace[-1] < 1e-3 * trace[0]
    # compare with the injected scales: log(|X_perturbed| / |X_true|) per segment
    d_pert = np.linalg.norm(p.points[:, :3], axis=1)
    d_true = np.linalg.norm(p0.points[:, :3], axis=1)
    inj = np.log(d_pert / d_true)
    e = seg["eff"]
    err = [abs(eta[s] + inj[e == s].mean()) for s in np.nonzero(seg["active"])[0]]
    assert np.median(err) < 2e-3 and max(err) < 2e-2


def test_depth_step_clip_and_fixed_segments():
    """A large range error moves its segment by exactly eta_max per step; segments of the
    fixed keyframes and inactive segments stay at 0."""
    p, lab, _ = _depth_case(sigma=0.0)
    seg = O.depth_segments(p, lab)
    pix_off = np.concatenate([[0], np.cumsum(p.pixels_of())])
    k = 5
    s0 = int(seg["base"][k]) + 3
    pts = p.points.copy()
    a = pix_off[k]
    sel = seg["eff"][a:pix_off[k + 1]] == s0
    pts[a:pix_off[k + 1]][sel, :3] *= np.exp(2.0)
    import dataclasses
    pb = dataclasses.replace(p, points=pts)
    seg = O.depth_segments(pb, lab)
    eta, _ = O.depth_refine(pb, pb.poses_gt, np.zeros(seg["M"]), 1, seg)
    assert abs(eta[s0] + 0.5) < 1e-15
    assert np.all(eta[seg["fixed"]] == 0) and np.all(eta[~seg["active"]] == 0)
    assert len(seg["fixed"]) > 0


# ----------------------------------- front-end: projective matching and fusion (Sec. III-A)
def _pair(seed=71, H=32, W=40, shift=5, noise=0.0):
    from synth import make_cloud_problem
    p = make_cloud_problem(seed, [dict(agents=1, n_kf=4, H=H, W=W, period=30, shift=shift, n_inter=0,
                                       noise=noise)], dtype=np.float32)
    arrs = O.problem_arrays(p)
    e = 0
    i, j = int(p.edge_i[e]), int(p.edge_j[e])
    idx = p.match_idx[arrs["idx_off"][e]:arrs["idx_off"][e + 1]]
    Pi = p.points[arrs["pix_off"][i]:arrs["pix_off"][i + 1]]
    Pj = p.points[arrs["pix_off"][j]:arrs["pix_off"][j + 1]]
    Tji = O.sim3_inverse(O.pose_to_matrix(p.poses_gt[j])) @ O.pose_to_matrix(p.poses_gt[i])
    q = np.concatenate([O.transform(Tji, Pi[:, :3].astype(np.float64)), Pi[:, 3:4]], axis=1).astype(np.float32)
    return p, Pj, q, idx, H, W


def test_projective_match_recovers_exact_correspondences():
    """Keyframe i's points expressed in frame j's camera are matched to exactly the pixels of
    j that see the same surface point (the generator's correspondences), from the same
    pixel index as start; pixels outside the overlap end beyond the angle threshold."""
    p, Pj, q, idx, H, W = _pair()
    got, d = O.project_match(Pj, H, W, q, np.arange(H * W), max_steps=64, max_angle=0.002)
    valid = idx >= 0
    assert valid.mean() > 0.5
    np.testing.assert_array_equal(got[valid], idx[valid])
    # outside the overlap the best ray is on j's border and farther than the threshold
    assert (got[~valid] == -1).mean() > 0.9


def test_projective_match_equals_brute_force_argmin():
    """On a smooth central-camera ray image the descent reaches the global argmin of the
    FP32 ray distance over all pixels (ties: lowest distance found first), from a far start."""
    rng = np.random.default_rng(5)
    H, W, f = 24, 32, 30.0
    v, u = np.mgrid[0:H, 0:W]
    rays = np.stack([(u - W / 2 + 0.5) / f, (v - H / 2 + 0.5) / f, np.ones_like(u, dtype=float)], -1).reshape(-1, 3)
    depth = 2.0 + rng.uniform(size=H * W)
    frame = np.concatenate([rays * depth[:, None], np.ones((H * W, 1))], 1).astype(np.float32)
    qd = np.stack([rng.uniform(-0.5, 0.5, 200), rng.uniform(-0.35, 0.35, 200), np.ones(200)], -1) * 3.0
    query = np.concatenate([qd, np.ones((200, 1))], 1).astype(np.float32)
    got, d = O.project_match(frame, H, W, query, np.zeros(200, dtype=np.int64), max_steps=200, max_angle=1.0)
    R = O.ray_image_f32(frame)
    Qr = O.ray_image_f32(query)
    allD = O.ray_dist_f32(R[None, :, :], Qr[:, None, :])
    np.testing.assert_array_equal(d, allD.min(axis=1))
    assert np.all(got >= 0)


def test_fusion_closed_forms():
    """Eq. (fusion): equal confidences average, the confidence accumulates, and a prediction
    that already equals the map (through T_kf) leaves the map's points unchanged."""
    rng = np.random.default_rng(6)
    X = rng.normal(size=(50, 3)) + np.array([0, 0, 5.0])
    canon = np.concatenate([X, np.full((50, 1), 2.0)], 1)
    T = rand_sim3(rng)
    pred_same = np.concatenate([O.transform(O.sim3_inverse(T), X), np.full((50, 1), 3.0)], 1)
    out = O.fuse(canon, pred_same, T)
    np.testing.assert_allclose(out[:, :3], X, atol=1e-12)
    np.testing.assert_array_equal(out[:, 3], 5.0)
    Y = rng.normal(size=(50, 3))
    out2 = O.fuse(canon, np.concatenate([Y, np.full((50, 1), 2.0)], 1), np.eye(4))
    np.testing.assert_allclose(out2[:, :3], 0.5 * (X + Y), atol=1e-15)


# -------------------------------------------------- pose error reports (parity measure)
# Every pose comparison of the GPU parity tests goes through O.pose_errors, so its three
# figures are pinned to constructed pose pairs whose errors are known by construction:
# a rotation composed from a known rotation vector (library rotation algebra, not the
# oracle's), a translation moved by a known length, a scale multiplied by a known ratio.
def _random_poses(rng, n):
    from scipy.spatial.transform import Rotation
    p = np.zeros((n, 8))
    p[:, :3] = rng.normal(size=(n, 3)) * 4.0
    p[:, 3:7] = Rotation.random(n, random_state=rng.integers(1 << 31)).as_quat()
    p[:, 7] = rng.uniform(0.5, 2.0, size=n)
    return p


def _unit(rng):
    u = rng.normal(size=3)
    return u / np.linalg.norm(u)


@pytest.mark.parametrize("theta", [3.1, 2.0, 0.1, 1.5e-3, 1.0e-3, 1e-4, 1e-6, 1e-8])
def test_pose_errors_known_rotation_angle(theta):
    """The rotation error is the angle of R_a R_b^T (the reading ||Log(R_a R_b^T)||), to 1e-12
    relative at any angle, the largest over keyframes; translation and scale are untouched."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(int(theta * 1e9) % 1000 + 7)
    b = _random_poses(rng, 6)
    a = b.copy()
    for l in range(6):
        ang = theta if l == 4 else theta * 0.25 * (l + 1) / 6
        a[l, 3:7] = (Rotation.from_rotvec(ang * _unit(rng)) * Rotation.from_quat(b[l, 3:7])).as_quat()
    err = O.pose_errors(a, b)
    assert abs(err["rot"] - theta) <= 1e-12 * theta + 1e-15, (err["rot"], theta)
    assert err["trans"] == 0.0 and err["scale"] == 0.0


def test_pose_errors_quaternion_sign_and_identity():
    """q and -q are one rotation (error 0); equal poses give exactly zero errors."""
    rng = np.random.default_rng(11)
    b = _random_poses(rng, 5)
    assert O.pose_errors(b, b) == dict(rot=0.0, trans=0.0, scale=0.0)
    a = b.copy()
    a[:, 3:7] = -a[:, 3:7]
    assert O.pose_errors(a, b)["rot"] <= 1e-15


@pytest.mark.parametrize("delta", [2.5, 1e-3, 1e-9])
def test_pose_errors_known_translation_offset(delta):
    """Camera centres at c +/- r e_x, c +/- r e_y have RMS radius r about their mean; a centre
    moved by delta reports delta / max(||t_b||, r) (relative to the larger of its own norm and
    the trajectory radius), or delta / max(||t_b||, ref) for a given reference length."""
    rng = np.random.default_rng(3)
    r = 3.0
    for c in (np.zeros(3), np.array([0.0, 0.0, 12.0])):
        b = _random_poses(rng, 4)
        b[:, :3] = c + r * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]], dtype=float)
        a = b.copy()
        a[2, :3] += delta * _unit(rng)
        a[1, :3] += 0.5 * delta * _unit(rng)
        want = delta / max(np.hypot(r, c[2]), r)
        err = O.pose_errors(a, b)
        # the offset itself is stored to the rounding of coordinates of size ||c|| + r
        ulp = 8 * np.finfo(float).eps * (np.linalg.norm(c) + r)
        assert abs(err["trans"] - want) <= 1e-12 * want + ulp / max(np.hypot(r, c[2]), r), (c, err, want)
        assert err["rot"] == 0.0 and err["scale"] == 0.0
        err = O.pose_errors(a, b, ref_scale=100.0)
        assert abs(err["trans"] - delta / 100.0) <= 1e-12 * delta / 100.0 + ulp / 100.0
    # the translation of an unmoved keyframe does not count, however far the others moved
    b = _random_poses(rng, 3)
    assert O.pose_errors(b, b, ref_scale=1.0)["trans"] == 0.0


@pytest.mark.parametrize("ratio", [0.3, -0.3, 1e-6, -1e-9])
def test_pose_errors_known_scale_ratio(ratio):
    """s_a = s_b (1 + rho) reports |rho|, the largest over keyframes."""
    rng = np.random.default_rng(5)
    b = _random_poses(rng, 5)
    a = b.copy()
    a[3, 7] = b[3, 7] * (1.0 + ratio)
    a[0, 7] = b[0, 7] * (1.0 + 0.5 * ratio)
    err = O.pose_errors(a, b)
    assert abs(err["scale"] - abs(ratio)) <= 1e-12 * abs(ratio) + 4e-16, (err, ratio)
    assert err["rot"] == 0.0 and err["trans"] == 0.0
