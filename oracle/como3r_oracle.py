"""Plain FP64 CPU oracle of the unified multi-agent Sim(3) Gauss-Newton refinement.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference that the CUDA
library is checked against.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline / reference legs may import it; the library never does, and
it shares no code with the library (its only inputs are the arrays of a problem).

It follows CoMo3R-SLAM (arXiv 2605.30488), Section III, step by step, with dense
matrices and no blocking or fusion:

* pose T = [sR t; 0 1] in Sim(3) maps camera to world; T_ij = T_i^{-1} T_j (Sec. III-A);
* ray operator psi(X) = X / ||X|| and the 4-vector ray-plus-range residual (Eq. residual);
* whitening Sigma_mn = Sigma / q_mn, Sigma = diag(sigma_r^2 I_3, sigma_d^2), and a
  component-wise Huber kernel with IRLS weight w(r) = min(1, kappa / |r|) (Sec. III-A);
* the global cost over intra- and inter-agent edges with the first anchor fixed
  (Eq. global);
* left perturbation T <- Exp(tau) T, tau = (v, omega, zeta), analytic Jacobians
  (Eq. jacobian) chained to both endpoints by -/+ Ad_{T_i^{-1}} (Sec. III-D);
* the regularised normal equations (Eq. normal) with the epsilon escalation
  eps_r = eps_0 * 100^r, at most six attempts, zero update if all fail (Sec. III-D);
* closed-form Umeyama alignment (Eq. align, Eq. umeyama), the bidirectional support gate
  of cross-agent candidates (Sec. III-B) and the gauge transport with its endpoint
  fallback (Sec. III-C).

Readings where the paper is silent (each also listed in the design notes):

* q_mn = sqrt(c_i,m * c_j,n) from the per-pixel confidences supplied with the pointmaps
  (they play the role of the descriptor confidences Q);
* rho(r) = r^2 / 2 for |r| <= kappa, kappa |r| - kappa^2 / 2 beyond, so rho'(r) = w(r) r;
* g = sum J^T W e is the gradient of E_global and the step solves (...) tau = -g;
* W_c = w(r_c) q / sigma_c^2, H = sum J^T W J (Gauss-Newton with IRLS weights);
* back-end lambda defaults to 0; a factorisation "fails" when a pivot is not > 0 or is
  not finite; attempts r = 0..5 use eps_r = 1e-6 * 100^r;
* a match is skipped when ||X_i,m|| or ||T_ij X_j,n|| is not > 1e-12, when
  c_i,m * c_j,n is negative, or when any of them is not finite;
* the anchor is removed from the unknowns (all seven of its degrees of freedom); a
  connected component of the edge graph that does not contain it gets its own
  deterministic reference, its lowest keyframe id (Sec. III-C: until a component is
  joined to agent 0's, a deterministic reference is selected for it), so every
  component's gauge is fixed and no update is decided by the eps regulariser alone.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

DEGENERATE = 1e-12


# Every routine below also runs on complex arrays: the derivative of the refined cost is
# checked by the complex-step method (perturb an input by i h, read Im(L) / h), so norms
# are sqrt(sum x^2) rather than absolute values and every branch (Huber region, pivot
# test, degenerate-match test) is decided on the real part.  For real inputs the values
# are unchanged.
def _norm(X: np.ndarray, keepdims: bool = False) -> np.ndarray:
    return np.sqrt(np.sum(X * X, axis=-1, keepdims=keepdims))


def _abs_real_sign(r: np.ndarray) -> np.ndarray:
    """|r| for real r; for complex r the analytic continuation r * sign(Re r)."""
    return np.where(r.real >= 0, r, -r)


def _dtype(*xs) -> type:
    return np.result_type(*[np.asarray(x).dtype for x in xs], np.float64)


# =============================================================== Sim(3) (Sec. III-A, III-D)
def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion stored (x, y, z, w)."""
    x, y, z, w = [float(v) for v in q]
    n = math.sqrt(x * x + y * y + z * z + w * w)
    x, y, z, w = x / n, y / n, z / n, w / n
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def pose_to_matrix(p: np.ndarray) -> np.ndarray:
    """4x4 similarity [sR t; 0 1] of a pose stored (tx, ty, tz, qx, qy, qz, qw, s) (Sec. III-A)."""
    T = np.eye(4)
    T[:3, :3] = p[7] * quat_to_rot(p[3:7])
    T[:3, 3] = p[:3]
    return T


def matrix_to_pose(T: np.ndarray) -> np.ndarray:
    """Inverse of pose_to_matrix: s = det(sR)^(1/3), R projected to SO(3) by SVD, q with w >= 0."""
    sR = T[:3, :3]
    s = np.cbrt(np.linalg.det(sR))
    U, _, Vt = np.linalg.svd(sR / s)
    R = U @ Vt
    from scipy.spatial.transform import Rotation
    q = Rotation.from_matrix(R).as_quat()  # (x, y, z, w)
    if q[3] < 0:
        q = -q
    return np.concatenate([T[:3, 3], q, [s]])


def sim3_inverse(T: np.ndarray) -> np.ndarray:
    return np.linalg.inv(T)


def skew(w: np.ndarray) -> np.ndarray:
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def hat(tau: np.ndarray) -> np.ndarray:
    """sim(3) generator of tau = (v, omega, zeta): [[omega^ + zeta I, v], [0, 0]] (Sec. III-D)."""
    X = np.zeros((4, 4), dtype=_dtype(tau))
    X[:3, :3] = np.array(skew(tau[3:6])) + tau[6] * np.eye(3)
    X[:3, 3] = tau[:3]
    return X


def exp_sim3(tau: np.ndarray) -> np.ndarray:
    """Exp(tau) as the matrix exponential of hat(tau) (library expm, scaling and squaring)."""
    tau = np.asarray(tau)
    return scipy.linalg.expm(hat(tau if np.iscomplexobj(tau) else tau.astype(np.float64)))


def log_sim3(T: np.ndarray) -> np.ndarray:
    """Inverse of exp_sim3 through the principal matrix logarithm (error reports only)."""
    L = np.real(scipy.linalg.logm(T))
    A = L[:3, :3]
    zeta = np.trace(A) / 3.0
    W = 0.5 * (A - A.T)
    return np.array([L[0, 3], L[1, 3], L[2, 3], W[2, 1], W[0, 2], W[1, 0], zeta])


def adjoint(T: np.ndarray) -> np.ndarray:
    """7x7 Ad_T with T hat(tau) T^{-1} = hat(Ad_T tau) for tau = (v, omega, zeta).

    With T = (sR, t): v' = sR v + [t]x R omega - zeta t, omega' = R omega, zeta' = zeta.
    """
    sR = T[:3, :3]
    det = np.linalg.det(sR)
    s = det ** (1.0 / 3.0) if np.iscomplexobj(det) else np.cbrt(det)
    R = sR / s
    t = T[:3, 3]
    Ad = np.zeros((7, 7), dtype=_dtype(T))
    Ad[:3, :3] = sR
    Ad[:3, 3:6] = np.array(skew(t)) @ R
    Ad[:3, 6] = -t
    Ad[3:6, 3:6] = R
    Ad[6, 6] = 1.0
    return Ad


# ============================================== residual, whitening, Huber (Sec. III-A)
def psi(X: np.ndarray) -> np.ndarray:
    """Ray operator psi(X) = X / ||X|| (row-wise)."""
    return X / _norm(X, keepdims=True)


def transform(T: np.ndarray, X: np.ndarray) -> np.ndarray:
    return X @ T[:3, :3].T + T[:3, 3]


def residual(Tij: np.ndarray, Xi: np.ndarray, Xj: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """e_mn = [psi(T_ij X_j,n) - psi(X_i,m); ||T_ij X_j,n|| - ||X_i,m||] (Eq. residual)."""
    x = transform(Tij, Xj)
    e = np.empty((x.shape[0], 4), dtype=_dtype(x, Xi))
    with np.errstate(invalid="ignore", divide="ignore"):
        e[:, :3] = psi(x) - psi(Xi)
    e[:, 3] = _norm(x) - _norm(Xi)
    return e, x


def whiten(e: np.ndarray, q: np.ndarray, sigma_ray: float, sigma_dist: float) -> np.ndarray:
    """r = Sigma_mn^{-1/2} e with Sigma_mn = diag(sigma_r^2, sigma_r^2, sigma_r^2, sigma_d^2) / q."""
    sig = np.array([sigma_ray, sigma_ray, sigma_ray, sigma_dist])
    return np.sqrt(q)[:, None] * e / sig[None, :]


def huber_rho(r: np.ndarray, kappa: float) -> np.ndarray:
    a = _abs_real_sign(r)
    return np.where(a.real <= kappa, 0.5 * r * r, kappa * a - 0.5 * kappa * kappa)


def huber_weight(r: np.ndarray, kappa: float) -> np.ndarray:
    """IRLS weight w(r) = min(1, kappa / |r|), equal to 1 at r = 0."""
    a = _abs_real_sign(r)
    with np.errstate(divide="ignore"):
        return np.where(a.real <= kappa, 1.0, kappa / np.where(a.real > 0, a, 1.0))


# ========================================================== Jacobians (Eq. jacobian)
def jacobian_rel(x: np.ndarray) -> np.ndarray:
    """d e / d tau for the left perturbation x <- Exp(tau) x, one 4x7 block per row of x.

    Product of the printed factors: Dx/Dtau = [I, -[x]x, x], Dpsi/Dx = (I - x x^T / d^2) / d,
    Dd/Dx = x^T / d.
    """
    M = x.shape[0]
    d = _norm(x)
    Dx = np.zeros((M, 3, 7), dtype=_dtype(x))
    Dx[:, :, 0:3] = np.eye(3)
    Dx[:, 0, 4], Dx[:, 0, 5] = x[:, 2], -x[:, 1]   # -[x]x
    Dx[:, 1, 3], Dx[:, 1, 5] = -x[:, 2], x[:, 0]
    Dx[:, 2, 3], Dx[:, 2, 4] = x[:, 1], -x[:, 0]
    Dx[:, :, 6] = x
    outer = x[:, :, None] * x[:, None, :]
    Dpsi = (np.eye(3)[None] - outer / (d * d)[:, None, None]) / d[:, None, None]
    Dd = (x / d[:, None])[:, None, :]
    J = np.empty((M, 4, 7), dtype=_dtype(x))
    J[:, :3, :] = Dpsi @ Dx
    J[:, 3:, :] = Dd @ Dx
    return J


# ========================================================== problem access helpers
def problem_arrays(prob) -> Dict[str, np.ndarray]:
    """The arrays of a problem as FP64 views (storage values upcast exactly)."""
    pix = prob.pixels_of()
    return dict(points=np.asarray(prob.points, dtype=np.float64),
                pix_off=np.concatenate([[0], np.cumsum(pix)]).astype(np.int64),
                idx_off=np.concatenate([[0], np.cumsum(pix[prob.edge_i])]).astype(np.int64))


def edge_matches(prob, arrs, e: int):
    """Valid (m, n) pairs of edge e and the points/confidences they touch."""
    i, j = int(prob.edge_i[e]), int(prob.edge_j[e])
    idx = prob.match_idx[arrs["idx_off"][e]:arrs["idx_off"][e + 1]]
    m = np.nonzero(idx >= 0)[0]
    n = idx[m].astype(np.int64)
    Pi = arrs["points"][arrs["pix_off"][i] + m]
    Pj = arrs["points"][arrs["pix_off"][j] + n]
    return i, j, m, n, Pi, Pj


# ======================================== one edge, linearised (Eq. global, jacobian)
def linearize_edge(Ti: np.ndarray, Tj: np.ndarray, Pi: np.ndarray, Pj: np.ndarray,
                   params: Dict[str, float]) -> Dict[str, np.ndarray]:
    """Residuals, IRLS weights, edge Jacobians and the blocks one edge adds.

    Returns the relative-pose blocks H_rel = sum J^T W J, g_rel = sum J^T W e (J w.r.t. a
    left perturbation of T_ij), the endpoint blocks H_ii, H_jj, H_ij, g_i, g_j built from
    per-match J_i = -J Ad, J_j = J Ad with Ad = Ad_{T_i^{-1}}, the cost and the counts.
    """
    Tij = sim3_inverse(Ti) @ Tj
    Xi, ci = Pi[:, :3], Pi[:, 3]
    Xj, cj = Pj[:, :3], Pj[:, 3]
    e, x = residual(Tij, Xi, Xj)
    di = _norm(Xi)
    d = _norm(x)
    cc = ci * cj
    with np.errstate(invalid="ignore"):
        ok = ((di.real > DEGENERATE) & (d.real > DEGENERATE) & (cc.real >= 0) & np.isfinite(di) & np.isfinite(d)
              & np.isfinite(cc))
    ok &= np.all(np.isfinite(e), axis=1)
    e, x, cc = e[ok], x[ok], cc[ok]
    q = np.sqrt(cc)
    r = whiten(e, q, params["sigma_ray"], params["sigma_dist"])
    w = huber_weight(r, params["huber_k"])
    sig = np.array([params["sigma_ray"]] * 3 + [params["sigma_dist"]])
    W = w * q[:, None] / (sig * sig)[None, :]
    cost = huber_rho(r, params["huber_k"]).sum()
    cost = complex(cost) if np.iscomplexobj(cost) else float(cost)
    J = jacobian_rel(x)
    Ad = adjoint(sim3_inverse(Ti))
    Ji = -J @ Ad
    Jj = J @ Ad
    ein = lambda A, B: np.einsum("mci,mc,mcj->ij", A, W, B, optimize=True)
    return dict(
        H_rel=ein(J, J), g_rel=np.einsum("mci,mc,mc->i", J, W, e, optimize=True),
        H_ii=ein(Ji, Ji), H_jj=ein(Jj, Jj), H_ij=ein(Ji, Jj),
        g_i=np.einsum("mci,mc,mc->i", Ji, W, e, optimize=True),
        g_j=np.einsum("mci,mc,mc->i", Jj, W, e, optimize=True),
        cost=cost, n_valid=int(ok.size), n_skipped=int((~ok).sum()), Ad=Ad)


def build_system(prob, poses: np.ndarray, graph: int = 0, arrs=None, T_global=None):
    """Dense normal equations of one graph: H (7N x 7N), g (7N), cost, per-edge records.

    Keyframes of the graph are numbered locally from 0; the anchor is still included.
    The poses come from `poses` (stored form) or, when given, from the list of 4x4
    matrices `T_global` indexed by global keyframe id.
    """
    arrs = arrs or problem_arrays(prob)
    params = prob.params()
    k0, k1 = int(prob.kf_offset[graph]), int(prob.kf_offset[graph + 1])
    N = k1 - k0
    T = [pose_to_matrix(poses[k]) for k in range(k0, k1)] if T_global is None else T_global[k0:k1]
    dt = _dtype(arrs["points"], *T)
    H = np.zeros((7 * N, 7 * N), dtype=dt)
    g = np.zeros(7 * N, dtype=dt)
    cost = 0.0
    records = []
    for e in range(int(prob.edge_offset[graph]), int(prob.edge_offset[graph + 1])):
        i, j, m, n, Pi, Pj = edge_matches(prob, arrs, e)
        li, lj = i - k0, j - k0
        rec = linearize_edge(T[li], T[lj], Pi, Pj, params)
        si, sj = slice(7 * li, 7 * li + 7), slice(7 * lj, 7 * lj + 7)
        H[si, si] += rec["H_ii"]
        H[sj, sj] += rec["H_jj"]
        H[si, sj] += rec["H_ij"]
        H[sj, si] += rec["H_ij"].T
        g[si] += rec["g_i"]
        g[sj] += rec["g_j"]
        cost += rec["cost"]
        records.append(rec)
    return H, g, cost, records


# ============================= regularised normal equations (Eq. normal, Sec. III-D)
def cholesky(A: np.ndarray) -> Optional[np.ndarray]:
    """Textbook Cholesky-Crout A = L L^T; None when a pivot is not > 0 or not finite."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        piv = A[j, j] - L[j, :j] @ L[j, :j]
        if not (np.isfinite(piv) and piv.real > 0.0):
            return None
        L[j, j] = np.sqrt(piv)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def component_anchors(prob, graph: int = 0) -> List[int]:
    """Local ids of the fixed keyframes of one graph: the given anchor for its connected
    component, the lowest keyframe id for every other component (edges define adjacency)."""
    k0, k1 = int(prob.kf_offset[graph]), int(prob.kf_offset[graph + 1])
    parent = list(range(k1 - k0))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for e in range(int(prob.edge_offset[graph]), int(prob.edge_offset[graph + 1])):
        a, b = find(int(prob.edge_i[e]) - k0), find(int(prob.edge_j[e]) - k0)
        if a != b:
            parent[max(a, b)] = min(a, b)
    anchor = int(prob.anchor[graph]) - k0
    fixed = {find(anchor): anchor}
    for k in range(k1 - k0):
        fixed.setdefault(find(k), k)
    return sorted(fixed.values())


def damped_solve(H: np.ndarray, g: np.ndarray, anchor, lam: float, eps0: float,
                 max_attempts: int) -> Tuple[np.ndarray, int, bool]:
    """Solve (H + lam diag(H) + eps_r I) tau = -g over all keyframes but the anchor(s).

    eps_r = eps0 * 100^r for r = 0 .. max_attempts-1; the first successful
    factorisation is used; if none succeeds the update is zero.  Returns (tau [N, 7],
    attempts made, success).
    """
    N = H.shape[0] // 7
    fixed = {int(anchor)} if np.isscalar(anchor) else {int(a) for a in anchor}
    keep = np.array([k for k in range(7 * N) if k // 7 not in fixed], dtype=np.int64)
    Hr = H[np.ix_(keep, keep)]
    gr = g[keep]
    tau = np.zeros(7 * N, dtype=_dtype(H, g))
    for r in range(max_attempts):
        eps = eps0 * 100.0 ** r
        A = Hr + lam * np.diag(np.diag(Hr)) + eps * np.eye(Hr.shape[0])
        L = cholesky(A)
        if L is None:
            continue
        y = scipy.linalg.solve_triangular(L, -gr, lower=True)
        tau[keep] = scipy.linalg.solve_triangular(L.T, y, lower=False)
        return tau.reshape(N, 7), r + 1, True
    return tau.reshape(N, 7), max_attempts, False


# ======================================================= Gauss-Newton (Sec. III-D)
def retract(poses: np.ndarray, tau: np.ndarray, k0: int = 0) -> np.ndarray:
    """T_i <- Exp(tau_i) T_i for the keyframes k0 .. k0 + len(tau) - 1."""
    out = poses.copy()
    for l in range(tau.shape[0]):
        if not np.any(tau[l]):
            continue
        out[k0 + l] = matrix_to_pose(exp_sim3(tau[l]) @ pose_to_matrix(poses[k0 + l]))
    return out


def gn_step(prob, poses: np.ndarray, arrs=None) -> Tuple[np.ndarray, List[dict]]:
    """One iteration for every graph: linearise, solve the damped system, retract."""
    arrs = arrs or problem_arrays(prob)
    out = poses.copy()
    infos = []
    for gidx in range(prob.num_graphs):
        k0 = int(prob.kf_offset[gidx])
        H, g, cost, recs = build_system(prob, poses, gidx, arrs)
        tau, attempts, ok = damped_solve(H, g, component_anchors(prob, gidx), prob.lam, prob.eps0,
                                         prob.max_attempts)
        out = retract(out, tau, k0)
        infos.append(dict(cost=cost, attempts=attempts, ok=ok, H=H, g=g, tau=tau,
                          n_skipped=sum(r["n_skipped"] for r in recs)))
    return out, infos


def gn_solve(prob, poses: np.ndarray, iters: int) -> Tuple[np.ndarray, np.ndarray]:
    """`iters` GN iterations; returns the poses and the cost trace [iters + 1, G]."""
    arrs = problem_arrays(prob)
    trace = np.zeros((iters + 1, prob.num_graphs))
    for k in range(iters):
        poses, infos = gn_step(prob, poses, arrs)
        trace[k] = [inf["cost"] for inf in infos]
    trace[iters] = [build_system(prob, poses, gidx, arrs)[2] for gidx in range(prob.num_graphs)]
    return poses, trace


def total_cost(prob, poses: np.ndarray) -> np.ndarray:
    arrs = problem_arrays(prob)
    return np.array([build_system(prob, poses, gidx, arrs)[2] for gidx in range(prob.num_graphs)])


# ============== refined cost as a function of depth and confidence (Sec. III-E)
# The pose-depth alternation of Sec. III-E feeds the refined back-end cost back into the
# dense structure.  Here the structure is parameterised per pixel by its log-range l_p
# (X_p = exp(l_p) psi(X_p): moving l_p slides the point along its fixed viewing ray, so a
# log-depth and a log-range change have the same derivative) and its confidence c_p.  The
# refined cost is L(theta) = sum over graphs of E_global(T^K(theta), theta): K Gauss-Newton
# iterations from fixed initial poses, then the cost.  Its derivative is checked by the
# complex-step method, which differentiates exactly the steps above (IRLS weights, the
# damped factorisation, the retraction) without any hand-derived adjoint.
def reparameterised_points(prob, dlog=None, dconf=None) -> np.ndarray:
    """Stored pointmaps with every point scaled by exp(dlog_p) along its ray and every
    confidence shifted by dconf_p ([sum P] each; real or complex)."""
    pts = np.asarray(prob.points, dtype=np.float64)
    dt = _dtype(pts, 0.0 if dlog is None else dlog, 0.0 if dconf is None else dconf)
    out = pts.astype(dt)
    if dlog is not None:
        out[:, :3] = out[:, :3] * np.exp(dlog)[:, None]
    if dconf is not None:
        out[:, 3] = out[:, 3] + dconf
    return out


def gn_trajectory(prob, poses0: np.ndarray, iters: int, arrs) -> List[np.ndarray]:
    """The iterations of gn_solve with every pose kept as a 4x4 similarity matrix and
    updated by T <- Exp(tau) T (matrix exponential); runs in the dtype of the arrays.
    Returns the matrices T^K, indexed by global keyframe id."""
    T = [pose_to_matrix(p).astype(_dtype(arrs["points"])) for p in poses0]
    for _ in range(iters):
        steps = []
        for gidx in range(prob.num_graphs):
            H, g, _, _ = build_system(prob, None, gidx, arrs, T_global=T)
            tau, _, _ = damped_solve(H, g, component_anchors(prob, gidx), prob.lam, prob.eps0, prob.max_attempts)
            steps.append((int(prob.kf_offset[gidx]), tau))
        for k0, tau in steps:
            for l in range(tau.shape[0]):
                if np.any(tau[l] != 0):
                    T[k0 + l] = exp_sim3(tau[l]) @ T[k0 + l]
    return T


def refined_cost(prob, poses0: np.ndarray, iters: int, dlog=None, dconf=None, envelope: bool = False):
    """L = sum_g E_g(T^K, theta) at theta shifted by (dlog, dconf).

    Unrolled (default): T^K comes from `iters` iterations run at the shifted theta.
    Envelope: T^K comes from the unshifted theta and only the explicit dependence of the
    cost on theta remains (the partial derivative at fixed poses)."""
    arrs = problem_arrays(prob)
    arrs_theta = dict(arrs, points=reparameterised_points(prob, dlog, dconf))
    T = gn_trajectory(prob, poses0, iters, arrs if envelope else arrs_theta)
    return sum(build_system(prob, None, gidx, arrs_theta, T_global=T)[2] for gidx in range(prob.num_graphs))


def refined_cost_derivative(prob, poses0: np.ndarray, iters: int, vlog=None, vconf=None, envelope: bool = False,
                            h: float = 1e-30) -> float:
    """Directional derivative of refined_cost along (vlog, vconf) by the complex step,
    Im L(theta + i h v) / h (Squire and Trapp, 1998): no subtractive cancellation, so it is
    exact to rounding for any small h; every branch is taken on the real part."""
    dl = None if vlog is None else 1j * h * np.asarray(vlog, dtype=np.float64)
    dc = None if vconf is None else 1j * h * np.asarray(vconf, dtype=np.float64)
    return float(np.imag(refined_cost(prob, poses0, iters, dl, dc, envelope)) / h)


# ================================================== Umeyama (Eq. align, Eq. umeyama)
def umeyama(x: np.ndarray, y: np.ndarray) -> Tuple[float, np.ndarray, np.ndarray]:
    """(s, R, t) minimising sum ||x_l - (s R y_l + t)||^2 in closed form."""
    mx, my = x.mean(axis=0), y.mean(axis=0)
    xc, yc = x - mx, y - my
    A = xc.T @ yc / x.shape[0]
    U, lam, Vt = np.linalg.svd(A)
    S = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt)) or 1.0])
    R = U @ S @ Vt
    s = float(np.trace(S @ np.diag(lam)) / ((yc * yc).sum() / x.shape[0]))
    t = mx - s * R @ my
    return s, R, t


# ============================ cross-agent verification and gauge synchronisation
# Sec. III-B (bidirectional support gate) and Sec. III-C (Eq. align, Eq. umeyama, and the
# endpoint transform below N_c^min correspondences).
#
# Readings: a match of pixel m (of the view whose pixels are listed) is "valid" when its
# index is >= 0, and "high-confidence" when moreover c_m * c_n >= q_min^2, i.e.
# q_mn = sqrt(c_m c_n) >= q_min, tested on the exact product of the stored confidences
# (exact in FP64 for FP16 / FP32 storage) against q_min^2 rounded once to FP64; nu of a
# view = its high-confidence matches / its pixel count; the alignment uses the
# high-confidence matches of the forward direction (pixels of i matched into j), lifted
# with the current poses; a match whose points are not finite is neither counted nor used.
def support_mask(Pa: np.ndarray, Pb: np.ndarray, idx: np.ndarray, q_min: float) -> np.ndarray:
    """High-confidence valid matches of the pixels of view a into view b (boolean [P_a])."""
    idx = np.asarray(idx, dtype=np.int64)
    ok = idx >= 0
    n = np.where(ok, idx, 0)
    ca = Pa[:, 3].astype(np.float64)
    cb = Pb[n, 3].astype(np.float64)
    fin = np.isfinite(Pa.astype(np.float64)).all(axis=1) & np.isfinite(Pb[n].astype(np.float64)).all(axis=1)
    return ok & fin & (ca * cb >= float(q_min) * float(q_min))


def gauge_candidate(Ti: np.ndarray, Tj: np.ndarray, Pi: np.ndarray, Pj: np.ndarray, idx_ij: np.ndarray,
                    idx_ji: np.ndarray, q_min: float = 1.5, nu_min: float = 0.1, nc_min: int = 64) -> dict:
    """One inter-agent candidate (i, j): the support fractions nu_i, nu_j, the admission
    decision min(nu_i, nu_j) >= nu_min (Sec. III-B), and the similarity T* that maps j's
    component onto i's (Sec. III-C): Umeyama on the lifted correspondences
    x = T_i X_i,m, y = T_j X_j,n when there are at least nc_min of them, else the
    endpoint transform T_i T_j^{-1}.  T* is to be left-multiplied onto the moving poses."""
    mf = support_mask(Pi, Pj, idx_ij, q_min)
    mb = support_mask(Pj, Pi, idx_ji, q_min)
    nu_i = float(mf.sum()) / Pi.shape[0]
    nu_j = float(mb.sum()) / Pj.shape[0]
    m = np.nonzero(mf)[0]
    n = np.asarray(idx_ij, dtype=np.int64)[m]
    x = transform(Ti, Pi[m, :3].astype(np.float64))
    y = transform(Tj, Pj[n, :3].astype(np.float64))
    Nc = int(m.size)
    if Nc >= nc_min:
        s, R, t = umeyama(x, y)
        Ts = np.eye(4)
        Ts[:3, :3] = s * R
        Ts[:3, 3] = t
        fallback = False
    else:
        Ts = Ti @ sim3_inverse(Tj)
        fallback = True
    res = x - transform(Ts, y) if Nc else np.zeros((0, 3))
    rms = float(np.sqrt((res * res).sum(axis=1).mean())) if Nc else 0.0
    return dict(nu_i=nu_i, nu_j=nu_j, n_i=int(mf.sum()), n_j=int(mb.sum()), n_c=Nc,
                admitted=bool(min(nu_i, nu_j) >= nu_min), fallback=fallback, T=Ts, rms=rms)


def gauge_transport(poses: np.ndarray, Ts: np.ndarray, members: Sequence[int]) -> np.ndarray:
    """Left-multiplies T* onto the poses of the moving component's keyframes (Sec. III-C)."""
    out = np.array(poses, dtype=np.float64, copy=True)
    for k in members:
        out[k] = matrix_to_pose(Ts @ pose_to_matrix(out[k]))
    return out


# ======================= terminal segment-level structure refinement (Sec. III-E)
# Eq. depth_parameter, Eq. depth_data, Eq. depth_total and the Jacobi-style damped Newton
# update described after them.
#
# Readings: segment labels are given per pixel (the SLIC clustering is not part of the
# method's hot path); a pixel takes part when its label is >= 0, its confidence >= c_min
# (1.5), its point is finite with range > 1e-12, and its segment has >= min_pixels (16)
# such pixels -- otherwise its point stays at the snapshot (eta = 0 for it).  Global
# segment ids are k's base + label (base = sum of (max label + 1) of earlier keyframes).
# Delta_gh (g < h) is the mean, over the unordered 4-adjacent pixel pairs (p in g,
# p' in h) of a keyframe, of log d_p - log d_p' of the snapshot.  The normal equations are
# those of the stacked weighted least-squares problem, which the printed H_prior =
# lambda_prior I fixes: the boundary and prior terms enter as lambda * (.)^2 / 2 blocks
# beside the data term's Huber costs (rho = r^2 / 2 inside the breakpoint):
#   E' = E_data + lambda_smooth / 2 * E_bnd + lambda_prior / 2 * E_prior,  g = dE'/d eta.
# The Huber breakpoint is the graph's kappa.  The 1x1 step is the LM step of the
# back-end's damping form, delta = -g / ((1 + lambda_lm) H), clipped to |delta| <= eta_max;
# segments of the fixed keyframes (the anchor and every other component's reference)
# and inactive segments do not move.  A match touches the segments of its two pixels
# (either may be none); the per-match degenerate rule is the pose path's.
DEPTH_DEFAULTS = dict(c_min=1.5, min_pixels=16, sigma_point=0.05, lambda_smooth=1.0, lambda_prior=1.0,
                      lambda_lm=0.05, eta_max=0.5)


def depth_segments(prob, labels: np.ndarray, c_min: float = 1.5, min_pixels: int = 16, **_) -> dict:
    """Effective global segment of every pixel (-1: none), segment count M, the boundary
    pairs (g, h, Delta_gh), fixed segments, and the snapshot rays / log-ranges."""
    arrs = problem_arrays(prob)
    P = arrs["points"]
    X = P[:, :3]
    with np.errstate(invalid="ignore", over="ignore"):
        d = np.sqrt((X * X).sum(axis=1))
        fin = np.isfinite(P).all(axis=1) & (d > DEGENERATE)
    logd = np.where(fin, np.log(np.where(fin, d, 1.0)), 0.0)
    psi_ = np.where(fin[:, None], X / np.where(fin, d, 1.0)[:, None], 0.0)
    labels = np.asarray(labels, dtype=np.int64)
    eff = np.full(labels.shape, -1, dtype=np.int64)
    fixed_kf = set()
    for g in range(prob.num_graphs):
        k0 = int(prob.kf_offset[g])
        fixed_kf.update(k0 + a for a in component_anchors(prob, g))
    base, M = [], 0
    pairs: Dict[Tuple[int, int], List[float]] = {}
    fixed = []
    for g in range(prob.num_graphs):
        H, W = int(prob.height[g]), int(prob.width[g])
        for k in range(int(prob.kf_offset[g]), int(prob.kf_offset[g + 1])):
            a0, a1 = arrs["pix_off"][k], arrs["pix_off"][k + 1]
            L = labels[a0:a1]
            Mk = int(L.max()) + 1 if (L >= 0).any() else 0
            ok = (L >= 0) & fin[a0:a1] & (P[a0:a1, 3] >= c_min)
            cnt = np.bincount(L[ok], minlength=Mk) if Mk else np.zeros(0, dtype=np.int64)
            act = cnt >= min_pixels
            e = np.where(ok & (L >= 0) & act[np.maximum(L, 0)] if Mk else ok & False, M + L, -1)
            eff[a0:a1] = e
            if k in fixed_kf:
                fixed += list(range(M, M + Mk))
            E2 = e.reshape(H, W)
            LD = logd[a0:a1].reshape(H, W)
            for (ea, eb, la, lb) in ((E2[:, :-1], E2[:, 1:], LD[:, :-1], LD[:, 1:]),
                                     (E2[:-1, :], E2[1:, :], LD[:-1, :], LD[1:, :])):
                sel = (ea >= 0) & (eb >= 0) & (ea != eb)
                for u, v, lu, lv in zip(ea[sel], eb[sel], la[sel], lb[sel]):
                    key, diff = ((int(u), int(v)), lu - lv) if u < v else ((int(v), int(u)), lv - lu)
                    acc = pairs.setdefault(key, [0.0, 0])
                    acc[0] += diff
                    acc[1] += 1
            base.append(M)
            M += Mk
    bnd = [(g_, h_, sm / n) for (g_, h_), (sm, n) in sorted(pairs.items())]
    active = np.zeros(M, dtype=bool)
    active[eff[eff >= 0]] = True
    return dict(eff=eff, M=M, base=np.array(base, dtype=np.int64), pairs=bnd, fixed=np.array(sorted(set(fixed)),
                dtype=np.int64), active=active, logd=logd, psi=psi_, conf=P[:, 3].copy(), arrs=arrs)


def depth_terms(prob, poses: np.ndarray, eta: np.ndarray, seg: dict, sigma_point: float = 0.05,
                lambda_smooth: float = 1.0, lambda_prior: float = 1.0, **_) -> Tuple[float, np.ndarray, np.ndarray]:
    """(E', g, H) at eta: the objective, its full gradient and the Jacobi diagonal (the
    cross-segment data term J_g^T W J_h and the off-diagonal boundary pair dropped)."""
    M = seg["M"]
    eta = np.asarray(eta)
    g = np.zeros(M, dtype=eta.dtype)
    Hd = np.zeros(M)
    E = 0.0 * eta.sum()
    arrs, eff, logd, psi_, conf = seg["arrs"], seg["eff"], seg["logd"], seg["psi"], seg["conf"]
    kappa = prob.huber_k
    T = [pose_to_matrix(p) for p in poses]
    for e in range(prob.num_edges):
        i, j = int(prob.edge_i[e]), int(prob.edge_j[e])
        idx = prob.match_idx[arrs["idx_off"][e]:arrs["idx_off"][e + 1]]
        m = np.nonzero(idx >= 0)[0]
        n = idx[m].astype(np.int64)
        pm, pn = arrs["pix_off"][i] + m, arrs["pix_off"][j] + n
        si, sj = eff[pm], eff[pn]
        eti = np.where(si >= 0, eta[np.maximum(si, 0)], 0.0)
        etj = np.where(sj >= 0, eta[np.maximum(sj, 0)], 0.0)
        Xi = (np.exp(logd[pm] + eti))[:, None] * psi_[pm]
        Xj = (np.exp(logd[pn] + etj))[:, None] * psi_[pn]
        Tij = sim3_inverse(T[i]) @ T[j]
        Y = transform(Tij, Xj)
        cc = conf[pm] * conf[pn]
        ok = (np.isfinite(arrs["points"][pm]).all(1) & np.isfinite(arrs["points"][pn]).all(1)
              & (_norm(Xi).real > DEGENERATE) & (_norm(Y).real > DEGENERATE) & (cc >= 0))
        if not ok.any():
            continue
        Xi, Y, cc, si, sj = Xi[ok], Y[ok], cc[ok], si[ok], sj[ok]
        k = np.sqrt(np.sqrt(cc)) / sigma_point
        r = k[:, None] * (Y - Xi)
        w = huber_weight(r, kappa)
        E = E + huber_rho(r, kappa).sum()
        Jg = -k[:, None] * Xi
        Jh = k[:, None] * (Y - Tij[:3, 3])
        for sg, J in ((si, Jg), (sj, Jh)):
            a = sg >= 0
            np.add.at(g, sg[a], (w * r * J).sum(axis=1)[a])
            np.add.at(Hd, sg[a], (w * J * J).real.sum(axis=1)[a])
    for (a, b, delta) in seg["pairs"]:
        res = eta[a] - eta[b] + delta
        E = E + 0.5 * lambda_smooth * res * res
        g[a] += lambda_smooth * res
        g[b] -= lambda_smooth * res
        Hd[a] += lambda_smooth
        Hd[b] += lambda_smooth
    act = seg["active"]
    E = E + 0.5 * lambda_prior * (eta[act] * eta[act]).sum()
    g[act] += lambda_prior * eta[act]
    Hd[act] += lambda_prior
    return E, g, Hd


def depth_refine(prob, poses: np.ndarray, eta0: np.ndarray, iters: int, seg: dict, **params):
    """Up to `iters` Jacobi 1x1 damped Newton steps (poses fixed); returns (eta, trace of E')."""
    p = dict(DEPTH_DEFAULTS)
    p.update(params)
    eta = np.array(eta0, dtype=np.float64, copy=True)
    movable = seg["active"].copy()
    movable[seg["fixed"]] = False
    trace = []
    for _ in range(iters):
        E, g, Hd = depth_terms(prob, poses, eta, seg, **p)
        trace.append(float(E))
        step = np.zeros_like(eta)
        mv = movable & (Hd > 0)
        step[mv] = np.clip(-g[mv] / ((1.0 + p["lambda_lm"]) * Hd[mv]), -p["eta_max"], p["eta_max"])
        eta = eta + step
    trace.append(float(depth_terms(prob, poses, eta, seg, **p)[0]))
    return eta, np.array(trace)


# ================== front-end: projective ray matching and fusion (Sec. III-A)
# Matching minimises the angular discrepancy on the frame's predicted ray image,
# p* = argmin_p |psi([X^f_f]_p) - psi(x)|^2, for every queried point x.  Reading (the paper
# cites its iterative solver without printing it): a deterministic descent over pixels --
# from a start pixel, move to the best of the 8 neighbours (fixed order, strictly smaller
# distance, first in order on ties) while it improves, at most max_steps moves -- with
# every distance in FP32, each operation correctly rounded in this order:
#   n = sqrt((x0*x0 + x1*x1) + x2*x2), psi = (x0/n, x1/n, x2/n),
#   d = ((a0-b0)*(a0-b0) + (a1-b1)*(a1-b1)) + (a2-b2)*(a2-b2),
# so that the integer result is the same on any IEEE implementation.  A query whose
# point is not finite or has zero norm, or whose final distance exceeds d_max (the
# squared chord of max_angle: 2 - 2 cos(max_angle), rounded to FP32), gets -1.  Frame
# pixels whose ray is not finite are never entered.
_NB8 = ((-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1))


def ray_image_f32(P: np.ndarray) -> np.ndarray:
    """psi of every point in FP32 with the fixed operation order (NaN for a zero or
    non-finite point)."""
    x = np.asarray(P[:, :3], dtype=np.float32)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        n = np.sqrt((x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2])
        r = x / n[:, None]
    bad = ~(np.isfinite(r).all(axis=1) & (n > 0))
    r[bad] = np.float32(np.nan)
    return r


def ray_dist_f32(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    d0, d1, d2 = a[..., 0] - b[..., 0], a[..., 1] - b[..., 1], a[..., 2] - b[..., 2]
    return (d0 * d0 + d1 * d1) + d2 * d2


def project_match(frame_points: np.ndarray, H: int, W: int, query_points: np.ndarray, init: np.ndarray,
                  max_steps: int = 64, max_angle: float = 0.01) -> Tuple[np.ndarray, np.ndarray]:
    """(pixel of f or -1, final FP32 distance) for every query (see the reading above)."""
    rays = ray_image_f32(frame_points)
    q = ray_image_f32(query_points)
    Q = q.shape[0]
    cur = np.clip(np.asarray(init, dtype=np.int64), 0, H * W - 1)
    with np.errstate(invalid="ignore"):
        dcur = ray_dist_f32(rays[cur], q)
    dcur = np.where(np.isnan(dcur), np.float32(np.inf), dcur).astype(np.float32)
    active = np.isfinite(q).all(axis=1)
    for _ in range(max_steps):
        if not active.any():
            break
        y, x = cur // W, cur % W
        best = dcur.copy()
        bidx = cur.copy()
        for dy, dx in _NB8:
            ny, nx = y + dy, x + dx
            inside = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
            cand = np.where(inside, ny * W + nx, 0)
            with np.errstate(invalid="ignore"):
                d = ray_dist_f32(rays[cand], q)
            better = active & inside & (d < best)  # NaN compares false
            best = np.where(better, d, best)
            bidx = np.where(better, cand, bidx)
        moved = bidx != cur
        active = active & moved
        cur, dcur = bidx, best
    dmax = np.float32(2.0 - 2.0 * math.cos(max_angle))
    ok = np.isfinite(q).all(axis=1) & (dcur <= dmax)
    return np.where(ok, cur, -1).astype(np.int64), dcur


def fuse(canon: np.ndarray, pred: np.ndarray, T_kf: np.ndarray) -> np.ndarray:
    """Eq. (fusion): X_k <- (C_k X_k + C_f (T_kf X_f)) / (C_k + C_f), C_k <- C_k + C_f for
    every pixel, with canon = (X_k, C_k) and pred = (X^k_f in f's frame, C^k_f)."""
    ck = canon[:, 3:4].astype(np.float64)
    cf = pred[:, 3:4].astype(np.float64)
    Y = transform(T_kf, pred[:, :3].astype(np.float64))
    out = np.empty_like(canon, dtype=np.float64)
    out[:, :3] = (ck * canon[:, :3] + cf * Y) / (ck + cf)
    out[:, 3:4] = ck + cf
    return out


# =================================================================== error reports
def pose_errors(pa: np.ndarray, pb: np.ndarray, ref_scale: Optional[float] = None) -> Dict[str, float]:
    """Max over keyframes of rotation angle (rad), relative translation and relative scale error.

    Rotation error is the angle of R_a R_b^T, i.e. ||Log(R_a R_b^T)||, taken as
    atan2(sin, cos) of the relative rotation (sin from its skew part, cos from its trace),
    which keeps full relative accuracy at small and near-pi angles alike.  Translation
    error is ||t_a - t_b|| / max(||t_b||, ref), ref = RMS distance of the reference camera
    centres from their mean unless given.  Scale error is |s_a / s_b - 1|.
    """
    tb = pb[:, :3]
    ref = ref_scale if ref_scale is not None else float(np.sqrt(((tb - tb.mean(0)) ** 2).sum(1).mean()))
    rot, tra, sca = 0.0, 0.0, 0.0
    for a, b in zip(pa, pb):
        M = quat_to_rot(a[3:7]) @ quat_to_rot(b[3:7]).T
        sin_t = 0.5 * float(np.linalg.norm([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]))
        cos_t = 0.5 * (float(np.trace(M)) - 1.0)
        rot = max(rot, math.atan2(sin_t, cos_t))
        tra = max(tra, float(np.linalg.norm(a[:3] - b[:3]) / max(np.linalg.norm(b[:3]), ref, 1e-300)))
        sca = max(sca, abs(a[7] / b[7] - 1.0))
    return dict(rot=rot, trans=tra, scale=sca)
