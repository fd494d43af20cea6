"""The epsilon escalation of Eq. (normal) (Sec. III-D) with retries that succeed.

A factorisation attempt r uses eps_r = eps0 * 100^r; when a pivot is not > 0 or not
finite the attempt fails and the next one restarts from the undamped system.  To reach
attempt k on purpose, a test setting of the library, COMO3R_TEST_DIAG_SHIFT=<s0>,<s1>,...
(off unless set), lowers graph g's assembled diagonal by s_g before every solve.  With
H_r the oracle's system without the fixed keyframes, l its smallest eigenvalue and

    s = l + 10 eps_{k-1},

the damped matrix H_r - s I + eps_r I has smallest eigenvalue eps_r - 10 eps_{k-1}: at
most -9 eps_{k-1} for every r < k (the attempt must fail) and +90 eps_{k-1} at r = k (it
succeeds).  eps0 is set to a fixed fraction of ||H_r|| so that these margins stay far
above the rounding of either form.  The oracle's damped_solve on the same shifted H
decides the attempts and gives tau and the poses; the GPU must agree in all three solver
variants (one CTA per graph, one cluster per graph, one grid over all SMs), and in a
batch where only one graph is shifted.  Host-made input only: no fault, no trap.
"""
import numpy as np
import pytest

from oracle import como3r_oracle as O
from synth import make_problem, make_workload
from tests.gpu_helpers import oracle_dense_without_anchor, pose_err, rel_fro

FP64_TOL = 1e-9
MIXED_TOL = 1e-5
# eps0 as a fraction of the largest eigenvalue of H_r: the FP64 form rounds at ~1e-13 of
# ||H|| and the mixed form's H differs from the oracle's by ~1e-6 relative
EPS_FRAC = {"plain": 1e-7, "mixed": 1e-3}


def reduced_spectrum(prob, poses, graph):
    """(smallest, largest) eigenvalue of graph `graph`'s oracle H without its fixed keyframes."""
    H, _, _, _ = O.build_system(prob, poses, graph)
    fixed = set(O.component_anchors(prob, graph))
    keep = [k for k in range(H.shape[0]) if k // 7 not in fixed]
    ev = np.linalg.eigvalsh(H[np.ix_(keep, keep)])
    return float(ev[0]), float(ev[-1])


def shifted_problem(prob, eps_frac, k_by_graph):
    """A copy of `prob` with eps0 = eps_frac * max_g lambda_max, and the per-graph shifts that
    make graph g's first k attempts fail (k = 0: no shift)."""
    import copy
    specs = [reduced_spectrum(prob, prob.poses_init, g) for g in range(prob.num_graphs)]
    eps0 = eps_frac * max(hi for _, hi in specs)
    shifts = [0.0 if k == 0 else lo + 10.0 * eps0 * 100.0 ** (k - 1) for (lo, _), k in zip(specs, k_by_graph)]
    p = copy.copy(prob)
    p.eps0 = eps0
    return p, shifts


def oracle_shifted_iters(prob, poses, shifts, iters):
    """The oracle's iterations with graph g's H lowered by shifts[g] I before every solve;
    returns poses, the first iteration's (tau [N, 7], attempts per graph) and the cost trace."""
    arrs = O.problem_arrays(prob)
    first = None
    trace = np.zeros((iters + 1, prob.num_graphs))
    for it in range(iters):
        out = poses.copy()
        tau_all = np.zeros((prob.num_kf, 7))
        attempts = []
        for g in range(prob.num_graphs):
            k0 = int(prob.kf_offset[g])
            H, gv, cost, _ = O.build_system(prob, poses, g, arrs)
            tau, att, ok = O.damped_solve(H - shifts[g] * np.eye(H.shape[0]), gv, O.component_anchors(prob, g),
                                          prob.lam, prob.eps0, prob.max_attempts)
            assert ok
            tau_all[k0:k0 + tau.shape[0]] = tau
            attempts.append(att)
            trace[it, g] = cost
            out = O.retract(out, tau, k0)
        if first is None:
            first = (tau_all, attempts)
        poses = out
    trace[iters] = [O.build_system(prob, poses, g, arrs)[2] for g in range(prob.num_graphs)]
    return poses, first, trace


@pytest.fixture(scope="module")
def tiny():
    return make_workload("two_agent_6kf_64x48", seed=0)


@pytest.fixture(scope="module")
def batch3():
    return make_problem(22, agents=2, n_kf=4, H=24, W=32, f=25.0, n_inter=1, num_graphs=3, name="batch3")


@pytest.mark.parametrize("k", [1, 3, 5])
def test_oracle_shift_reaches_attempt_k(tiny, k):
    """CPU check of the construction itself: the oracle fails exactly the first k attempts."""
    p, shifts = shifted_problem(tiny, EPS_FRAC["plain"], [k])
    _, (tau, attempts), _ = oracle_shifted_iters(p, p.poses_init, shifts, 1)
    assert attempts == [k + 1]
    assert np.all(np.isfinite(tau)) and np.any(tau != 0)


# ------------------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30488_b300 import build
    build.build()
    from paper_2605_30488_b300 import como3r
    return como3r


def torch_poses(p):
    import torch
    return torch.tensor(p, dtype=torch.float64, device="cuda").contiguous()


VARIANTS = {"cta": dict(COMO3R_SOLVE_CLUSTER="0", COMO3R_SOLVE_GRID="0"),
            "cluster": dict(COMO3R_SOLVE_CLUSTER="4", COMO3R_SOLVE_GRID="0"),
            "grid": dict(COMO3R_SOLVE_CLUSTER="0", COMO3R_SOLVE_GRID="1"),
            # batches: one graph by a cluster of the CTA-group launch, or every graph
            "group1": dict(COMO3R_SOLVE_GROUPS="1"),
            "group3": dict(COMO3R_SOLVE_GROUPS="3")}


def set_variant(monkeypatch, variant, shifts):
    for k, v in VARIANTS[variant].items():
        monkeypatch.setenv(k, v)
    monkeypatch.setenv("COMO3R_TEST_DIAG_SHIFT", ",".join(repr(float(s)) for s in shifts))


def check_variant(C, g, variant):
    st = g.stats()
    ctas = st["solve_ctas"]
    if variant.startswith("group"):
        assert ctas == 8 and st["solve_groups"] == int(variant[5:]), (variant, st)
        return
    assert (ctas == 1) if variant == "cta" else (ctas == 4 if variant == "cluster" else ctas > 4), (variant, ctas)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", ["cta", "cluster", "grid"])
@pytest.mark.parametrize("k", [1, 3, 5])
def test_retry_succeeds_at_attempt_k_fp64(C, tiny, variant, k, monkeypatch):
    """Attempts r < k fail, attempt k succeeds: the GPU's attempt count, its shifted system,
    its step tau and the retracted poses equal the oracle's (1e-9), then three more
    iterations under the same shift follow the oracle's poses and cost trace."""
    import torch
    p, shifts = shifted_problem(tiny, EPS_FRAC["plain"], [k])
    set_variant(monkeypatch, variant, shifts)
    po1, (tau_o, att_o), _ = oracle_shifted_iters(p, p.poses_init, shifts, 1)
    assert att_o == [k + 1]
    N = p.num_kf
    H = torch.zeros((7 * N, 7 * N), dtype=torch.float64, device="cuda")
    gv = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
    poses = torch_poses(p.poses_init)
    with C.Graph(p, mode=C.PLAIN_FP64) as g:
        check_variant(C, g, variant)
        st, info = g.gn_step(poses, H, gv)
        tau = g.last_step()
        # the system the solver saw: the oracle's H with its diagonal lowered (fixed rows zero)
        Ho, go, _, _ = oracle_dense_without_anchor(p, p.poses_init)
        fixed = set(O.component_anchors(p, 0))
        for kk in range(N):
            if kk not in fixed:
                Ho[7 * kk:7 * kk + 7, 7 * kk:7 * kk + 7] -= shifts[0] * np.eye(7)
        assert rel_fro(H.cpu().numpy(), Ho) <= FP64_TOL
        assert info[0]["attempts"] == k + 1 and info[0]["solved"] and not (st & C.WARN_SOLVE_FAILED)
        assert rel_fro(tau, tau_o) <= FP64_TOL, rel_fro(tau, tau_o)
        assert max(pose_err(poses.cpu().numpy(), po1).values()) <= FP64_TOL
        st, trace, info = g.solve(poses, 3)
    po4, _, to = oracle_shifted_iters(p, po1, shifts, 3)
    assert max(pose_err(poses.cpu().numpy(), po4).values()) <= FP64_TOL
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)


@pytest.mark.gpu
def test_retry_succeeds_mixed(C, tiny, monkeypatch):
    """The same retry in the mixed form (FP32 residuals, FP64 solve): attempt 3 succeeds and
    the step matches the oracle's to the mixed tolerance."""
    p, shifts = shifted_problem(tiny, EPS_FRAC["mixed"], [3])
    set_variant(monkeypatch, "cta", shifts)
    po1, (tau_o, att_o), _ = oracle_shifted_iters(p, p.poses_init, shifts, 1)
    poses = torch_poses(p.poses_init)
    with C.Graph(p, mode=C.MIXED) as g:
        st, info = g.gn_step(poses)
        tau = g.last_step()
    assert info[0]["attempts"] == att_o[0] == 4 and info[0]["solved"]
    assert rel_fro(tau, tau_o) <= MIXED_TOL
    assert max(pose_err(poses.cpu().numpy(), po1).values()) <= MIXED_TOL


@pytest.mark.gpu
@pytest.mark.parametrize("variant", ["cta", "cluster", "group1", "group3"])
def test_retry_in_one_graph_of_a_batch(C, batch3, variant, monkeypatch):
    """Three graphs in one launch, only graph 1 shifted: graphs 0 and 2 solve at the first
    attempt, graph 1 at its fourth; every graph's step equals the oracle's."""
    p, shifts = shifted_problem(batch3, EPS_FRAC["plain"], [0, 3, 0])
    set_variant(monkeypatch, variant, shifts)
    po1, (tau_o, att_o), _ = oracle_shifted_iters(p, p.poses_init, shifts, 1)
    assert att_o == [1, 4, 1]
    poses = torch_poses(p.poses_init)
    with C.Graph(p, mode=C.PLAIN_FP64) as g:
        check_variant(C, g, variant)
        st, info = g.gn_step(poses)
        tau = g.last_step()
    assert [x["attempts"] for x in info] == att_o and all(x["solved"] for x in info)
    for gi in range(3):
        k0, k1 = int(p.kf_offset[gi]), int(p.kf_offset[gi + 1])
        assert rel_fro(tau[k0:k1], tau_o[k0:k1]) <= FP64_TOL, gi
    assert max(pose_err(poses.cpu().numpy(), po1).values()) <= FP64_TOL
