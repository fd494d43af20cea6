"""GPU parity: the CUDA library through its C ABI against the FP64 CPU oracle.

Tolerances (from the stated targets): the all-FP64 form matches the oracle to 1e-9
relative (Hessian / gradient Frobenius norm, per-edge blocks, cost, poses as rotation
angle / relative translation / relative scale); the mixed form matches to 1e-5 on the
Hessian and on converged poses.  Inputs are the same stored values on both sides
(FP16 / FP32 storage upcast exactly by the oracle).
"""
import dataclasses

import numpy as np
import pytest

from oracle import como3r_oracle as O
from synth import make_problem, make_workload
from tests.gpu_helpers import oracle_dense_without_anchor, pose_err, rel_fro

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-5


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
def tiny():
    return make_workload("two_agent_6kf_64x48", seed=0)


@pytest.fixture(scope="module")
def tiny_exact():
    return make_problem(3, noise=0.0, outlier=0.0, exact=True, name="noise-free")


@pytest.fixture(scope="module")
def mid():
    # 2 agents x 8 keyframes at 160x120 (19200 px: 3 work items per edge, ragged last one), FP32
    return make_problem(5, agents=2, n_kf=8, H=120, W=160, f=125.0, noise=0.01, conf="lognormal",
                        outlier=0.15, skip_max=4, n_inter=4, exact=False, dtype=np.float32, name="mid")


def pin_residual_kernel(monkeypatch):
    """Fix the residual kernel's autotuned launch configuration, work-item size and schedule
    weights, so that two graphs of one problem sum the per-match terms in the same grouping
    (bitwise comparisons of two solver variants)."""
    monkeypatch.setenv("COMO3R_K1_CFG", "1")
    monkeypatch.setenv("COMO3R_K1_CHUNK", "1024")
    monkeypatch.setenv("COMO3R_K1_WEIGHTS", "1,1")


def torch_poses(p):
    import torch
    return torch.tensor(p, dtype=torch.float64, device="cuda").contiguous()


def edge_records(C, g, poses):
    import torch
    rec = torch.zeros((g.E, C.EDGE_RECORD), dtype=torch.float64, device="cuda")
    st, cost = g.linearize(torch_poses(poses), rec)
    return st, cost, rec.cpu().numpy()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_edge_blocks_match_oracle(C, tiny, mid, mode):
    for prob in (tiny, mid):
        m = C.PLAIN_FP64 if mode == "plain" else C.MIXED
        with C.Graph(prob, mode=m) as g:
            st, cost, rec = edge_records(C, g, prob.poses_init)
        _, _, E, recs = O.build_system(prob, prob.poses_init, 0)
        tol = FP64_TOL if mode == "plain" else MIXED_TOL
        for e, r in enumerate(recs):
            Hg = rec[e, :49].reshape(7, 7)
            assert rel_fro(Hg, r["H_rel"]) <= tol, (prob.name, e)
            # g_rel is a sum with cancellation: compare against the scale of its terms (H-weighted)
            gscale = max(np.linalg.norm(r["g_rel"]), 1e-3 * np.sqrt(np.abs(np.diag(r["H_rel"])).max()))
            assert np.linalg.norm(rec[e, 49:56] - r["g_rel"]) <= (tol if mode == "plain" else 1e-4) * gscale
            assert abs(rec[e, 56] - r["cost"]) <= tol * max(r["cost"], 1e-300)
            assert rec[e, 57] == r["n_valid"] and rec[e, 58] == r["n_skipped"]
        assert abs(cost[0] - E) <= tol * E


def test_gn_step_system_and_poses_fp64(C, tiny, mid):
    import torch
    for prob in (tiny, mid):
        N = prob.num_kf
        H = torch.zeros((7 * N, 7 * N), dtype=torch.float64, device="cuda")
        gv = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
        poses = torch_poses(prob.poses_init)
        with C.Graph(prob, mode=C.PLAIN_FP64) as g:
            st, info = g.gn_step(poses, H, gv)
        Ho, go, Eo, _ = oracle_dense_without_anchor(prob, prob.poses_init)
        assert rel_fro(H.cpu().numpy(), Ho) <= FP64_TOL
        assert rel_fro(gv.cpu().numpy(), go) <= FP64_TOL
        new_o, infos = O.gn_step(prob, prob.poses_init)
        err = pose_err(poses.cpu().numpy(), new_o)
        assert max(err.values()) <= FP64_TOL, err
        assert info[0]["attempts"] == infos[0]["attempts"] and info[0]["solved"]
        assert abs(info[0]["cost"] - Eo) <= FP64_TOL * Eo


def test_solve_fp64_matches_oracle(C, tiny):
    poses = torch_poses(tiny.poses_init)
    with C.Graph(tiny, mode=C.PLAIN_FP64) as g:
        st, trace, info = g.solve(poses, tiny.iters)
    po, to = O.gn_solve(tiny, tiny.poses_init, tiny.iters)
    err = pose_err(poses.cpu().numpy(), po)
    assert max(err.values()) <= FP64_TOL, err
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)


def test_solve_mixed_matches_oracle(C, tiny, mid):
    for prob in (tiny, mid):
        poses = torch_poses(prob.poses_init)
        with C.Graph(prob, mode=C.MIXED) as g:
            st, trace, info = g.solve(poses, 15)
        po, to = O.gn_solve(prob, prob.poses_init, 15)
        err = pose_err(poses.cpu().numpy(), po)
        assert max(err.values()) <= MIXED_TOL, (prob.name, err)
        np.testing.assert_allclose(trace[-1], to[-1], rtol=MIXED_TOL)


def test_noise_free_recovery_gpu(C, tiny_exact):
    for mode, tol in ((C.PLAIN_FP64, 1e-10), (C.MIXED, 1e-5)):
        poses = torch_poses(tiny_exact.poses_init)
        with C.Graph(tiny_exact, mode=mode) as g:
            g.solve(poses, 10)
        err = pose_err(poses.cpu().numpy(), tiny_exact.poses_gt)
        assert max(err.values()) <= tol, (mode, err)


def test_fp16_storage_mixed(C):
    prob = make_problem(7, agents=2, n_kf=6, H=96, W=128, f=100.0, noise=0.01, conf="lognormal",
                        outlier=0.15, skip_max=2, n_inter=3, exact=False, dtype=np.float16, name="f16",
                        band=(0.2, 1.0))
    with C.Graph(prob, mode=C.MIXED) as g:
        st, cost, rec = edge_records(C, g, prob.poses_init)
    _, _, E, recs = O.build_system(prob, prob.poses_init, 0)
    for e, r in enumerate(recs):
        if r["n_valid"]:
            assert rel_fro(rec[e, :49].reshape(7, 7), r["H_rel"]) <= MIXED_TOL


def test_retract_matches_expm(C):
    import torch
    rng = np.random.default_rng(0)
    taus = [rng.normal(size=7) * s for s in (1.0, 0.3, 1e-2, 1e-4, 1e-7)]
    taus += [np.r_[rng.normal(size=3), 0, 0, 0, 0.0], np.r_[rng.normal(size=3), 1e-9, 0, 0, 0.3],
             np.r_[rng.normal(size=3), rng.normal(size=3), 0.0], np.zeros(7)]
    tau = np.array(taus)
    base = np.array([O.matrix_to_pose(O.exp_sim3(rng.normal(size=7) * 0.5)) for _ in taus])
    tt = torch.tensor(tau, device="cuda")
    pp = torch_poses(base)
    C.sim3_retract(tt, pp)
    torch.cuda.synchronize()
    got = pp.cpu().numpy()
    for k in range(len(taus)):
        want = O.exp_sim3(tau[k]) @ O.pose_to_matrix(base[k])
        np.testing.assert_allclose(O.pose_to_matrix(got[k]), want, rtol=0, atol=1e-13 * max(1, np.abs(want).max()))


def test_cost_trace_is_monotone_fp64(C, mid):
    poses = torch_poses(mid.poses_init)
    with C.Graph(mid, mode=C.PLAIN_FP64) as g:
        st, trace, info = g.solve(poses, 8)
    assert trace[-1, 0] < trace[0, 0]


def test_bad_match_index_rejected(C, tiny):
    import copy
    bad = copy.deepcopy(tiny)
    bad.match_idx = bad.match_idx.copy()
    bad.match_idx[17] = 64 * 48  # one past the last pixel of j
    with pytest.raises(C.Como3rError) as ei:
        C.Graph(bad, mode=C.MIXED)
    assert ei.value.code == C.ERR_INVALID_ARG


def test_zero_scale_pose_gives_zero_update(C, tiny):
    """A keyframe of scale 0 poisons its blocks (non-finite Ad): every attempt fails, update is zero."""
    p = tiny.poses_init.copy()
    p[3, 7] = 0.0
    poses = torch_poses(p)
    with C.Graph(tiny, mode=C.PLAIN_FP64) as g:
        st, info = g.gn_step(poses)
    assert st & C.WARN_SOLVE_FAILED
    assert info[0]["attempts"] == tiny.max_attempts and not info[0]["solved"]
    np.testing.assert_array_equal(poses.cpu().numpy(), p)


def test_host_pose_buffers_and_copy_inputs(C, tiny):
    """Poses may live in host memory and inputs may be copied from host memory (e2e path)."""
    import torch
    ph = torch.tensor(tiny.poses_init, dtype=torch.float64).pin_memory()
    with C.Graph(tiny, mode=C.PLAIN_FP64, copy_inputs=True) as g:
        st, trace, info = g.solve(ph, 3)
        g.update_inputs(torch.from_numpy(tiny.points).pin_memory(),
                        torch.from_numpy(tiny.match_idx).pin_memory())
    po, _ = O.gn_solve(tiny, tiny.poses_init, 3)
    assert max(pose_err(ph.numpy(), po).values()) <= FP64_TOL


def test_batched_graphs_match_individual(C):
    """Three independent graphs of different sizes in one handle equal three separate runs."""
    specs = [dict(agents=2, n_kf=5, H=48, W=64, f=50.0), dict(agents=1, n_kf=7, H=60, W=80, f=60.0),
             dict(agents=3, n_kf=4, H=48, W=64, f=50.0, n_inter=3)]
    batch = make_problem(21, noise=0.005, outlier=0.1, exact=True, graph_specs=specs, name="batch",
                         dtype=np.float32)
    poses = torch_poses(batch.poses_init)
    with C.Graph(batch, mode=C.PLAIN_FP64) as g:
        st, trace, info = g.solve(poses, 6)
    po, to = O.gn_solve(batch, batch.poses_init, 6)
    assert max(pose_err(poses.cpu().numpy(), po).values()) <= FP64_TOL
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)


@pytest.mark.parametrize("groups", ["1", "2", "3"])
def test_group_solve_matches_oracle(C, groups, monkeypatch):
    """A batch solved by one launch of CTA groups (COMO3R_SOLVE_GROUPS=k: the k slowest
    graphs each by a cluster of 8 CTAs with cluster barriers, the others each by one CTA,
    factors in global memory; a cluster-solved graph may take the other ordering): the
    oracle's FP64 poses and cost trace after six iterations."""
    specs = [dict(agents=2, n_kf=5, H=48, W=64, f=50.0), dict(agents=1, n_kf=7, H=60, W=80, f=60.0),
             dict(agents=3, n_kf=4, H=48, W=64, f=50.0, n_inter=3)]
    batch = make_problem(21, noise=0.005, outlier=0.1, exact=True, graph_specs=specs, name="batch",
                         dtype=np.float32)
    monkeypatch.setenv("COMO3R_SOLVE_GROUPS", groups)
    poses = torch_poses(batch.poses_init)
    with C.Graph(batch, mode=C.PLAIN_FP64) as g:
        st = g.stats()
        assert st["solve_groups"] == int(groups) and st["solve_ctas"] == 8, st
        st, trace, info = g.solve(poses, 6)
    assert all(x["solved"] for x in info)
    po, to = O.gn_solve(batch, batch.poses_init, 6)
    assert max(pose_err(poses.cpu().numpy(), po).values()) <= FP64_TOL
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)


@pytest.mark.parametrize("cfg", [0, 1, 2, 3, 4, 5, 6])
def test_every_residual_kernel_configuration(C, mid, tiny, cfg, monkeypatch):
    """Each launch configuration the autotuner may choose gives the oracle's edge blocks
    (mixed form on FP32 and FP16 storage; the FP64 form for the configurations that have
    one)."""
    monkeypatch.setenv("COMO3R_K1_CFG", str(cfg))
    mid16 = dataclasses.replace(mid, points=mid.points.astype(np.float16))
    cases = [(mid, C.MIXED, MIXED_TOL), (mid16, C.MIXED, MIXED_TOL)]
    cases += [(tiny, C.PLAIN_FP64, FP64_TOL)] if cfg in (0, 1, 4) else []
    for prob, mode, tol in cases:
        with C.Graph(prob, mode=mode) as g:
            st, cost, rec = edge_records(C, g, prob.poses_init)
            stats = g.stats()
            assert stats["block"] % 100 == cfg
            assert stats["k1_stalls"] == 0
        _, _, E, recs = O.build_system(prob, prob.poses_init, 0)
        for e, r in enumerate(recs):
            assert rel_fro(rec[e, :49].reshape(7, 7), r["H_rel"]) <= tol, (cfg, mode, e)
            assert abs(rec[e, 56] - r["cost"]) <= tol * r["cost"]
            assert rec[e, 57] == r["n_valid"] and rec[e, 58] == r["n_skipped"]


def test_lm_damping_matches_oracle(C, tiny):
    """lambda > 0 (the LM damping H + lambda diag(H) of the local and tracking solves):
    one FP64 step and a 5-iteration solve against the oracle."""
    p = dataclasses.replace(tiny, lam=0.05)
    poses = torch_poses(p.poses_init)
    with C.Graph(p, mode=C.PLAIN_FP64) as g:
        st, info = g.gn_step(poses)
    new_o, _ = O.gn_step(p, p.poses_init)
    assert max(pose_err(poses.cpu().numpy(), new_o).values()) <= FP64_TOL
    poses = torch_poses(p.poses_init)
    with C.Graph(p, mode=C.PLAIN_FP64) as g:
        st, trace, info = g.solve(poses, 5)
    po, to = O.gn_solve(p, p.poses_init, 5)
    assert max(pose_err(poses.cpu().numpy(), po).values()) <= FP64_TOL
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)


def test_batched_tracking(C):
    """Ray-range tracking of 12 frames (one per agent) against their keyframes in one
    launch: 12 one-edge graphs (the keyframe fixed, the frame's Sim(3) free), LM damped."""
    prob = make_problem(21, agents=1, n_kf=2, H=48, W=64, f=50.0, noise=0.005, outlier=0.1, exact=False,
                        num_graphs=12, name="tracking")
    prob = dataclasses.replace(prob, lam=0.01)
    assert prob.num_edges == 12 and prob.num_kf == 24
    for mode, tol in ((C.PLAIN_FP64, FP64_TOL), (C.MIXED, MIXED_TOL)):
        poses = torch_poses(prob.poses_init)
        with C.Graph(prob, mode=mode) as g:
            st, trace, info = g.solve(poses, 8)
        po, to = O.gn_solve(prob, prob.poses_init, 8)
        assert max(pose_err(poses.cpu().numpy(), po).values()) <= tol, mode
        assert all(x["solved"] for x in info)


@pytest.mark.parametrize("ctas", ["0", "4"])
def test_graphs_of_different_sizes_alive_together(C, tiny, mid, ctas, monkeypatch):
    """A graph created after a larger one plans less shared memory for its solver; the
    larger graph's solves (and vjp substitutions) still launch and give the oracle's steps."""
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", ctas)
    po, to = O.gn_solve(mid, mid.poses_init, 3)
    with C.Graph(mid, mode=C.PLAIN_FP64) as big:
        with C.Graph(tiny, mode=C.PLAIN_FP64) as small:
            assert big.stats()["solve_ctas"] == small.stats()["solve_ctas"] == max(int(ctas), 1)
            poses_s = torch_poses(tiny.poses_init)
            small.solve(poses_s, 2)
            poses = torch_poses(mid.poses_init)
            st, trace, info = big.solve(poses, 3)
            assert all(x["solved"] for x in info)
            st, gl, gc, loss = big.vjp(torch_poses(mid.poses_init), 2, C.VJP_UNROLLED)
            assert np.isfinite(gl.double().cpu().numpy()).all()
    assert max(pose_err(poses.cpu().numpy(), po).values()) <= FP64_TOL
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)


@pytest.mark.parametrize("ctas", [2, 4, 8, 16])
def test_multi_sm_solve_matches_oracle(C, tiny, mid, ctas, monkeypatch):
    """The multi-SM factorisation (one cluster of `ctas` CTAs per graph, columns spread over
    them) gives the oracle's FP64 steps and solves, alone and for a batch of graphs."""
    # the residual kernel's configuration is autotuned per graph by timing; pin it so that
    # the two graphs differ only in the solver
    pin_residual_kernel(monkeypatch)
    for prob in (tiny, mid):
        out = {}
        for c in (0, ctas):
            monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", str(c))
            poses = torch_poses(prob.poses_init)
            with C.Graph(prob, mode=C.PLAIN_FP64) as g:
                assert g.stats()["solve_ctas"] == max(c, 1)
                st, trace, info = g.solve(poses, 6)
            out[c] = (poses.cpu().numpy(), trace)
        # the same task order: bitwise the single-CTA result
        np.testing.assert_array_equal(out[ctas][0], out[0][0])
        np.testing.assert_array_equal(out[ctas][1], out[0][1])
    po, to = O.gn_solve(tiny, tiny.poses_init, 6)
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", str(ctas))
    poses = torch_poses(tiny.poses_init)
    with C.Graph(tiny, mode=C.PLAIN_FP64) as g:
        st, trace, info = g.solve(poses, 6)
    assert max(pose_err(poses.cpu().numpy(), po).values()) <= FP64_TOL
    np.testing.assert_allclose(trace, to, rtol=FP64_TOL)
    for v in ("COMO3R_K1_CFG", "COMO3R_K1_CHUNK", "COMO3R_K1_WEIGHTS"):  # the mixed batch: autotuned
        monkeypatch.delenv(v)
    # a batch of three 2-agent graphs at 64x48 (at 32x24 with one inter-agent edge the second
    # agent's gauge is so weakly tied that FP32 summation order alone moves the converged
    # poses by up to ~1.4e-5, depending on the residual kernel's configuration)
    batch = make_problem(22, agents=2, n_kf=4, H=48, W=64, f=50.0, n_inter=2, num_graphs=3, name="batch3-64x48")
    poses = torch_poses(batch.poses_init)
    with C.Graph(batch, mode=C.MIXED) as g:
        st, trace, info = g.solve(poses, 6)
    po, _ = O.gn_solve(batch, batch.poses_init, 6)
    assert max(pose_err(poses.cpu().numpy(), po).values()) <= MIXED_TOL


def test_multi_sm_solve_failure_gives_zero_update(C, tiny, monkeypatch):
    """Every attempt fails in the multi-SM solve too (all CTAs agree), and the update is zero."""
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", "4")
    p = tiny.poses_init.copy()
    p[3, 7] = 0.0
    poses = torch_poses(p)
    with C.Graph(tiny, mode=C.PLAIN_FP64) as g:
        st, info = g.gn_step(poses)
    assert st & C.WARN_SOLVE_FAILED
    assert info[0]["attempts"] == tiny.max_attempts and not info[0]["solved"]
    np.testing.assert_array_equal(poses.cpu().numpy(), p)


def test_grid_solve_matches_single_cta(C, tiny, mid, monkeypatch):
    """The grid-wide factorisation (the level task lists over every warp of one CTA per SM,
    a grid barrier between phases, the factor in global memory) is bitwise the single-CTA
    solve, and within FP64 tolerance of the oracle's."""
    pin_residual_kernel(monkeypatch)  # the same residual kernel schedule in both graphs
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", "0")
    res = {}
    for name, prob in (("tiny", tiny), ("mid", mid)):
        out = {}
        for grid in ("0", "1"):
            monkeypatch.setenv("COMO3R_SOLVE_GRID", grid)
            poses = torch_poses(prob.poses_init)
            with C.Graph(prob, mode=C.PLAIN_FP64) as g:
                assert (g.stats()["solve_ctas"] > 1) == (grid == "1")
                st, trace, info = g.solve(poses, 6)
            assert info[0]["solved"]
            out[grid] = (poses.cpu().numpy(), trace)
        np.testing.assert_array_equal(out["1"][0], out["0"][0])
        np.testing.assert_array_equal(out["1"][1], out["0"][1])
        res[name] = out["1"]
    po, to = O.gn_solve(tiny, tiny.poses_init, 6)
    assert max(pose_err(res["tiny"][0], po).values()) <= FP64_TOL
    np.testing.assert_allclose(res["tiny"][1], to, rtol=FP64_TOL)


@pytest.fixture(scope="module")
def wide_top():
    # 2 agents x 12 keyframes with skips up to 3 and 16 inter-agent edges: the top of its
    # elimination tree has a one-column level with five off-diagonal blocks (8 + 35 rows),
    # factored as a wide four-warp panel whose rows beyond 32 are solved afterwards
    return make_problem(5, agents=2, n_kf=12, H=24, W=32, f=25.0, n_inter=16, skip_max=3, name="wide-top")


def test_wide_panels_match_oracle_in_every_solver(C, wide_top, monkeypatch):
    """The wide four-warp panel gives the same factor in the one-CTA, cluster (4 and 8 CTAs)
    and grid-wide solves (bitwise: the same operations per entry in the same order) and the
    oracle's FP64 steps."""
    pin_residual_kernel(monkeypatch)
    out = {}
    for name, env in (("cta", dict(COMO3R_SOLVE_CLUSTER="0", COMO3R_SOLVE_GRID="0")),
                      ("cluster4", dict(COMO3R_SOLVE_CLUSTER="4", COMO3R_SOLVE_GRID="0")),
                      ("cluster8", dict(COMO3R_SOLVE_CLUSTER="8", COMO3R_SOLVE_GRID="0")),
                      ("grid", dict(COMO3R_SOLVE_CLUSTER="0", COMO3R_SOLVE_GRID="1"))):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        poses = torch_poses(wide_top.poses_init)
        with C.Graph(wide_top, mode=C.PLAIN_FP64) as g:
            st, trace, info = g.solve(poses, 5)
        assert all(x["solved"] for x in info), name
        out[name] = (poses.cpu().numpy(), trace)
    for name in ("cluster4", "cluster8", "grid"):
        np.testing.assert_array_equal(out[name][0], out["cta"][0])
        np.testing.assert_array_equal(out[name][1], out["cta"][1])
    po, to = O.gn_solve(wide_top, wide_top.poses_init, 5)
    assert max(pose_err(out["cta"][0], po).values()) <= FP64_TOL
    np.testing.assert_allclose(out["cta"][1], to, rtol=FP64_TOL)


def test_grid_solve_failure_gives_zero_update(C, tiny, monkeypatch):
    """Every attempt fails in the grid-wide solve too (all CTAs take the decision from the
    same flag after a grid barrier): the update is zero and the warning is set; the next
    call on the same graph starts from clean flags."""
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", "0")
    monkeypatch.setenv("COMO3R_SOLVE_GRID", "1")
    p = tiny.poses_init.copy()
    p[3, 7] = 0.0
    poses = torch_poses(p)
    with C.Graph(tiny, mode=C.PLAIN_FP64) as g:
        assert g.stats()["solve_ctas"] > 1
        st, info = g.gn_step(poses)
        poses2 = torch_poses(tiny.poses_init)
        st2, info2 = g.gn_step(poses2)
    assert st & C.WARN_SOLVE_FAILED
    assert info[0]["attempts"] == tiny.max_attempts and not info[0]["solved"]
    np.testing.assert_array_equal(poses.cpu().numpy(), p)
    assert info2[0]["solved"] and not (st2 & C.WARN_SOLVE_FAILED)


def test_grid_barrier_wait_limit(C, tiny, monkeypatch):
    """A grid barrier whose count nothing completes (a test setting expects one arrival that
    never comes) runs out its wait limit instead of hanging: every CTA leaves, the solve
    reports the zero update and its warning, and the poses are unchanged."""
    import time
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", "0")
    monkeypatch.setenv("COMO3R_SOLVE_GRID", "1")
    monkeypatch.setenv("COMO3R_GRID_BARRIER_EXTRA", "1")
    poses = torch_poses(tiny.poses_init)
    with C.Graph(tiny, mode=C.PLAIN_FP64) as g:
        assert g.stats()["solve_ctas"] > 1
        t0 = time.time()
        st, info = g.gn_step(poses)
        dt = time.time() - t0
    assert st & C.WARN_SOLVE_FAILED and not info[0]["solved"]
    np.testing.assert_array_equal(poses.cpu().numpy(), tiny.poses_init)
    assert dt < 60, dt


@pytest.mark.parametrize("ctas", [0, 4])
def test_solve_timestamps(C, ctas, monkeypatch):
    """Device-clock stamps of a call: start after the pose upload, each graph's end after
    it and inside the call's wall time; the last gn_step's stamps replace the solve's."""
    import time
    import torch
    monkeypatch.setenv("COMO3R_SOLVE_CLUSTER", str(ctas))
    batch = make_problem(22, agents=2, n_kf=4, H=24, W=32, f=25.0, n_inter=1, num_graphs=3, name="batch3")
    poses = torch_poses(batch.poses_init)
    with C.Graph(batch, mode=C.MIXED) as g:
        assert g.stats()["solve_ctas"] == max(ctas, 1)
        torch.cuda.synchronize()
        w0 = time.time_ns()
        g.solve(poses, 5)
        torch.cuda.synchronize()
        wall = time.time_ns() - w0
        t0, done = g.timestamps()
        assert t0 > 0 and done.shape == (3,)
        assert np.all(done > t0) and np.all(done - t0 <= wall)
        g.gn_step(poses)
        t1, done1 = g.timestamps()
        assert t1 > done.max() and np.all(done1 > t1)
