"""Full-size parity against the FP64 oracle, through stored oracle goldens.

The oracle needs minutes to hours per full-size workload, so its results were written
once by `tests/golden/make_fullsize_goldens.py` (oracle calls only) and are read here;
the inputs are regenerated from their seeds and checked against the stored fingerprint
first.  Tolerances are the stated targets: the all-FP64 form within 1e-9 relative of the
oracle (Hessian and gradient Frobenius norms, cost trace, poses as rotation angle /
relative translation / relative scale); the mixed form within 1e-5 on the Hessian and on
the poses after the iterations.  Gradients of the refined cost (Sec. III-E) come out of
the library rounded to FP32, so directional values are compared at 1e-6 relative (to the
sum of the terms' magnitudes) in the FP64 form.  On the 4 x 30 adjoint workload the mixed form is checked through
the envelope gradient only: its 8 IRLS iterations are far from converged and the unrolled
derivative through them amplifies the FP32 trajectory's 1e-7..1e-6 relative pose error to
O(1) changes, so the mixed unrolled gradient there is not an estimate of the FP64 one (the
unrolled mixed gradient is compared with the oracle on the small and mid problems).
"""
import os

import numpy as np
import pytest

from tests.golden import fullsize as F
from tests.gpu_helpers import pose_err, rel_fro

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-5
GRAD_TOL = 1e-6     # FP64 form: FP32 rounding of the exported gradients
MIXED_GRAD_TOL = 1e-5


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30488_b300 import build
    build.build()
    from paper_2605_30488_b300 import como3r
    return como3r


def dev(a):
    import torch
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda").contiguous()


def dense_from_blocks(gold, N):
    H = np.zeros((7 * N, 7 * N))
    for (r, c), b in zip(gold["H_block_rc"].astype(int), gold["H_blocks"]):
        H[7 * r:7 * r + 7, 7 * c:7 * c + 7] = b.reshape(7, 7)
        if r != c:
            H[7 * c:7 * c + 7, 7 * r:7 * r + 7] = b.reshape(7, 7).T
    return H


# ------------------------------------------------------------- 2 agents x 40 keyframes
@pytest.fixture(scope="module")
def two_agent():
    if not os.path.exists(F.PATHS["two_agent_40kf"]):
        pytest.skip("golden two_agent_40kf not written yet")
    p = F.problem("two_agent_40kf")
    gold = F.load("two_agent_40kf")
    F.check_fingerprint(p, gold)
    return p, gold


@pytest.mark.parametrize("mode_name", ["plain", "mixed"])
def test_two_agent_40kf_system_matches_oracle(C, two_agent, mode_name):
    """The assembled H and g at the initial poses (Eq. global, Sec. III-D)."""
    import torch
    p, gold = two_agent
    N = p.num_kf
    Ho = dense_from_blocks(gold, N)
    assert abs(np.linalg.norm(Ho) / gold["H_fro"][0] - 1) <= 1e-12  # the golden's own consistency
    H = torch.zeros((7 * N, 7 * N), dtype=torch.float64, device="cuda")
    gv = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
    mode = C.PLAIN_FP64 if mode_name == "plain" else C.MIXED
    with C.Graph(p, mode=mode) as g:
        st, info = g.gn_step(dev(p.poses_init), H, gv)
    tol = FP64_TOL if mode_name == "plain" else MIXED_TOL
    assert rel_fro(H.cpu().numpy(), Ho) <= tol
    assert rel_fro(gv.cpu().numpy(), gold["g"]) <= (FP64_TOL if mode_name == "plain" else 1e-4)
    assert abs(info[0]["cost"] / gold["cost_init"][0] - 1) <= tol


@pytest.mark.parametrize("mode_name", ["plain", "mixed"])
def test_two_agent_40kf_iterations_match_oracle(C, two_agent, mode_name):
    """15 Gauss-Newton iterations from the initial poses: poses and cost trace."""
    p, gold = two_agent
    mode = C.PLAIN_FP64 if mode_name == "plain" else C.MIXED
    poses = dev(p.poses_init)
    with C.Graph(p, mode=mode) as g:
        st, trace, info = g.solve(poses, F.ITERS["two_agent_40kf"])
    err = pose_err(poses.cpu().numpy(), gold["poses"])
    tol = FP64_TOL if mode_name == "plain" else MIXED_TOL
    assert max(err.values()) <= tol, err
    if mode_name == "plain":
        np.testing.assert_allclose(trace[:, 0], gold["trace"], rtol=FP64_TOL)
    else:
        assert abs(trace[-1, 0] / gold["trace"][-1] - 1) <= MIXED_TOL


# ----------------------------------------------- 4 agents x 150 keyframes, FP16 storage
@pytest.fixture(scope="module")
def team():
    if not os.path.exists(F.PATHS["team_4x150_f16"]):
        pytest.skip("golden team_4x150_f16 not written yet")
    p = F.problem("team_4x150_f16")
    gold = F.load("team_4x150_f16")
    F.check_fingerprint(p, gold)
    return p, gold


@pytest.mark.parametrize("mode_name", ["plain", "mixed"])
def test_team_4x150_f16_matches_oracle(C, team, mode_name):
    """Sampled per-edge blocks at the initial poses, then 10 iterations (one persistent
    residual launch per iteration, replayed as a CUDA graph), on the FP16-stored inputs
    with per-edge band masks: poses and final cost against the oracle's."""
    import torch
    p, gold = team
    mode = C.PLAIN_FP64 if mode_name == "plain" else C.MIXED
    tol = FP64_TOL if mode_name == "plain" else MIXED_TOL
    poses = dev(p.poses_init)
    with C.Graph(p, mode=mode) as g:
        rec = torch.zeros((g.E, C.EDGE_RECORD), dtype=torch.float64, device="cuda")
        g.linearize(poses, rec)
        rec = rec.cpu().numpy()
        for e, r in zip(gold["edge_sample"].astype(int), gold["edge_records"]):
            assert rel_fro(rec[e, :49], r[:49]) <= tol, e
            assert abs(rec[e, 56] / r[56] - 1) <= tol, e
            assert rec[e, 57] == r[57] and rec[e, 58] == r[58], e
        st, trace, info = g.solve(poses, F.ITERS["team_4x150_f16"])
    err = pose_err(poses.cpu().numpy(), gold["poses"])
    assert max(err.values()) <= tol, err
    assert abs(trace[-1, 0] / gold["trace"][-1] - 1) <= tol


# ------------------------------------------------- adjoint: 4 agents x 30 keyframes
@pytest.fixture(scope="module")
def adjoint():
    if not os.path.exists(F.PATHS["adjoint_4x30"]):
        pytest.skip("golden adjoint_4x30 not written yet")
    p = F.problem("adjoint_4x30")
    gold = F.load("adjoint_4x30")
    F.check_fingerprint(p, gold)
    return p, gold


def vjp(C, p, mode, vjp_mode):
    g = C.Graph(p, mode=mode)
    st, gl, gc, loss = g.vjp(dev(p.poses_init), F.ITERS["adjoint_4x30"], vjp_mode)
    out = gl.double().cpu().numpy(), gc.double().cpu().numpy(), float(loss.sum())
    g.close()
    return out


def directions(seed, n):
    rng = np.random.default_rng(int(seed))
    return rng.normal(size=n), rng.normal(size=n)


def test_adjoint_4x30_unrolled_fp64_matches_oracle(C, adjoint):
    """The FP64 unrolled gradient through 8 iterations: the loss, the complex-step
    directional derivatives along two seeded dense directions, the complex-step derivative
    of four single pixels, and the central differences (step 1e-4) of the 64 seeded pixels
    that cross no Huber kink, within the central differences' own error."""
    p, gold = adjoint
    gl, gc, loss = vjp(C, p, C.PLAIN_FP64, C.VJP_UNROLLED)
    assert abs(loss / gold["loss"][0] - 1) <= FP64_TOL
    for seed, ref in zip(gold["dir_seeds"], gold["dir_unrolled"]):
        vl, vc = directions(seed, gl.size)
        got = float(gl @ vl + gc @ vc)
        mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
        assert abs(got - ref) <= GRAD_TOL * mag, (seed, got, ref, mag)
    pix = gold["pixels"].astype(np.int64)
    g_at = np.where(gold["fd_which"] == 0, gl[pix], gc[pix])
    scale = np.abs(g_at).max()
    for k, ex in zip(gold["exact_idx"].astype(int), gold["exact"]):
        assert abs(g_at[k] - ex) <= GRAD_TOL * max(abs(ex), 1e-3 * scale), (k, g_at[k], ex)
    # central differences: their error, measured where the exact value is known, bounds the
    # comparison (truncation and the rounding of the FP64 cost divided by 2h)
    ex_idx = gold["exact_idx"].astype(int)
    fd_err = np.abs(gold["fd"][ex_idx] - gold["exact"]).max()
    keep = gold["fd_excluded"] == 0
    assert keep.sum() >= 48, keep.sum()
    bad = np.abs(g_at - gold["fd"]) > 4 * fd_err + 1e-6 * np.abs(gold["fd"])
    assert not np.any(bad & keep), (np.nonzero(bad & keep)[0], fd_err)
    # On this workload the central differences are noise-dominated (the 8 unconverged IRLS
    # iterations amplify the rounding of the FP64 cost: ~170 RMS against derivatives of
    # 0.05..2000), so also as a whole: their differences from the library's gradient have
    # the spread of their own noise measured at the exact pixels, which a missing, halved
    # or sign-flipped gradient exceeds (~350, ~220, ~660 here)
    noise = np.sqrt(np.mean((gold["fd"][ex_idx] - gold["exact"]) ** 2))
    spread = np.sqrt(np.mean((g_at - gold["fd"])[keep] ** 2))
    assert spread <= 1.25 * noise, (spread, noise)


# Per-pixel envelope derivatives, compared relative to the largest of the 64 of the same
# quantity: (FP64) the envelope is taken at the library's own T^8, which differs from the
# oracle's by the rounding of 8 unconverged IRLS iterations (the refined cost by ~2e-10
# relative), and a pixel whose terms cancel to 1/300 of that scale sees it at ~1e-5 of its
# own value; (mixed) a ray residual is the difference of two nearly equal unit directions,
# so its FP32 rounding error relative to itself is ~u32 / |r|, up to ~1e-3 for the small
# residuals of well-matched pixels, which a per-pixel derivative inherits (dense
# directional sums average it out and are held to the mixed form's 1e-5).
PIXEL_TOL = {"plain": GRAD_TOL, "mixed": 1e-3}


@pytest.mark.parametrize("mode_name", ["plain", "mixed"])
def test_adjoint_4x30_envelope_matches_oracle(C, adjoint, mode_name):
    """The envelope gradient (partial derivative at fixed T^8) of the 64 seeded pixels and
    along the two seeded directions, against the oracle's complex step."""
    p, gold = adjoint
    mode = C.PLAIN_FP64 if mode_name == "plain" else C.MIXED
    tol = GRAD_TOL if mode_name == "plain" else MIXED_GRAD_TOL
    gl, gc, loss = vjp(C, p, mode, C.VJP_ENVELOPE)
    assert abs(loss / gold["loss"][0] - 1) <= (FP64_TOL if mode_name == "plain" else MIXED_TOL)
    pix = gold["pixels"].astype(np.int64)
    env = gold["envelope"]
    sl, sc = np.abs(env[:, 0]).max(), np.abs(env[:, 1]).max()
    ptol = PIXEL_TOL[mode_name]
    for k, q in enumerate(pix):
        assert abs(gl[q] - env[k, 0]) <= ptol * sl, (k, gl[q], env[k, 0], sl)
        assert abs(gc[q] - env[k, 1]) <= ptol * sc, (k, gc[q], env[k, 1], sc)
    for seed, ref in zip(gold["dir_seeds"], gold["dir_envelope"]):
        vl, vc = directions(seed, gl.size)
        got = float(gl @ vl + gc @ vc)
        mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
        assert abs(got - ref) <= tol * mag, (seed, got, ref, mag)

