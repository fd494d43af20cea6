"""Writes the full-size oracle goldens (fullsize_*.txt beside this file).

Usage (from the repository root; the full-size ones take minutes to hours of CPU):
    python -m tests.golden.make_fullsize_goldens two_agent_6kf      (seconds)
    python -m tests.golden.make_fullsize_goldens two_agent_40kf
    python -m tests.golden.make_fullsize_goldens team_4x150_f16
    python -m tests.golden.make_fullsize_goldens adjoint_4x30 [--workers 6]

Every value written comes from `oracle/` (the FP64 CPU oracle) on the seeded inputs that
`tests/golden/fullsize.py` defines; nothing here touches the CUDA library.

two_agent_40kf (Eq. global, Eq. normal, Sec. III-D): the dense H and g of the initial
poses (fixed keyframes' rows and columns zero, as the library exports them; nonzero 7x7
blocks of the lower triangle only), and the poses and cost trace of 15 iterations.
team_4x150_f16: the per-edge blocks of 8 sampled edges at the initial poses, and the
poses and cost trace of 10 iterations, on the FP16-rounded inputs.
adjoint_4x30 (Sec. III-E, Eq. 8): the refined cost L = E(T^8(theta), theta) with theta =
per-pixel log-range and confidence:
  * its complex-step directional derivatives along two seeded dense directions, unrolled
    through the 8 iterations and at fixed T^8 (envelope);
  * for 64 seeded pixels (streamed pixels with a valid match), the envelope derivative
    w.r.t. the pixel's log-range and confidence (complex step over the edges that touch
    the pixel's keyframe: no other edge depends on it);
  * central differences of the unrolled L at step 1e-4: log-range for the first 32
    pixels, confidence for the other 32.  A pixel is excluded, and counted, when the +h
    and -h trajectories put any match it takes part in on different Huber branches
    (|r_c| <= kappa or not), since a central difference across the kink of the IRLS
    weight does not estimate the derivative;
  * the exact (complex-step) unrolled derivatives of four of those pixels, to measure
    the central differences' own error.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

from oracle import como3r_oracle as O
from tests.golden import fullsize as F

H_STEP = 1e-4
N_PIX = 64


def _header(name, prob, extra):
    return "\n".join([
        f"Full-size golden '{name}', written by tests/golden/make_fullsize_goldens.py from the FP64",
        "oracle only (oracle/como3r_oracle.py) on the seeded inputs of tests/golden/fullsize.py.",
        f"Inputs: {prob.name}, {prob.num_kf} keyframes, {prob.num_edges} edges, {prob.valid_matches()} valid matches,",
        f"storage {prob.points.dtype}.",
    ] + extra)


def _fp_entries(prob):
    return {"fp_" + k: v for k, v in F.fingerprint(prob).items()}


def dense_blocks(prob, poses):
    """Nonzero 7x7 blocks (r >= c) of the oracle's H with the fixed keyframes removed, and g."""
    H, g, E, _ = O.build_system(prob, poses, 0)
    for a in O.component_anchors(prob, 0):
        H[7 * a:7 * a + 7, :] = 0.0
        H[:, 7 * a:7 * a + 7] = 0.0
        g[7 * a:7 * a + 7] = 0.0
    N = prob.num_kf
    rc, blocks = [], []
    for r in range(N):
        for c in range(r + 1):
            b = H[7 * r:7 * r + 7, 7 * c:7 * c + 7]
            if np.any(b != 0.0):
                rc.append((r, c))
                blocks.append(b.ravel())
    return np.array(rc, dtype=np.float64), np.array(blocks), g, E, float(np.linalg.norm(H))


def make_two_agent_40kf():
    name = "two_agent_40kf"
    prob = F.problem(name)
    t0 = time.time()
    rc, blocks, g, E0, hnorm = dense_blocks(prob, prob.poses_init)
    poses, trace = O.gn_solve(prob, prob.poses_init, F.ITERS[name])
    ent = _fp_entries(prob)
    ent.update(H_block_rc=rc, H_blocks=blocks, H_fro=hnorm, g=g, cost_init=E0, poses=poses, trace=trace[:, 0])
    F.write(F.PATHS[name], _header(name, prob, [
        "H_block_rc / H_blocks: the dense H at the initial poses as nonzero 7x7 blocks (row kf, col kf), r >= c;",
        "H_fro: its Frobenius norm (both triangles); g: the gradient (fixed keyframes zero).",
        f"poses / trace: {F.ITERS[name]} Gauss-Newton iterations from the initial poses (trace[k] = cost before",
        f"iteration k, trace[{F.ITERS[name]}] after the last). CPU time {time.time() - t0:.0f} s."]), ent)


def make_two_agent_6kf():
    name = "two_agent_6kf"
    prob = F.problem(name)
    t0 = time.time()
    poses, trace = O.gn_solve(prob, prob.poses_init, F.ITERS[name])
    ent = _fp_entries(prob)
    ent.update(poses=poses, trace=trace[:, 0])
    F.write(F.PATHS[name], _header(name, prob, [
        f"poses / trace: {F.ITERS[name]} Gauss-Newton iterations from the initial poses (trace[k] = cost before",
        f"iteration k, trace[{F.ITERS[name]}] after the last). CPU time {time.time() - t0:.1f} s."]), ent)


def make_team_4x150_f16():
    name = "team_4x150_f16"
    prob = F.problem(name)
    t0 = time.time()
    arrs = O.problem_arrays(prob)
    T = [O.pose_to_matrix(p) for p in prob.poses_init]
    sample = np.linspace(0, prob.num_edges - 1, 8).astype(int)
    recs = []
    for e in sample:
        i, j, m, n, Pi, Pj = O.edge_matches(prob, arrs, int(e))
        r = O.linearize_edge(T[i], T[j], Pi, Pj, prob.params())
        recs.append(np.concatenate([r["H_rel"].ravel(), r["g_rel"], [r["cost"], r["n_valid"], r["n_skipped"]]]))
    del arrs
    poses, trace = O.gn_solve(prob, prob.poses_init, F.ITERS[name])
    ent = _fp_entries(prob)
    ent.update(edge_sample=sample.astype(np.float64), edge_records=np.array(recs), poses=poses, trace=trace[:, 0])
    F.write(F.PATHS[name], _header(name, prob, [
        "edge_sample / edge_records: per sampled edge at the initial poses, H_rel (49), g_rel (7), cost,",
        "valid and skipped match counts.",
        f"poses / trace: {F.ITERS[name]} Gauss-Newton iterations (mixed-form inputs: the FP16 values upcast).",
        f"CPU time {time.time() - t0:.0f} s."]), ent)


# ------------------------------------------------------------------ adjoint_4x30
def seeded_direction(seed, n):
    rng = np.random.default_rng(seed)
    return rng.normal(size=n), rng.normal(size=n)


def seeded_pixels(prob):
    """64 seeded streamed pixels (global pixel ids) that have a valid match."""
    rng = np.random.default_rng(2024)
    pix_off, idx_off = prob.pix_offset(), prob.idx_offset()
    out = []
    edges = rng.permutation(prob.num_edges)
    k = 0
    while len(out) < N_PIX:
        e = int(edges[k % prob.num_edges])
        k += 1
        idx = prob.match_idx[idx_off[e]:idx_off[e + 1]]
        m = np.nonzero(idx >= 0)[0]
        if m.size == 0:
            continue
        p = int(pix_off[prob.edge_i[e]] + m[rng.integers(m.size)])
        if p not in out:
            out.append(p)
    return np.array(out, dtype=np.int64)


def _touching_edges(prob, p):
    pix_off = prob.pix_offset()
    k = int(np.searchsorted(pix_off, p, side="right") - 1)
    return k, [e for e in range(prob.num_edges) if prob.edge_i[e] == k or prob.edge_j[e] == k]


def envelope_pixel(prob, T, p, which, h=1e-30):
    """d/d theta_p of sum_e cost_e(T, theta) at fixed T by the complex step (only the edges
    touching the pixel's keyframe depend on it)."""
    _, edges = _touching_edges(prob, p)
    d = np.zeros(prob.points.shape[0], dtype=np.complex128)
    d[p] = 1j * h
    pts = O.reparameterised_points(prob, d if which == "log" else None, d if which == "conf" else None)
    arrs = dict(O.problem_arrays(prob), points=pts)
    tot = 0.0
    for e in edges:
        i, j, m, n, Pi, Pj = O.edge_matches(prob, arrs, e)
        tot += np.imag(O.linearize_edge(T[i], T[j], Pi, Pj, prob.params())["cost"]) / h
    return float(tot)


def _branches(prob, T, arrs, p):
    """Huber branch (|r_c| <= kappa) of every residual component of the matches pixel p
    takes part in (streamed or gathered), in a fixed order."""
    k, edges = _touching_edges(prob, p)
    pix_off = prob.pix_offset()
    prm = prob.params()
    out = []
    for e in edges:
        i, j, m, n, Pi, Pj = O.edge_matches(prob, arrs, e)
        sel = (pix_off[i] + m == p) | (pix_off[j] + n == p)
        if not np.any(sel):
            continue
        Tij = O.sim3_inverse(T[i]) @ T[j]
        ev, _ = O.residual(Tij, Pi[sel, :3], Pj[sel, :3])
        r = O.whiten(ev, np.sqrt(np.maximum(Pi[sel, 3] * Pj[sel, 3], 0.0)), prm["sigma_ray"], prm["sigma_dist"])
        out.append(np.abs(r) <= prm["huber_k"])
    return np.concatenate([b.ravel() for b in out]) if out else np.zeros(0, bool)


_PROB = None


def _worker_init():
    """Worker processes load the inputs once (from the generator's cache the parent filled)."""
    global _PROB
    _PROB = F.problem("adjoint_4x30")


def _fd_task(args):
    """Central difference of the unrolled refined cost along one pixel parameter."""
    p, which = args
    prob = _PROB
    iters = F.ITERS["adjoint_4x30"]
    vals, br = [], []
    for sgn in (1.0, -1.0):
        d = np.zeros(prob.points.shape[0])
        d[p] = sgn * H_STEP
        pts = O.reparameterised_points(prob, d if which == "log" else None, d if which == "conf" else None)
        arrs = dict(O.problem_arrays(prob), points=pts)
        T = O.gn_trajectory(prob, prob.poses_init, iters, arrs)
        vals.append(sum(O.build_system(prob, None, g, arrs, T_global=T)[2] for g in range(prob.num_graphs)))
        br.append(_branches(prob, T, arrs, p))
    crossed = br[0].shape != br[1].shape or bool(np.any(br[0] != br[1]))
    return (vals[0] - vals[1]) / (2 * H_STEP), crossed


def _exact_task(args):
    p, which = args
    prob = _PROB
    v = np.zeros(prob.points.shape[0])
    v[p] = 1.0
    return O.refined_cost_derivative(prob, prob.poses_init, F.ITERS["adjoint_4x30"],
                                     v if which == "log" else None, v if which == "conf" else None)


def _dir_task(args):
    seed, envelope = args
    prob = _PROB
    vl, vc = seeded_direction(seed, prob.points.shape[0])
    return O.refined_cost_derivative(prob, prob.poses_init, F.ITERS["adjoint_4x30"], vl, vc, envelope=envelope)


def make_adjoint_4x30(workers: int):
    name = "adjoint_4x30"
    # the ray-cast generator runs once; the workers read its cached arrays (and use one
    # BLAS thread each)
    os.environ.setdefault("COMO3R_SYNTH_CACHE", tempfile.mkdtemp(prefix="como3r_golden_"))
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = os.environ["MKL_NUM_THREADS"] = "1"
    prob = F.problem(name)
    iters = F.ITERS[name]
    t0 = time.time()
    pix = seeded_pixels(prob)
    which = ["log"] * (N_PIX // 2) + ["conf"] * (N_PIX // 2)
    exact_idx = [0, 1, N_PIX // 2, N_PIX // 2 + 1]
    tasks_fd = list(zip(pix.tolist(), which))
    dir_tasks = [(1, False), (2, False), (1, True), (2, True)]
    exact_tasks = [tasks_fd[k] for k in exact_idx]

    def local():
        # the trajectory, the loss and the envelope pixel derivatives, in this process
        arrs = O.problem_arrays(prob)
        T = O.gn_trajectory(prob, prob.poses_init, iters, arrs)
        L = sum(O.build_system(prob, None, g, arrs, T_global=T)[2] for g in range(prob.num_graphs))
        env = np.array([[envelope_pixel(prob, T, int(p), "log"), envelope_pixel(prob, T, int(p), "conf")]
                        for p in pix])
        poses, trace = O.gn_solve(prob, prob.poses_init, iters)
        return L, env, poses, trace

    if workers <= 1:
        global _PROB
        _PROB = prob
        dirs = np.array([_dir_task(t) for t in dir_tasks])
        exact = np.array([_exact_task(t) for t in exact_tasks])
        fd = [_fd_task(t) for t in tasks_fd]
        L, env, poses, trace = local()
    else:
        with mp.get_context("spawn").Pool(workers, initializer=_worker_init) as pool:
            r_dir = pool.map_async(_dir_task, dir_tasks, chunksize=1)
            r_exact = pool.map_async(_exact_task, exact_tasks, chunksize=1)
            r_fd = pool.map_async(_fd_task, tasks_fd, chunksize=1)
            L, env, poses, trace = local()
            dirs = np.array(r_dir.get())
            exact = np.array(r_exact.get())
            fd = r_fd.get()
    fd_val = np.array([v for v, _ in fd])
    crossed = np.array([c for _, c in fd], dtype=np.float64)
    ent = _fp_entries(prob)
    ent.update(loss=L, trace=trace[:, 0], poses=poses, dir_seeds=np.array([1.0, 2.0]),
               dir_unrolled=dirs[:2], dir_envelope=dirs[2:], pixels=pix.astype(np.float64),
               fd_which=np.array([0.0 if w == "log" else 1.0 for w in which]), fd=fd_val, fd_excluded=crossed,
               envelope=env, exact_idx=np.array(exact_idx, dtype=np.float64), exact=exact)
    F.write(F.PATHS[name], _header(name, prob, [
        f"loss: refined cost after {iters} iterations; trace / poses: those iterations.",
        "dir_unrolled / dir_envelope: complex-step derivative along the seeded direction (vlog, vconf) =",
        "np.random.default_rng(seed).normal(size=P) twice, for seeds dir_seeds (unrolled; at fixed T^8).",
        "pixels: global pixel ids; envelope [64, 2]: d/d log-range, d/d confidence at fixed T^8.",
        f"fd: central difference (step {H_STEP}) of the unrolled loss along log-range (fd_which 0) or",
        "confidence (1) of each pixel; fd_excluded 1 where the +h / -h trajectories put a match of the",
        f"pixel on different Huber branches ({int(crossed.sum())} of {N_PIX} excluded).",
        "exact: complex-step unrolled derivative of the pixels at exact_idx (same parameter as fd).",
        f"CPU time {time.time() - t0:.0f} s with {workers} worker processes."]), ent)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=list(F.PATHS))
    ap.add_argument("--workers", type=int, default=6)
    a = ap.parse_args(argv)
    if a.which == "two_agent_40kf":
        make_two_agent_40kf()
    elif a.which == "two_agent_6kf":
        make_two_agent_6kf()
    elif a.which == "team_4x150_f16":
        make_team_4x150_f16()
    else:
        make_adjoint_4x30(a.workers)


if __name__ == "__main__":
    sys.exit(main())
