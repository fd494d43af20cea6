"""Shared-canvas graphs: exact dense correspondences for any edge topology, generated fast.

Used for the workloads that ray casting makes too slow to generate (long chains with
loop closures, 4 x 150 keyframe teams, batches of dozens of graphs).  Recipe (one
``numpy.random.Generator(PCG64(seed))``):

* World: a canvas of Hc x Wc world points around the origin.  Canvas cell (a, b) holds
  the point at direction (azimuth, elevation) = ((b / Wc - 1/2) * 200 deg,
  (a / Hc - 1/2) * 100 deg) and distance 8 m + 2 m * (smooth field in a, b), i.e. a
  panorama-like smooth surface seen from inside.
* Cameras: keyframe k of agent g sits within 1.5 m of the origin (a smooth path per
  agent) with a smooth rotation, gauge scale s_g ~ U[0.5, 2] per agent.
* Views: keyframe k sees the H x W window of the canvas starting at cell o_k, which moves
  along a smooth closed path of period ``period`` keyframes (so keyframes k and
  k - period share their window); pixel (v, u) of k holds the canvas point
  (v + o_k.row, u + o_k.col) expressed in k's camera frame and divided by s_g.
* Edge (i, j): pixel m = (v, u) of i is matched to the pixel of j that holds the same
  canvas point, (v + o_i.row - o_j.row, u + o_i.col - o_j.col), if it lies inside j's
  window, else -1; so matched pixels are the same world point (the residual vanishes at
  ground truth) and the matches form a shifted, coherent gather with a non-overlap band.
* Edges: sequential (k, k+1), covisibility (k, k+2) for even k, loop closures
  (k, k - loop) for k = loop, 2 loop, ..., and for teams ``n_inter`` inter-agent pairs
  with the most shared canvas cells (each agent linked to an earlier one first); with
  ``reverse_inter`` the inter-agent pairs are listed again in the other direction (the
  two decoded directions of a cross-agent candidate).
* Noise, outliers and confidences as in the ray-cast scenes: points scaled along their
  ray by (1 + noise N(0,1)), a fraction ``outlier`` of each edge's matches redirected to
  a uniformly drawn pixel of j, confidences lognormal(1, 0.5).  With ``band = (lo, hi)``
  each edge keeps only the matches of a column band of i covering a fraction U[lo, hi]
  of the image width at a uniformly drawn position (uneven per-edge valid counts).
* Initial poses: ground truth with a body-frame perturbation (rotation ``pert_rot``,
  offset ``pert_trans``, scale ``pert_scale`` or its inverse); anchors unperturbed.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

from .scene import Problem, _axis_angle, quat_from_matrix


def _smooth_field(rng, Hc: int, Wc: int) -> np.ndarray:
    """Sum of a few random low-frequency sinusoids in [-1, 1]."""
    a = np.arange(Hc)[:, None] / Hc
    b = np.arange(Wc)[None, :] / Wc
    f = np.zeros((Hc, Wc))
    for _ in range(4):
        ka, kb = rng.uniform(0.5, 3.0, size=2)
        pa, pb = rng.uniform(0, 2 * math.pi, size=2)
        f += np.sin(2 * math.pi * ka * a + pa) * np.cos(2 * math.pi * kb * b + pb)
    return f / 4.0


def _canvas(rng, Hc: int, Wc: int) -> np.ndarray:
    az = (np.arange(Wc) / Wc - 0.5) * math.radians(200.0)
    el = (np.arange(Hc) / Hc - 0.5) * math.radians(100.0)
    d = 8.0 + 2.0 * _smooth_field(rng, Hc, Wc)
    ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
    dirs = np.stack([ce * np.cos(az)[None, :], ce * np.sin(az)[None, :], np.broadcast_to(se, (Hc, Wc))], axis=-1)
    return dirs * d[..., None]


def _graph(rng, *, agents: int, n_kf: int, H: int, W: int, period: int, shift: int, loop: int, n_inter: int,
           noise: float, outlier: float, pert_rot: float, pert_trans: float, pert_scale: float, kf_base: int,
           dtype=np.float32, reverse_inter: bool = False, band: Optional[Sequence[float]] = None):
    Hc, Wc = H + 2 * shift + 2, W + 2 * shift + 2
    world = _canvas(rng, Hc, Wc).reshape(-1, 3)
    N = agents * n_kf
    P = H * W
    scale = rng.uniform(0.5, 2.0, size=agents)
    agent_of = np.repeat(np.arange(agents), n_kf).astype(np.int32)
    # window origins: a smooth closed path per agent (period keyframes), inside the canvas
    orig = np.zeros((N, 2), dtype=np.int64)
    Rs, cs = [], []
    for g in range(agents):
        ph = rng.uniform(0, 2 * math.pi)
        ph_cam = rng.uniform(0, 2 * math.pi)
        for k in range(n_kf):
            t = 2 * math.pi * k / period + ph
            orig[g * n_kf + k] = (int(round(shift * (1 + math.sin(t)))), int(round(shift * (1 + math.cos(t)))))
            tc = 2 * math.pi * k / period + ph_cam
            cs.append(np.array([1.2 * math.cos(tc), 1.2 * math.sin(tc), 0.3 * math.sin(2 * tc)]))
            yaw = 0.4 * math.sin(tc) + g * 0.3
            pitch = 0.1 * math.cos(tc)
            Rz = np.array([[math.cos(yaw), -math.sin(yaw), 0], [math.sin(yaw), math.cos(yaw), 0], [0, 0, 1]])
            Ry = np.array([[math.cos(pitch), 0, math.sin(pitch)], [0, 1, 0], [-math.sin(pitch), 0, math.cos(pitch)]])
            Rs.append(Rz @ Ry)
    rows = np.arange(P) // W
    cols = np.arange(P) % W
    # pointmaps
    pts = np.zeros((N, P, 4), dtype=dtype)
    for k in range(N):
        cell = (rows + orig[k, 0]) * Wc + (cols + orig[k, 1])
        Xw = world[cell]
        Xc = (Xw - cs[k]) @ Rs[k]  # R^T (X - c)
        if noise > 0:
            Xc = Xc * (1.0 + noise * rng.normal(size=(P, 1)))
        pts[k, :, :3] = Xc / scale[agent_of[k]]
        pts[k, :, 3] = rng.lognormal(1.0, 0.5, size=P)
    # edges
    edges = []
    for g in range(agents):
        b = g * n_kf
        edges += [(b + k, b + k + 1) for k in range(n_kf - 1)]
        edges += [(b + k, b + k + 2) for k in range(0, n_kf - 2, 2)]
        if loop > 0:
            edges += [(b + k - loop, b + k) for k in range(loop, n_kf, loop)]
    if agents > 1 and n_inter > 0:
        def shared(i, j):
            d = np.abs(orig[i] - orig[j])
            return max(0, H - d[0]) * max(0, W - d[1])
        inter = []
        for g in range(1, agents):
            best = max(((shared(i, j), i, j) for i in range(g * n_kf, (g + 1) * n_kf, 3)
                        for j in range(0, g * n_kf, 3)))
            inter.append((best[2], best[1]))
        cand = sorted(((shared(i, j), j, i) for i in range(n_kf, N, 5) for j in range(0, N, 5)
                       if agent_of[j] < agent_of[i]), reverse=True)
        for sc, j, i in cand:
            if len(inter) >= n_inter:
                break
            if (j, i) not in inter and sc > 0:
                inter.append((j, i))
        edges += inter
        if reverse_inter:  # the same pairs in the other direction (pixels of the later agent listed)
            edges += [(j, i) for (i, j) in inter]
    idx = []
    for (i, j) in edges:
        dv = orig[i, 0] - orig[j, 0]
        du = orig[i, 1] - orig[j, 1]
        v2, u2 = rows + dv, cols + du
        ok = (v2 >= 0) & (v2 < H) & (u2 >= 0) & (u2 < W)
        out = np.where(ok, v2 * W + u2, -1).astype(np.int32)
        if outlier > 0:
            vm = np.nonzero(ok)[0]
            pick = vm[rng.random(vm.size) < outlier]
            out[pick] = rng.integers(0, P, size=pick.size)
        if band is not None:  # valid-pixel mask: a column band covering U[band] of the image
            width = max(1, int(round(rng.uniform(band[0], band[1]) * W)))
            u0 = int(rng.integers(0, W - width + 1))
            out[(cols < u0) | (cols >= u0 + width)] = -1
        idx.append(out)
    # poses
    gt = np.zeros((N, 8))
    init = np.zeros((N, 8))
    for k in range(N):
        s = scale[agent_of[k]]
        gt[k, :3] = cs[k]
        gt[k, 3:7] = quat_from_matrix(Rs[k])
        gt[k, 7] = s
        if k == 0:
            init[k] = gt[k]
            continue
        dR = _axis_angle(rng.normal(size=3), pert_rot)
        dvv = rng.normal(size=3)
        dvv *= pert_trans / np.linalg.norm(dvv)
        ds = pert_scale if rng.random() < 0.5 else 1.0 / pert_scale
        init[k, :3] = cs[k] + s * Rs[k] @ dvv
        init[k, 3:7] = quat_from_matrix(Rs[k] @ dR)
        init[k, 7] = s * ds
    ei = np.array([e[0] for e in edges], dtype=np.int32) + kf_base
    ej = np.array([e[1] for e in edges], dtype=np.int32) + kf_base
    return dict(points=pts.reshape(N * P, 4), agent_of=agent_of, edge_i=ei, edge_j=ej,
                match_idx=np.concatenate(idx).astype(np.int32), poses_gt=gt, poses_init=init, N=N)


def make_cloud_problem(seed: int = 0, graph_specs: Optional[Sequence[dict]] = None, *, dtype=np.float32,
                       iters: int = 10, name: str = "cloud", **defaults) -> Problem:
    """A batch of shared-canvas graphs (one per entry of ``graph_specs``; keys: agents,
    n_kf, H, W, period, shift, loop, n_inter, noise, outlier, pert_rot, pert_trans,
    pert_scale, reverse_inter, band)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = dict(agents=1, n_kf=20, H=48, W=64, period=100, shift=8, loop=0, n_inter=4, noise=0.0, outlier=0.0,
                pert_rot=0.05, pert_trans=0.1, pert_scale=1.05, reverse_inter=False, band=None)
    base.update(defaults)
    specs = list(graph_specs) if graph_specs is not None else [base]
    parts: List[dict] = []
    kf_off, e_off, hs, ws, anchors = [0], [0], [], [], []
    for spec in specs:
        sp = dict(base)
        sp.update(spec)
        g = _graph(rng, kf_base=kf_off[-1], dtype=dtype, **sp)
        anchors.append(kf_off[-1])
        parts.append(g)
        kf_off.append(kf_off[-1] + g["N"])
        e_off.append(e_off[-1] + len(g["edge_i"]))
        hs.append(sp["H"])
        ws.append(sp["W"])
    cat = lambda key: np.concatenate([p[key] for p in parts])
    return Problem(
        name=name, kf_offset=np.array(kf_off, np.int32), height=np.array(hs, np.int32),
        width=np.array(ws, np.int32), agent_of=cat("agent_of"),
        points=parts[0]["points"] if len(parts) == 1 else cat("points"),
        edge_offset=np.array(e_off, np.int32), edge_i=cat("edge_i"), edge_j=cat("edge_j"),
        match_idx=cat("match_idx"), anchor=np.array(anchors, np.int32), poses_gt=cat("poses_gt"),
        poses_init=cat("poses_init"), iters=iters)
