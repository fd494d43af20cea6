"""Shared-canvas graph batches built directly in device memory, for workloads whose
pointmaps and match indices (tens of GB) are too large to generate on the host.

Same recipe as ``synth.cloud`` (a smooth panorama-like canvas of world points; keyframe k
of an agent sees an H x W window of it that moves along a smooth closed path; matched
pixels of an edge are the same canvas cell, so residuals vanish at ground truth without
noise; sequential, (k, k+2) covisibility, loop-closure and inter-agent edges; noise along
the ray, outliers redirected to a uniformly drawn pixel, lognormal(1, 0.5) confidences;
initial poses perturbed in the body frame), with two differences of implementation:

* the per-keyframe and per-edge quantities (window paths, camera paths, agent scales,
  edge lists, pose perturbations) come from ``numpy.random.Generator(PCG64(seed))`` on
  the host, and every per-pixel random number (depth noise, confidence, outlier choice
  and target) from a ``torch.Generator`` on the device seeded with ``seed`` -- so a batch
  is a deterministic function of (seed, specs, torch version, device kind), but not the
  same numbers as ``synth.cloud`` for the same seed;
* pixels and matches are produced keyframe-chunk by keyframe-chunk on the device, in the
  storage dtype, so the host holds only the graph description.

``make_cloud_batch_gpu`` returns the ``Problem`` (host description; ``points`` and
``match_idx`` are empty placeholders) and the two device tensors to hand to
``como3r.Graph(prob, points=..., match_idx=...)``.  ``graph_subproblem`` copies one graph
of such a batch back to the host as a self-contained ``Problem`` (keyframe and edge ids
re-based), which the oracle can evaluate.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from .scene import Problem, _axis_angle, quat_from_matrix

_DEFAULTS = dict(agents=1, n_kf=20, H=48, W=64, period=100, shift=8, loop=0, n_inter=4, noise=0.0, outlier=0.0,
                 pert_rot=0.05, pert_trans=0.1, pert_scale=1.05, reverse_inter=False)


def _graph_meta(rng, *, agents: int, n_kf: int, H: int, W: int, period: int, shift: int, loop: int, n_inter: int,
                noise: float, outlier: float, pert_rot: float, pert_trans: float, pert_scale: float,
                reverse_inter: bool = False) -> dict:
    """Host part of one graph: canvas field, window origins, cameras, edges and poses."""
    Hc, Wc = H + 2 * shift + 2, W + 2 * shift + 2
    field = [tuple(rng.uniform(0.5, 3.0, size=2)) + tuple(rng.uniform(0, 2 * math.pi, size=2)) for _ in range(4)]
    N = agents * n_kf
    scale = rng.uniform(0.5, 2.0, size=agents)
    agent_of = np.repeat(np.arange(agents), n_kf).astype(np.int32)
    orig = np.zeros((N, 2), dtype=np.int64)
    Rs = np.zeros((N, 3, 3))
    cs = np.zeros((N, 3))
    for g in range(agents):
        ph = rng.uniform(0, 2 * math.pi)
        ph_cam = rng.uniform(0, 2 * math.pi)
        for k in range(n_kf):
            t = 2 * math.pi * k / period + ph
            q = g * n_kf + k
            orig[q] = (int(round(shift * (1 + math.sin(t)))), int(round(shift * (1 + math.cos(t)))))
            tc = 2 * math.pi * k / period + ph_cam
            cs[q] = (1.2 * math.cos(tc), 1.2 * math.sin(tc), 0.3 * math.sin(2 * tc))
            yaw = 0.4 * math.sin(tc) + g * 0.3
            pitch = 0.1 * math.cos(tc)
            Rz = np.array([[math.cos(yaw), -math.sin(yaw), 0], [math.sin(yaw), math.cos(yaw), 0], [0, 0, 1]])
            Ry = np.array([[math.cos(pitch), 0, math.sin(pitch)], [0, 1, 0], [-math.sin(pitch), 0, math.cos(pitch)]])
            Rs[q] = Rz @ Ry
    edges: List[Tuple[int, int]] = []
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
        inter: List[Tuple[int, int]] = []
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
    return dict(H=H, W=W, Hc=Hc, Wc=Wc, field=field, N=N, scale=scale, agent_of=agent_of, orig=orig, Rs=Rs, cs=cs,
                edges=edges, gt=gt, init=init, noise=noise, outlier=outlier)


def _canvas(torch, m: dict, device) -> "torch.Tensor":
    Hc, Wc = m["Hc"], m["Wc"]
    a = torch.arange(Hc, device=device, dtype=torch.float64)[:, None] / Hc
    b = torch.arange(Wc, device=device, dtype=torch.float64)[None, :] / Wc
    f = torch.zeros((Hc, Wc), device=device, dtype=torch.float64)
    for ka, kb, pa, pb in m["field"]:
        f += torch.sin(2 * math.pi * ka * a + pa) * torch.cos(2 * math.pi * kb * b + pb)
    d = 8.0 + 2.0 * (f / 4.0)
    az = (torch.arange(Wc, device=device, dtype=torch.float64) / Wc - 0.5) * math.radians(200.0)
    el = (torch.arange(Hc, device=device, dtype=torch.float64) / Hc - 0.5) * math.radians(100.0)
    ce, se = torch.cos(el)[:, None], torch.sin(el)[:, None]
    dirs = torch.stack([ce * torch.cos(az)[None, :], ce * torch.sin(az)[None, :], se.expand(Hc, Wc)], dim=-1)
    return (dirs * d[..., None]).reshape(-1, 3)


def make_cloud_batch_gpu(seed: int, graph_specs: Sequence[dict], *, device: str = "cuda", storage=None,
                         iters: int = 10, name: str = "cloud-gpu", kf_chunk: int = 32, edge_chunk: int = 64,
                         **defaults):
    """A batch of shared-canvas graphs (one per entry of ``graph_specs``; keys as in
    ``synth.cloud.make_cloud_problem``) with pointmaps and match indices in device memory.

    Returns (problem, points [sum P_k, 4] in ``storage`` (default float32), match_idx int32)."""
    import torch
    storage = storage or torch.float32
    rng = np.random.Generator(np.random.PCG64(seed))
    base = dict(_DEFAULTS)
    base.update(defaults)
    metas = []
    for spec in graph_specs:
        sp = dict(base)
        sp.update(spec)
        metas.append(_graph_meta(rng, **sp))
    kf_off = np.cumsum([0] + [m["N"] for m in metas]).astype(np.int64)
    e_off = np.cumsum([0] + [len(m["edges"]) for m in metas]).astype(np.int64)
    px_kf = np.concatenate([np.full(m["N"], m["H"] * m["W"], dtype=np.int64) for m in metas])
    px_off = np.concatenate([[0], np.cumsum(px_kf)])
    n_slots = sum(len(m["edges"]) * m["H"] * m["W"] for m in metas)
    points = torch.empty((int(px_off[-1]), 4), dtype=storage, device=device)
    midx = torch.empty(int(n_slots), dtype=torch.int32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    slot = 0
    for gi, m in enumerate(metas):
        H, W, Wc = m["H"], m["W"], m["Wc"]
        P = H * W
        world = _canvas(torch, m, device)
        rows = torch.arange(P, device=device, dtype=torch.int64) // W
        cols = torch.arange(P, device=device, dtype=torch.int64) % W
        orig = torch.as_tensor(m["orig"], device=device)
        Rs = torch.as_tensor(m["Rs"], device=device)
        cs = torch.as_tensor(m["cs"], device=device)
        inv_s = torch.as_tensor(1.0 / m["scale"][m["agent_of"]], device=device)
        k0 = int(kf_off[gi])
        for a in range(0, m["N"], kf_chunk):
            b = min(m["N"], a + kf_chunk)
            cell = (rows[None, :] + orig[a:b, 0, None]) * Wc + (cols[None, :] + orig[a:b, 1, None])
            Xw = world[cell]  # [n, P, 3]
            Xc = torch.bmm(Xw - cs[a:b, None, :], Rs[a:b])  # R^T (X - c) as row vectors
            if m["noise"] > 0:
                Xc = Xc * (1.0 + m["noise"] * torch.randn((b - a, P, 1), generator=gen, device=device,
                                                          dtype=torch.float64))
            Xc = Xc * inv_s[a:b, None, None]
            conf = torch.exp(1.0 + 0.5 * torch.randn((b - a, P), generator=gen, device=device, dtype=torch.float64))
            p0 = int(px_off[k0 + a])
            dst = points[p0:p0 + (b - a) * P].view(b - a, P, 4)
            dst[..., :3] = Xc.to(storage)
            dst[..., 3] = conf.to(storage)
            del Xw, Xc, conf
        ei = np.array([e[0] for e in m["edges"]], dtype=np.int64)
        ej = np.array([e[1] for e in m["edges"]], dtype=np.int64)
        for a in range(0, len(ei), edge_chunk):
            b = min(len(ei), a + edge_chunk)
            dv = torch.as_tensor(m["orig"][ei[a:b], 0] - m["orig"][ej[a:b], 0], device=device)
            du = torch.as_tensor(m["orig"][ei[a:b], 1] - m["orig"][ej[a:b], 1], device=device)
            v2 = rows[None, :] + dv[:, None]
            u2 = cols[None, :] + du[:, None]
            ok = (v2 >= 0) & (v2 < H) & (u2 >= 0) & (u2 < W)
            out = torch.where(ok, v2 * W + u2, torch.full_like(v2, -1))
            if m["outlier"] > 0:
                pick = ok & (torch.rand(ok.shape, generator=gen, device=device) < m["outlier"])
                target = torch.randint(0, P, ok.shape, generator=gen, device=device)
                out = torch.where(pick, target, out)
            n = (b - a) * P
            midx[slot:slot + n] = out.reshape(-1).to(torch.int32)
            slot += n
            del v2, u2, ok, out
        del world
    agent_of = np.concatenate([m["agent_of"] for m in metas]).astype(np.int32)
    ei = np.concatenate([np.array([e[0] for e in m["edges"]], dtype=np.int64) + kf_off[g]
                         for g, m in enumerate(metas)]).astype(np.int32)
    ej = np.concatenate([np.array([e[1] for e in m["edges"]], dtype=np.int64) + kf_off[g]
                         for g, m in enumerate(metas)]).astype(np.int32)
    prob = Problem(
        name=name, kf_offset=kf_off.astype(np.int32), height=np.array([m["H"] for m in metas], np.int32),
        width=np.array([m["W"] for m in metas], np.int32), agent_of=agent_of,
        points=np.zeros((0, 4), dtype=np.float32), edge_offset=e_off.astype(np.int32), edge_i=ei, edge_j=ej,
        match_idx=np.zeros(0, dtype=np.int32), anchor=kf_off[:-1].astype(np.int32),
        poses_gt=np.concatenate([m["gt"] for m in metas]), poses_init=np.concatenate([m["init"] for m in metas]),
        iters=iters)
    return prob, points, midx


def graph_subproblem(prob: Problem, points, midx, g: int, poses: Optional[np.ndarray] = None) -> Problem:
    """Graph g of a device batch as a host ``Problem`` of one graph (ids re-based)."""
    k0, k1 = int(prob.kf_offset[g]), int(prob.kf_offset[g + 1])
    e0, e1 = int(prob.edge_offset[g]), int(prob.edge_offset[g + 1])
    P = int(prob.height[g]) * int(prob.width[g])
    px = prob.pixels_of().astype(np.int64)
    p0 = int(px[:k0].sum())
    slot_len = px[prob.edge_i.astype(np.int64)]
    s0 = int(slot_len[:e0].sum())
    n_slots = (e1 - e0) * P
    return Problem(
        name=f"{prob.name}[{g}]", kf_offset=np.array([0, k1 - k0], np.int32), height=prob.height[g:g + 1].copy(),
        width=prob.width[g:g + 1].copy(), agent_of=prob.agent_of[k0:k1].copy(),
        points=points[p0:p0 + (k1 - k0) * P].cpu().numpy(),
        edge_offset=np.array([0, e1 - e0], np.int32), edge_i=(prob.edge_i[e0:e1] - k0).astype(np.int32),
        edge_j=(prob.edge_j[e0:e1] - k0).astype(np.int32),
        match_idx=midx[s0:s0 + n_slots].cpu().numpy(), anchor=np.array([0], np.int32),
        poses_gt=prob.poses_gt[k0:k1].copy(),
        poses_init=(prob.poses_init if poses is None else poses)[k0:k1].copy(), iters=prob.iters,
        sigma_ray=prob.sigma_ray, sigma_dist=prob.sigma_dist, huber_k=prob.huber_k, lam=prob.lam, eps0=prob.eps0,
        max_attempts=prob.max_attempts)


def batch64_specs(seed: int = 5, n_graphs: int = 64, noise: float = 0.01, outlier: float = 0.15) -> List[dict]:
    """The 64-graph batch of uneven sizes: per graph 2-4 agents, 10-200 keyframes per agent,
    one resolution of 256x192, 384x288, 512x384; windows move by up to a tenth of the
    width along a 40-keyframe closed path; inter-agent edges ~2 % of the edges."""
    rng = np.random.default_rng(seed)
    res = [(192, 256), (288, 384), (384, 512)]
    specs = []
    for _ in range(n_graphs):
        H, W = res[int(rng.integers(0, 3))]
        agents, n_kf = int(rng.integers(2, 5)), int(rng.integers(10, 201))
        specs.append(dict(agents=agents, n_kf=n_kf, H=H, W=W, period=40, shift=W // 10, loop=0,
                          n_inter=max(agents - 1, int(round(0.03 * agents * n_kf))), noise=noise, outlier=outlier))
    return specs


def chain2000_spec(noise: float = 0.01, outlier: float = 0.02) -> List[dict]:
    """The long-horizon chain: one agent, 2,000 keyframes at 512x384, loop-closure edges
    (k - 100, k) every 100 keyframes (the window path closes every 100 keyframes)."""
    return [dict(agents=1, n_kf=2000, H=384, W=512, period=100, shift=51, loop=100, n_inter=0, noise=noise,
                 outlier=outlier)]
