"""Synthetic per-keyframe segment labels and per-segment range errors (inputs only).

The segment-level structure refinement takes segment labels as input (the paper draws
them with SLIC over normals and log-range, ~200 per keyframe); here every keyframe gets
compact Voronoi cells of jittered grid seeds (about ``n_seg`` cells, ids 0..n-1 in
row-major seed order, labels are local to the keyframe).  ``perturb_segment_ranges``
scales the range of every pixel of a segment by exp(delta_g), delta_g ~ N(0, sigma), to
stand in for the per-segment scale errors of predicted geometry.
"""
from __future__ import annotations

import math

import numpy as np


def voronoi_labels(H: int, W: int, n_seg: int, rng) -> np.ndarray:
    """int32 [H*W] labels of ~n_seg compact cells: the nearest of a grid of seeds, each
    jittered by up to 0.3 of its cell (so the nearest seed of a pixel is always one of
    the 3 x 3 cells around the pixel's own cell, the only ones compared)."""
    gy = max(1, int(round(math.sqrt(n_seg * H / W))))
    gx = max(1, int(round(n_seg / gy)))
    ch, cw = H / gy, W / gx
    sy = (np.arange(gy)[:, None] + 0.5 + rng.uniform(-0.3, 0.3, size=(gy, gx))) * ch
    sx = (np.arange(gx)[None, :] + 0.5 + rng.uniform(-0.3, 0.3, size=(gy, gx))) * cw
    yy, xx = np.mgrid[0:H, 0:W]
    cy = np.minimum((yy / ch).astype(np.int64), gy - 1)
    cx = np.minimum((xx / cw).astype(np.int64), gx - 1)
    best = np.full((H, W), np.inf)
    lab = np.zeros((H, W), dtype=np.int64)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ny, nx = cy + dy, cx + dx
            ok = (ny >= 0) & (ny < gy) & (nx >= 0) & (nx < gx)
            nyc, nxc = np.clip(ny, 0, gy - 1), np.clip(nx, 0, gx - 1)
            d = (yy + 0.5 - sy[nyc, nxc]) ** 2 + (xx + 0.5 - sx[nyc, nxc]) ** 2
            d = np.where(ok, d, np.inf)
            upd = d < best
            best[upd] = d[upd]
            lab[upd] = (nyc * gx + nxc)[upd]
    return lab.ravel().astype(np.int32)


def problem_labels(prob, n_seg: int = 200, seed: int = 0) -> np.ndarray:
    """Labels for every keyframe of a problem, concatenated like its pixels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for g in range(prob.num_graphs):
        H, W = int(prob.height[g]), int(prob.width[g])
        for _ in range(int(prob.kf_offset[g]), int(prob.kf_offset[g + 1])):
            out.append(voronoi_labels(H, W, n_seg, rng))
    return np.concatenate(out).astype(np.int32)


def perturb_segment_ranges(points: np.ndarray, labels: np.ndarray, pix_off: np.ndarray, sigma: float,
                           seed: int = 0) -> np.ndarray:
    """A copy of packed points whose ranges are scaled by exp(delta) per (keyframe, segment)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.array(points, copy=True)
    for k in range(len(pix_off) - 1):
        a, b = int(pix_off[k]), int(pix_off[k + 1])
        L = labels[a:b]
        n = int(L.max()) + 1 if (L >= 0).any() else 0
        delta = rng.normal(size=n) * sigma
        f = np.where(L >= 0, np.exp(delta[np.maximum(L, 0)]), 1.0).astype(np.float64)
        out[a:b, :3] = (out[a:b, :3].astype(np.float64) * f[:, None]).astype(out.dtype)
    return out
