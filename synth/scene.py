"""Procedural planes-and-boxes scenes, agent walks, pointmaps and dense correspondences.

Recipe (all draws from one ``numpy.random.Generator(PCG64(seed))``):

* Scene: ``n_planes`` planes with normals uniform on the sphere and offsets |d| in
  [6, 10] m (walls around the central region), plus ``n_boxes`` axis-aligned boxes with
  sides in [1, 5] m, all inside the cube [-10, 10]^3; hit points outside the cube are
  discarded, so a ray that leaves the cube without a hit yields no point.
* Agents: each walks ``n_kf`` keyframes in the central cube [-5, 5]^3 at constant height,
  0.5 m per step with a yaw change uniform in +-10 deg (+-25 deg when no such step is
  admissible), keeping >= 0.5 m clearance from every surface; when less than 4 m of
  free path lies ahead it turns (<= 25 deg per step) towards the most open heading.  Agent a > 0 starts within 1.5 m of a keyframe of an earlier agent with a
  heading within +-45 deg of it, so that the agents' views overlap somewhere.  Inter-agent
  edges: first, for every agent a > 0, the best-overlapping pair linking it to an earlier
  agent (so the map is connected), then the highest-overlap pairs (overlap >= 0.1 on a
  256-pixel sample), preferring keyframes not yet linked.
* Pinhole camera (x right, y down, z forward), principal point at the image centre,
  pixel (u, v) looks along ((u + 0.5 - W/2)/f, (v + 0.5 - H/2)/f, 1).
* Each agent a has a gauge scale s_a ~ U[0.5, 2]: keyframe pointmaps hold metric
  camera-frame points divided by s_a, and the ground-truth pose is (R_wc, c_w, s_a), so
  pose * point = the metric world point.
* Edge (i, j): every valid pixel m of i is carried to j with the ground-truth poses,
  projected, and kept when the projected range agrees with j's own range at that pixel
  to 1 % (visibility).  ``exact=True`` then writes the carried point into pixel n of j
  (first claim wins, edges taken in ascending (j, i)), so the matched pair is the same
  world point and the residual vanishes at ground truth.
* Noise: every valid point is scaled along its ray by (1 + noise * N(0, 1)).
* Outliers: a fraction of each edge's matches is redirected to a uniformly drawn valid
  pixel of j.  Optional per-edge column band masks keep a contiguous band of columns of
  width U[band_lo, band_hi] * W.
* Confidences per pixel: U[1, 5] ("uniform") or lognormal(mu=1, sigma=0.5).
* Initial poses: ground truth composed on the right with a body-frame perturbation of
  rotation angle ``pert_rot`` (random axis), offset ``pert_trans`` (random direction,
  in the pose's world units) and scale factor ``pert_scale`` or its inverse; the
  anchor (first keyframe of agent 0) is left at ground truth.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
from typing import Dict, List, Optional, Tuple

import numpy as np

CUBE = 10.0
CENTRAL = 5.0
CLEARANCE = 0.5


# ----------------------------------------------------------------------------- rotations
def matrix_from_quat(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion stored (x, y, z, w); vectorised over (..., 4)."""
    q = np.asarray(q, dtype=np.float64)
    x, y, z, w = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - z * w)
    R[..., 0, 2] = 2 * (x * z + y * w)
    R[..., 1, 0] = 2 * (x * y + z * w)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - x * w)
    R[..., 2, 0] = 2 * (x * z - y * w)
    R[..., 2, 1] = 2 * (y * z + x * w)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def quat_from_matrix(R: np.ndarray) -> np.ndarray:
    """Unit quaternion (x, y, z, w), w >= 0, of a single rotation matrix (Shepperd's branch choice)."""
    R = np.asarray(R, dtype=np.float64)
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    if tr > 0:
        S = math.sqrt(tr + 1.0) * 2
        q = [(R[2, 1] - R[1, 2]) / S, (R[0, 2] - R[2, 0]) / S, (R[1, 0] - R[0, 1]) / S, 0.25 * S]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        S = math.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [0.25 * S, (R[0, 1] + R[1, 0]) / S, (R[0, 2] + R[2, 0]) / S, (R[2, 1] - R[1, 2]) / S]
    elif R[1, 1] > R[2, 2]:
        S = math.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 1] + R[1, 0]) / S, 0.25 * S, (R[1, 2] + R[2, 1]) / S, (R[0, 2] - R[2, 0]) / S]
    else:
        S = math.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[0, 2] + R[2, 0]) / S, (R[1, 2] + R[2, 1]) / S, 0.25 * S, (R[1, 0] - R[0, 1]) / S]
    q = np.array(q)
    q /= np.linalg.norm(q)
    if q[3] < 0:
        q = -q
    return q


def _axis_angle(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rodrigues rotation about a unit axis (generator-side perturbations only)."""
    a = axis / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def pose_matrix(p: np.ndarray) -> np.ndarray:
    """4x4 similarity [sR t; 0 1] of a stored pose (tx, ty, tz, qx, qy, qz, qw, s): the input
    format, for building queries and fusion transforms on the host."""
    p = np.asarray(p, dtype=np.float64)
    T = np.eye(4)
    T[:3, :3] = p[7] * matrix_from_quat(p[3:7] / np.linalg.norm(p[3:7]))
    T[:3, 3] = p[:3]
    return T


def pose_from_matrix(T: np.ndarray) -> np.ndarray:
    """Stored pose (t, q, s) of a 4x4 similarity (s = cube root of det(sR))."""
    s = float(np.cbrt(np.linalg.det(T[:3, :3])))
    return np.concatenate([T[:3, 3], quat_from_matrix(T[:3, :3] / s), [s]])


def random_pose(rng: np.random.Generator, trans: float = 1.0, rot: float = 0.3, log_scale: float = 0.05) -> np.ndarray:
    """A stored pose with N(0, trans^2) translation, a rotation of angle |N(0, rot^2)| about a
    uniform axis and scale exp(N(0, log_scale^2))."""
    t = rng.normal(size=3) * trans
    R = _axis_angle(rng.normal(size=3), abs(rng.normal()) * rot)
    return np.concatenate([t, quat_from_matrix(R), [math.exp(rng.normal() * log_scale)]])


def _camera_rotation(yaw: float) -> np.ndarray:
    """Camera-to-world rotation: forward (z) horizontal at `yaw`, down (y) = -world z."""
    fwd = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    down = np.array([0.0, 0.0, -1.0])
    right = np.cross(down, fwd)
    return np.stack([right, down, fwd], axis=1)


# ----------------------------------------------------------------------------- geometry
@dataclasses.dataclass
class Geometry:
    plane_n: np.ndarray  # (P, 3) unit normals, plane n.x = d
    plane_d: np.ndarray  # (P,)
    box_lo: np.ndarray   # (B, 3)
    box_hi: np.ndarray   # (B, 3)


def make_geometry(rng: np.random.Generator, n_planes: int = 6, n_boxes: int = 3) -> Geometry:
    n = rng.normal(size=(n_planes, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d = rng.uniform(6.0, CUBE, size=n_planes) * rng.choice([-1.0, 1.0], size=n_planes)
    side = rng.uniform(1.0, 5.0, size=(n_boxes, 3))
    centre = rng.uniform(-CUBE + side / 2, CUBE - side / 2)
    return Geometry(n, d, centre - side / 2, centre + side / 2)


def clearance(geom: Geometry, p: np.ndarray) -> float:
    dp = np.abs(geom.plane_n @ p - geom.plane_d).min() if len(geom.plane_d) else np.inf
    outside = np.maximum(np.maximum(geom.box_lo - p, p - geom.box_hi), 0.0)
    inside = np.all((p >= geom.box_lo) & (p <= geom.box_hi), axis=1)
    db = np.where(inside, 0.0, np.linalg.norm(outside, axis=1))
    return float(min(dp, db.min() if len(db) else np.inf))


def raycast(geom: Geometry, origin: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Distance multiplier t of the first hit along origin + t * dirs (inf where none)."""
    best = np.full(dirs.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        for n, d in zip(geom.plane_n, geom.plane_d):
            den = dirs @ n
            t = (d - origin @ n) / den
            ok = np.isfinite(t) & (t > 1e-9)
            p = origin[None, :] + t[:, None] * dirs
            ok &= np.all(np.abs(p) <= CUBE, axis=1)
            best = np.where(ok & (t < best), t, best)
        inv = 1.0 / dirs
        for lo, hi in zip(geom.box_lo, geom.box_hi):
            t1 = (lo - origin) * inv
            t2 = (hi - origin) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=1)
            ok = (tmax >= tmin) & (tmin > 1e-9)
            best = np.where(ok & (tmin < best), tmin, best)
    return best


def pixel_rays(H: int, W: int, f: float) -> np.ndarray:
    v, u = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    return np.stack([(u + 0.5 - W / 2) / f, (v + 0.5 - H / 2) / f, np.ones_like(u)], axis=-1).reshape(-1, 3)


# ----------------------------------------------------------------------------- walks
def walk(geom: Geometry, rng: np.random.Generator, n_kf: int, start: np.ndarray, yaw: float,
         step: float = 0.5, yaw_step_deg: float = 10.0) -> List[Tuple[np.ndarray, float]]:
    """Random walk with bounded turns that steers towards open space before it is cornered."""
    def ok(r: np.ndarray) -> bool:
        return bool(np.all(np.abs(r) <= CENTRAL) and clearance(geom, r) >= CLEARANCE)

    def free_ahead(q: np.ndarray, y: float, limit: float = 8.0) -> float:
        d = np.array([math.cos(y), math.sin(y), 0.0])
        s = 0.0
        while s < limit and ok(q + (s + step) * d):
            s += step
        return s

    def wrap(a: float) -> float:
        return (a + math.pi) % (2 * math.pi) - math.pi

    out = [(start.copy(), yaw)]
    p = start.copy()
    max_turn = math.radians(2.5 * yaw_step_deg)
    for _ in range(n_kf - 1):
        if free_ahead(p, yaw) >= 4.0:
            base = [yaw + math.radians(rng.uniform(-yaw_step_deg, yaw_step_deg)) for _ in range(12)]
        else:  # turn towards the most open heading, at most 25 deg per step
            heads = np.linspace(-math.pi, math.pi, 36, endpoint=False)
            target = heads[int(np.argmax([free_ahead(p, h) for h in heads]))]
            turn = max(-max_turn, min(max_turn, wrap(target - yaw)))
            base = [yaw + turn + math.radians(rng.uniform(-2, 2)) for _ in range(4)]
            base += [yaw + rng.uniform(-max_turn, max_turn) for _ in range(12)]
        moved = False
        for y in base:
            q = p + step * np.array([math.cos(y), math.sin(y), 0.0])
            if ok(q):
                p, yaw, moved = q, y, True
                break
        if not moved:
            raise RuntimeError("walk: no admissible step")
        out.append((p.copy(), yaw))
    return out


def _free_start(geom: Geometry, rng: np.random.Generator, near: Optional[np.ndarray] = None,
                radius: float = 1.5) -> np.ndarray:
    for _ in range(10000):
        if near is None:
            p = np.array([rng.uniform(-CENTRAL + 1, CENTRAL - 1), rng.uniform(-CENTRAL + 1, CENTRAL - 1),
                          rng.uniform(-1.0, 1.0)])
        else:
            p = near + np.array([rng.uniform(-radius, radius), rng.uniform(-radius, radius), rng.uniform(-0.3, 0.3)])
        if np.all(np.abs(p) <= CENTRAL) and clearance(geom, p) >= CLEARANCE:
            return p
    raise RuntimeError("no free start position")


# ----------------------------------------------------------------------------- problem
@dataclasses.dataclass
class Problem:
    """One batch of independent pose graphs in a flat keyframe index space."""
    name: str
    kf_offset: np.ndarray    # int32 [G+1]
    height: np.ndarray       # int32 [G]
    width: np.ndarray        # int32 [G]
    agent_of: np.ndarray     # int32 [N]
    points: np.ndarray       # [sum P_k, 4] (x, y, z, confidence), storage dtype
    edge_offset: np.ndarray  # int32 [G+1]
    edge_i: np.ndarray       # int32 [E] (streamed keyframe, global id)
    edge_j: np.ndarray       # int32 [E] (gathered keyframe, global id)
    match_idx: np.ndarray    # int32 [sum_e P_{edge_i[e]}], pixel of j or -1
    anchor: np.ndarray       # int32 [G]
    poses_gt: np.ndarray     # float64 [N, 8] (tx, ty, tz, qx, qy, qz, qw, s)
    poses_init: np.ndarray   # float64 [N, 8]
    iters: int = 10
    sigma_ray: float = 0.003
    sigma_dist: float = 10.0
    huber_k: float = 1.345
    lam: float = 0.0
    eps0: float = 1e-6
    max_attempts: int = 6

    @property
    def num_graphs(self) -> int:
        return int(len(self.kf_offset) - 1)

    @property
    def num_kf(self) -> int:
        return int(self.kf_offset[-1])

    @property
    def num_edges(self) -> int:
        return int(len(self.edge_i))

    def pixels_of(self) -> np.ndarray:
        """Pixel count of every keyframe, int64 [N]."""
        hw = (self.height.astype(np.int64) * self.width.astype(np.int64))
        counts = np.zeros(self.num_kf, dtype=np.int64)
        for g in range(self.num_graphs):
            counts[self.kf_offset[g]:self.kf_offset[g + 1]] = hw[g]
        return counts

    def pix_offset(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.pixels_of())]).astype(np.int64)

    def idx_offset(self) -> np.ndarray:
        p = self.pixels_of()
        return np.concatenate([[0], np.cumsum(p[self.edge_i])]).astype(np.int64)

    def valid_matches(self) -> int:
        return int((self.match_idx >= 0).sum())

    def storage_bytes_per_pixel(self) -> int:
        return 4 * self.points.dtype.itemsize

    def params(self) -> Dict[str, float]:
        return dict(sigma_ray=self.sigma_ray, sigma_dist=self.sigma_dist, huber_k=self.huber_k,
                    lam=self.lam, eps0=self.eps0, max_attempts=self.max_attempts)


def _render(geom, rays, R, c):
    t = raycast(geom, c, rays @ R.T)
    valid = np.isfinite(t)
    X = np.where(valid[:, None], rays * np.where(valid, t, 0.0)[:, None], 0.0)
    return X, valid


def _project(Xc: np.ndarray, H: int, W: int, f: float):
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.floor(f * Xc[:, 0] / Xc[:, 2] + W / 2)
        v = np.floor(f * Xc[:, 1] / Xc[:, 2] + H / 2)
    ok = (Xc[:, 2] > 1e-6) & np.isfinite(u) & np.isfinite(v) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    n = np.where(ok, v * W + u, -1).astype(np.int64)
    return n, ok


def _overlap_score(Xw_i, valid_i, R_j, c_j, rng_j, H, W, f, sample):
    """Fraction of a pixel sample of i that is visible in j (ground-truth geometry)."""
    idx = sample[valid_i[sample]]
    if idx.size == 0:
        return 0.0
    Xc = (Xw_i[idx] - c_j) @ R_j
    n, ok = _project(Xc, H, W, f)
    r = np.linalg.norm(Xc, axis=1)
    vis = ok.copy()
    vis[ok] = np.abs(rng_j[n[ok]] - r[ok]) <= 0.01 * r[ok]
    return float(vis.sum()) / float(sample.size)


def _build_graph(rng, geom, *, agents, n_kf, H, W, f, noise, conf, outlier, skip_max, n_inter, exact,
                 band, pert_rot, pert_trans, pert_scale, kf_base, min_valid_frac=0.02):
    rays = pixel_rays(H, W, f)
    P = H * W
    # ---- walks
    walks = []
    for a in range(agents):
        if a == 0:
            start = _free_start(geom, rng)
            yaw = rng.uniform(-math.pi, math.pi)
        else:
            src = walks[rng.integers(0, a)]
            k = int(rng.integers(0, len(src)))
            start = _free_start(geom, rng, near=src[k][0])
            yaw = src[k][1] + math.radians(rng.uniform(-45, 45))
        walks.append(walk(geom, rng, n_kf, start, yaw))
    scale = rng.uniform(0.5, 2.0, size=agents)
    N = agents * n_kf
    Rs, cs, agent_of = [], [], []
    for a in range(agents):
        for (c, yaw) in walks[a]:
            Rs.append(_camera_rotation(yaw))
            cs.append(c)
            agent_of.append(a)
    # ---- render metric camera-frame points
    Xm = np.zeros((N, P, 3))
    valid = np.zeros((N, P), dtype=bool)
    for k in range(N):
        Xm[k], valid[k] = _render(geom, rays, Rs[k], cs[k])
    ranges = np.where(valid, np.linalg.norm(Xm, axis=2), np.inf)
    # ---- edges: sequential, (k, k+2) covisibility, inter-agent
    edges = []
    for a in range(agents):
        base = a * n_kf
        edges += [(base + k, base + k + 1) for k in range(n_kf - 1)]
        edges += [(base + k, base + k + 2) for k in range(0, n_kf - 2, 2) if k <= skip_max]
    if agents > 1 and n_inter > 0:
        sample = rng.choice(P, size=min(P, 256), replace=False)
        cand = []
        Xw = [Xm[k] @ Rs[k].T + cs[k] for k in range(N)]
        for i in range(N):
            for j in range(N):
                if agent_of[j] <= agent_of[i]:
                    continue
                s = _overlap_score(Xw[i], valid[i], Rs[j], cs[j], ranges[j], H, W, f, sample)
                if s >= 0.1:
                    cand.append((s, i, j))
        cand.sort(key=lambda t: -t[0])
        chosen, used = [], set()
        for a in range(1, agents):     # first link every agent to an earlier one (connected map)
            link = [(s, i, j) for s, i, j in cand if agent_of[j] == a and agent_of[i] < a]
            if not link:
                raise RuntimeError(f"agent {a} has no overlapping keyframe with an earlier agent")
            s, i, j = link[0]
            chosen.append((i, j)); used.update((i, j))
        for s, i, j in cand:           # prefer keyframes not yet linked across agents
            if len(chosen) >= n_inter:
                break
            if i in used or j in used or (i, j) in chosen:
                continue
            chosen.append((i, j)); used.update((i, j))
        for s, i, j in cand:
            if len(chosen) >= n_inter:
                break
            if (i, j) not in chosen:
                chosen.append((i, j))
        if len(chosen) < n_inter:
            raise RuntimeError(f"only {len(chosen)} overlapping inter-agent pairs (need {n_inter})")
        edges += chosen
    order = sorted(range(len(edges)), key=lambda e: (edges[e][1], edges[e][0]))
    # ---- correspondences (edges taken in ascending (j, i) so claims precede reuse)
    idx = {}
    claimed = np.zeros((N, P), dtype=bool)
    for e in order:
        i, j = edges[e]
        m = np.nonzero(valid[i])[0]
        Pw = Xm[i, m] @ Rs[i].T + cs[i]
        Xc = (Pw - cs[j]) @ Rs[j]
        n, ok = _project(Xc, H, W, f)
        r = np.linalg.norm(Xc, axis=1)
        ok[ok] &= np.abs(ranges[j][n[ok]] - r[ok]) <= 0.01 * r[ok]
        m, n, Xc = m[ok], n[ok], Xc[ok]
        if exact:
            keep = ~claimed[j, n]
            m, n, Xc = m[keep], n[keep], Xc[keep]
            _, first = np.unique(n, return_index=True)
            first.sort()
            m, n, Xc = m[first], n[first], Xc[first]
            claimed[j, n] = True
            Xm[j, n] = Xc
        if m.size < min_valid_frac * P:
            raise RuntimeError(f"edge ({i}, {j}) has only {m.size} matches")
        out = np.full(P, -1, dtype=np.int32)
        out[m] = n
        idx[e] = out
    # ---- outliers and band masks
    for e in range(len(edges)):
        i, j = edges[e]
        out = idx[e]
        vm = np.nonzero(out >= 0)[0]
        if outlier > 0 and vm.size:
            pick = vm[rng.random(vm.size) < outlier]
            vj = np.nonzero(valid[j])[0]
            out[pick] = vj[rng.integers(0, vj.size, size=pick.size)]
        if band is not None:
            frac = rng.uniform(band[0], band[1])
            width = max(1, int(round(frac * W)))
            u0 = int(rng.integers(0, W - width + 1))
            cols = np.arange(P) % W
            out[(cols < u0) | (cols >= u0 + width)] = -1
    # ---- noise, confidences, storage units
    if noise > 0:
        Xm = Xm * (1.0 + noise * rng.normal(size=(N, P)))[:, :, None]
    if conf == "uniform":
        c = rng.uniform(1.0, 5.0, size=(N, P))
    else:
        c = rng.lognormal(1.0, 0.5, size=(N, P))
    pts = np.zeros((N, P, 4))
    for k in range(N):
        pts[k, :, :3] = Xm[k] / scale[agent_of[k]]
        pts[k, :, 3] = c[k]
    pts[~valid] = 0.0
    # ---- poses
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
        axis = rng.normal(size=3)
        dR = _axis_angle(axis, pert_rot)
        dv = rng.normal(size=3)
        dv *= pert_trans / np.linalg.norm(dv)
        ds = pert_scale if rng.random() < 0.5 else 1.0 / pert_scale
        R1 = Rs[k] @ dR
        init[k, :3] = cs[k] + s * Rs[k] @ dv
        init[k, 3:7] = quat_from_matrix(R1)
        init[k, 7] = s * ds
    ei = np.array([edges[e][0] for e in range(len(edges))], dtype=np.int32) + kf_base
    ej = np.array([edges[e][1] for e in range(len(edges))], dtype=np.int32) + kf_base
    midx = np.concatenate([idx[e] for e in range(len(edges))]) if edges else np.zeros(0, np.int32)
    return dict(points=pts.reshape(N * P, 4), agent_of=np.array(agent_of, np.int32), edge_i=ei, edge_j=ej,
                match_idx=midx.astype(np.int32), poses_gt=gt, poses_init=init, N=N)


def make_problem(seed: int = 0, *, agents: int = 2, n_kf: int = 6, H: int = 48, W: int = 64, f: float = 50.0,
                 noise: float = 0.005, conf: str = "uniform", outlier: float = 0.10, skip_max: int = -1,
                 n_inter: int = 4, exact: bool = True, band: Optional[Tuple[float, float]] = None,
                 dtype=np.float64, iters: int = 10, pert_rot: float = 0.05, pert_trans: float = 0.1,
                 pert_scale: float = 1.05, n_planes: int = 6, n_boxes: int = 3, name: str = "custom",
                 num_graphs: int = 1, graph_specs: Optional[List[dict]] = None) -> Problem:
    """Build a seeded batch of ``num_graphs`` graphs (or one per entry of ``graph_specs``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = dict(agents=agents, n_kf=n_kf, H=H, W=W, f=f, noise=noise, conf=conf, outlier=outlier,
                skip_max=skip_max, n_inter=n_inter, exact=exact, band=band, pert_rot=pert_rot,
                pert_trans=pert_trans, pert_scale=pert_scale)
    specs = graph_specs if graph_specs is not None else [base] * num_graphs
    parts = []
    kf_off, e_off, hs, ws, anchors = [0], [0], [], [], []
    for spec in specs:
        sp = dict(base)
        sp.update(spec)
        for attempt in range(50):
            geom = make_geometry(rng, n_planes, n_boxes)
            try:
                g = _build_graph(rng, geom, kf_base=kf_off[-1], **sp)
                break
            except RuntimeError:
                continue
        else:
            raise RuntimeError("could not build a graph with the requested overlap")
        anchors.append(kf_off[-1])
        parts.append(g)
        kf_off.append(kf_off[-1] + g["N"])
        e_off.append(e_off[-1] + len(g["edge_i"]))
        hs.append(sp["H"]); ws.append(sp["W"])
    cat = lambda key: np.concatenate([p[key] for p in parts])
    return Problem(
        name=name,
        kf_offset=np.array(kf_off, np.int32), height=np.array(hs, np.int32), width=np.array(ws, np.int32),
        agent_of=cat("agent_of"), points=cat("points").astype(dtype), edge_offset=np.array(e_off, np.int32),
        edge_i=cat("edge_i"), edge_j=cat("edge_j"), match_idx=cat("match_idx"),
        anchor=np.array(anchors, np.int32), poses_gt=cat("poses_gt"), poses_init=cat("poses_init"), iters=iters)


# Named workloads: the paper's 512x384 pointmaps, 2-4 agent teams, long horizons.
WORKLOADS: Dict[str, dict] = {
    # 2 agents x 6 keyframes, 64x48, FP64 storage, 10 sequential + 4 inter-agent edges.
    "two_agent_6kf_64x48": dict(agents=2, n_kf=6, H=48, W=64, f=50.0, noise=0.005, conf="uniform",
                                outlier=0.10, skip_max=-1, n_inter=4, exact=True, dtype=np.float64, iters=10),
    # 2 agents x 40 keyframes, 512x384 FP32, 78 sequential + 34 (k, k+2) + 8 inter = 120 edges.
    "two_agent_40kf_512x384": dict(agents=2, n_kf=40, H=384, W=512, f=400.0, noise=0.01, conf="lognormal",
                                   outlier=0.15, skip_max=32, n_inter=8, exact=False, dtype=np.float32,
                                   iters=15),
    # 4 agents x 150 keyframes, 512x384 FP16 storage, column-band masks 20-100 %, 60 inter edges.
    "four_agent_150kf_512x384_f16": dict(agents=4, n_kf=150, H=384, W=512, f=400.0, noise=0.01,
                                         conf="lognormal", outlier=0.15, skip_max=10 ** 9, n_inter=60,
                                         exact=False, band=(0.2, 1.0), dtype=np.float16, iters=10),
    # 4 agents x 30 keyframes, 512x384 FP32 (adjoint workload), 8 GN iterations.
    "four_agent_30kf_512x384": dict(agents=4, n_kf=30, H=384, W=512, f=400.0, noise=0.01, conf="lognormal",
                                    outlier=0.15, skip_max=26, n_inter=8, exact=False, dtype=np.float32,
                                    iters=8),
}


def _cache_path(name: str, seed: int, overrides: dict) -> Optional[str]:
    root = os.environ.get("COMO3R_SYNTH_CACHE", "")
    if not root:
        return None
    src = open(__file__, "rb").read()
    key = hashlib.sha256(src + repr((name, seed, sorted(overrides.items()))).encode()).hexdigest()[:20]
    return os.path.join(root, f"{name}-{seed}-{key}.npz")


def make_workload(name: str, seed: int = 0, **overrides) -> Problem:
    """A named workload; cached as .npz under $COMO3R_SYNTH_CACHE when that is set."""
    path = _cache_path(name, seed, overrides)
    if path and os.path.exists(path):
        z = np.load(path)
        fields = {f.name: z[f.name] for f in dataclasses.fields(Problem) if f.name in z.files}
        scal = {k: v.item() for k, v in fields.items() if v.ndim == 0}
        fields.update(scal)
        fields["name"] = str(fields["name"])
        return Problem(**fields)
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    prob = make_problem(seed, name=name, **spec)
    if path:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, **{f.name: getattr(prob, f.name) for f in dataclasses.fields(Problem)})
        os.replace(tmp, path)
    return prob
