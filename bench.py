#!/usr/bin/env python
"""Benchmark of the unified multi-agent Sim(3) Gauss-Newton refinement on one B300.

Workload: 2 agents x 40 keyframes, 512x384 FP32 pointmaps (196,608 px each), 120 edges
(78 sequential, 34 (k, k+2), 8 inter-agent), 1 % depth noise, lognormal confidences,
15 % outlier correspondences, 15 GN iterations (synthetic, seeded; see synth/).

A step is one como3r_solve: 15 full GN iterations (edge prep, residual / Jacobian /
reduction, per-edge reduction, assembly, damped block Cholesky solve with eps
escalation, retraction) from the perturbed initial poses.  `value` is GN iterations/s of
the mixed form with inputs resident in HBM; the plain FP64 form is timed beside it.
`e2e` repeats the mixed measurement through the C ABI with host (pinned) buffers: every
step uploads the pointmaps and matches and reads the poses and cost trace back; two graphs
are used in turn on two streams (one host thread each), so that one step's upload overlaps
another step's solve (`e2e.serial`: one graph, one step after the other).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica of the workload (the graphs of a
batch are independent; there is no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "two_agent_40kf_512x384"
METRIC = "Sim(3) GN iters/s & Mresiduals/s, mixed vs FP64 form, % of HBM peak"
UNIT = "GN iters/s"
FALLBACK_HBM_GBS = 6400.0
PROFILE = os.path.join(ROOT, "profiles", "residual_reduce_two_agent_40kf_512x384.txt")
K1_SOURCE = os.path.join(ROOT, "paper_2605_30488_b300", "csrc", "k_residual.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-sample-edges", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["all", "mixed", "gauge", "depth", "cfg5", "front", "team", "adjoint4"],
                    default="all",
                    help="mixed: time only the resident mixed form; gauge / depth / cfg5 / front / team / "
                         "adjoint4: only the gauge synchronisation / the structure refinement / the 64-graph "
                         "batch and the 2,000-keyframe chain / the front-end kernels / the 4 x 150 FP16 team / "
                         "the 4 x 30 adjoint workload (profiling runs)")
    ap.add_argument("--no-team", action="store_true", help="skip the 4 x 150 FP16 team and the 4 x 30 adjoint")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-graph batch and the 2,000-keyframe chain (per-graph latency)")
    ap.add_argument("--batch-reps", type=int, default=3)
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(prob) -> int:
    """Bytes K1 must move per launch: all match indices of every edge (4 B per streamed
    pixel) plus, per valid match, the streamed and the gathered packed pixel."""
    pix = prob.pixels_of()
    b_px = prob.storage_bytes_per_pixel()
    return int(4 * pix[prob.edge_i].sum() + 2 * b_px * prob.valid_matches())


def k1_traffic_from_profile():
    """DRAM bytes per K1 launch from the committed ncu summary, if it was taken on the
    current K1 source (sha256 recorded in the summary); else None."""
    return traffic_from_profile(PROFILE, K1_SOURCE)


def traffic_from_profile(summary: str, source: str):
    """DRAM bytes per launch from a committed ncu summary (path under profiles/ or
    absolute), if it was taken on the kernel's current source file (sha256 recorded in the
    summary; path under the package's csrc/ or absolute); else None."""
    summary = summary if os.path.isabs(summary) else os.path.join(ROOT, "profiles", summary)
    source = source if os.path.isabs(source) else os.path.join(ROOT, "paper_2605_30488_b300", "csrc", source)
    try:
        txt = open(summary).read()
        src = hashlib.sha256(open(source, "rb").read()).hexdigest()
        fields = dict(l.split(":", 1) for l in txt.splitlines() if ":" in l)
        if fields.get("source_sha256", "").strip() != src:
            return None
        return float(fields["traffic_bytes_per_launch"].strip())
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples (200 ms) with host timestamps."""
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        if not inside:  # very short timed region: nearest samples around it
            near = sorted(self.samples, key=lambda ts: min(abs(ts[0] - t0), abs(ts[0] - t1)))[:3]
            inside = [s for _, s in near]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(s[0]) for s in inside if s[0].replace(".", "").isdigit()]
        smax = [float(s[1]) for s in inside if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in inside for n, v in zip(names, s[4:8]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inside)}


def measure_batched(C, torch, prob, points, midx, iters: int, reps: int) -> dict:
    """Mixed-form solves of a (device-generated) batch: per-graph latency from the
    library's device-clock stamps (start of the call -> end of the graph's last
    factorisation), pooled over `reps` calls, and aggregate residuals/s from CUDA events."""
    g = C.Graph(prob, mode=C.MIXED, points=points, match_idx=midx)
    stats = g.stats()
    poses0 = torch.tensor(prob.poses_init, dtype=torch.float64, device=points.device)
    work = poses0.clone()
    g.solve(work, iters, trace=False)  # warm-up (also captures the iteration graph)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, total_ms, solved = [], 0.0, True
    for _ in range(reps):
        work.copy_(poses0)
        torch.cuda.synchronize()
        ev0.record()
        st, _, info = g.solve(work, iters, trace=False)
        ev1.record()
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        t0, done = g.timestamps()
        lat.extend(((done - t0) / 1e6).tolist())
        solved = solved and all(x["solved"] for x in info)
    stages = g.time_stages(poses0, reps=3)
    g.close()
    lat = np.sort(np.asarray(lat))
    valid = int(stats["valid"])
    return {"graphs": prob.num_graphs, "keyframes": prob.num_kf, "edges": prob.num_edges,
            "pixels": int(prob.pixels_of().sum()), "valid_matches_per_iter": valid, "iters_per_call": iters,
            "calls": reps, "all_solved": bool(solved),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "min": float(lat[0]), "max": float(lat[-1])},
            "ms_per_call": total_ms / reps, "gn_iters_per_s": reps * iters / (total_ms / 1e3),
            "mresiduals_per_s": valid * reps * iters / (total_ms / 1e3) / 1e6, "stages_ms": stages,
            "plan": {k: stats[k] for k in ("items", "chunk", "block", "grid", "levels", "smem_solve", "solve_ctas")}}


def pipelined_e2e(C, torch, prob, pts_h, idx_h, iters: int, esteps: int, warmup: int, barrier, max_over_ranks):
    """End-to-end throughput of two graphs used in turn on two streams, one host thread
    each: every step uploads its pointmaps and matches from pinned host memory, solves and
    reads its poses and cost trace back (como3r_solve returns after the readback); one
    upload at a time holds the host-to-device link, so one graph's upload overlaps the
    other's solve.  Timed on the device: both streams wait on a
    start event of the current stream, which waits on both before the end event."""
    cur = torch.cuda.current_stream()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    graphs = [C.Graph(prob, mode=C.MIXED, points=pts_h, match_idx=idx_h, copy_inputs=True, stream=st)
              for st in streams]
    poses = [torch.tensor(prob.poses_init, dtype=torch.float64).pin_memory() for _ in graphs]
    init = torch.from_numpy(prob.poses_init)
    per = max(2, (esteps + 1) // 2)
    errors = []
    upload = threading.Lock()  # one upload on the link at a time: the two graphs alternate

    def run(k: int, n: int):
        try:
            with torch.cuda.stream(streams[k]):
                for _ in range(n):
                    poses[k].copy_(init)
                    with upload:
                        graphs[k].update_inputs(pts_h, idx_h)
                        streams[k].synchronize()
                    graphs[k].solve(poses[k], iters, trace=True)
        except Exception as e:  # surfaced after the join
            errors.append(e)

    def both(n: int):
        ts = [threading.Thread(target=run, args=(k, n)) for k in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errors:
            raise errors[0]

    both(max(1, min(warmup, 2)))
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for st in streams:
        st.wait_event(e0)
    both(per)
    for st in streams:
        cur.wait_stream(st)
    e1.record(cur)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    for g in graphs:
        g.close()
    return 2 * per * iters / (ms / 1e3), 2 * per


def measure_cfg5(C, torch, dev, reps: int) -> dict:
    """The 64-graph batch (2-4 agents, 10-200 keyframes per agent, 256x192..512x384, FP32,
    1 % depth noise, 15 % outliers) and the 2,000-keyframe chain (512x384, 2 % outliers,
    loop closures every 100 keyframes), both generated in device memory from seed 5."""
    from synth.cloud_gpu import batch64_specs, chain2000_spec, make_cloud_batch_gpu
    out = {}
    for key, specs, iters in (("batch64", batch64_specs(), 10), ("chain2000", chain2000_spec(), 10)):
        t = time.time()
        prob, pts, midx = make_cloud_batch_gpu(5, specs, device=str(dev), name=key)
        torch.cuda.synchronize()
        gen_s = time.time() - t
        r = measure_batched(C, torch, prob, pts, midx, iters, reps)
        r["generate_s"] = gen_s
        r["inputs_gb"] = (pts.numel() * pts.element_size() + midx.numel() * 4) / 1e9
        out[key] = r
        del pts, midx
        torch.cuda.empty_cache()
    return out


def measure_gauge(C, torch, dev, reps: int = 10) -> dict:
    """Cross-agent verification + gauge synchronisation (Sec. III-B/III-C) of 60 candidates
    at 512x384: the inter-agent pairs (both decoded directions) of a 4-agent x 40-keyframe
    FP32 team (1 % noise, 15 % outliers) generated in device memory, seed 7.  The pass
    over the matches is HBM-bound: 4 B per listed pixel of each direction plus the two
    packed pixels of every valid match."""
    from synth.cloud_gpu import make_cloud_batch_gpu
    spec = [dict(agents=4, n_kf=40, H=384, W=512, period=40, shift=51, n_inter=60, reverse_inter=True,
                 noise=0.01, outlier=0.15)]
    prob, pts, midx = make_cloud_batch_gpu(7, spec, device=str(dev), name="gauge-60")
    E, P = prob.num_edges, 384 * 512
    fw, bw = list(range(E - 120, E - 60)), list(range(E - 60, E))
    mij = torch.cat([midx[e * P:(e + 1) * P] for e in fw])
    mji = torch.cat([midx[e * P:(e + 1) * P] for e in bw])
    pix_off = np.arange(prob.num_kf + 1, dtype=np.int64) * P
    args = (pts, C.F32, pix_off, prob.edge_i[fw], prob.edge_j[fw], mij, mji, prob.poses_init)
    C.gauge_sync(*args)  # warm-up
    kms, calls = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res, ms = C.gauge_sync(*args, timing=True)
        calls.append((time.perf_counter() - t) * 1e3)
        kms.append(ms)
    valid = sum(r["valid_i"] + r["valid_j"] for r in res)
    bytes_alg = 4 * 2 * P * len(fw) + 2 * 16 * valid
    k_ms = statistics.median(kms)
    peak, _ = measured_hbm_peak()
    ach = bytes_alg / (k_ms / 1e3) / 1e9
    return {"candidates": len(fw), "pixels_per_view": P, "valid_matches": int(valid),
            "admitted": int(sum(r["admitted"] for r in res)), "fallbacks": int(sum(r["fallback"] > 0 for r in res)),
            "call_ms": statistics.median(calls), "kernel_ms": k_ms,
            "roofline": {"kernel": "align_reduce (mixed)", "bound": "hbm", "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_launch": int(bytes_alg),
                         "traffic": traffic_from_profile("align_reduce_gauge60_512x384.txt", "k_align.cu")}}


def measure_depth(C, torch, prob, iters: int = 10) -> dict:
    """Segment-level structure refinement (Sec. III-E) on the bench workload: 200 Voronoi
    segments per keyframe, per-segment range errors exp(N(0, 0.05)), `iters` Jacobi steps
    at the initial poses, mixed form.  The per-match pass is HBM-bound: 4 B per streamed
    pixel plus, per valid match, the two pixels' 20-B records (snapshot point and
    confidence, segment)."""
    import dataclasses
    from synth.segments import perturb_segment_ranges, problem_labels
    lab = problem_labels(prob, n_seg=200, seed=1)
    pix_off = np.concatenate([[0], np.cumsum(prob.pixels_of())])
    p = dataclasses.replace(prob, points=perturb_segment_ranges(prob.points, lab, pix_off, 0.05, seed=1))
    g = C.Graph(p, mode=C.MIXED)
    M = g.depth_setup(lab)
    poses = torch.tensor(p.poses_init, dtype=torch.float64, device="cuda")
    eta = torch.zeros(M, dtype=torch.float64, device="cuda")
    g.depth_refine(poses, eta, 2)  # warm-up
    eta.zero_()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    _, tr, match_ms = g.depth_refine(poses, eta, iters, timing=True)
    ev1.record()
    ev1.synchronize()
    call_ms = ev0.elapsed_time(ev1)
    g.close()
    valid = p.valid_matches()
    bytes_alg = 4 * int(p.pixels_of()[p.edge_i].sum()) + 40 * valid
    peak, _ = measured_hbm_peak()
    ach = bytes_alg / (match_ms / 1e3) / 1e9
    return {"segments": M, "iters": iters, "cost_first": float(tr[0]), "cost_last": float(tr[-1]),
            "call_ms": call_ms, "ms_per_iter": call_ms / (iters + 1), "match_ms": match_ms,
            "roofline": {"kernel": "depth_match (mixed)", "bound": "hbm", "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_launch": int(bytes_alg),
                         "traffic": traffic_from_profile("depth_match_two_agent_40kf_512x384.txt", "k_depth.cu")}}


def measure_front(C, torch, reps: int = 20) -> dict:
    """Front-end kernels (Sec. III-A) on a 512x384 pair with dense predicted pointmaps
    (shared-canvas generator, seed 82, 1 % noise): projective ray matching of all 196,608
    pixels of a keyframe into the frame (start = same pixel), and confidence-weighted
    fusion of one prediction into the keyframe's map (FP32: read 2 x 16 B, write 16 B per
    pixel), one keyframe per call and 80 keyframes in one packed call."""
    from synth import make_cloud_problem, pose_from_matrix, pose_matrix, random_pose
    p = make_cloud_problem(82, [dict(agents=1, n_kf=3, H=384, W=512, period=40, shift=51, n_inter=0, noise=0.01,
                                     outlier=0.0)], dtype=np.float32)
    P = 384 * 512
    i, j = int(p.edge_i[0]), int(p.edge_j[0])
    Tji = np.linalg.inv(pose_matrix(p.poses_init[j])) @ pose_matrix(p.poses_init[i])
    Xi = p.points[i * P:(i + 1) * P].astype(np.float64)
    q = np.concatenate([Xi[:, :3] @ Tji[:3, :3].T + Tji[:3, 3], Xi[:, 3:4]], 1).astype(np.float32)
    frame = torch.from_numpy(np.ascontiguousarray(p.points[j * P:(j + 1) * P])).cuda()
    qd = torch.from_numpy(q).cuda()
    init = torch.arange(P, dtype=torch.int32, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m = C.project_match(frame, 384, 512, qd, init=init)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        m = C.project_match(frame, 384, 512, qd, init=init)
    ev1.record()
    ev1.synchronize()
    match_ms = ev0.elapsed_time(ev1) / reps
    canon = frame.clone()
    T = pose_from_matrix(np.linalg.inv(Tji))
    C.fuse(canon, qd, T)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        C.fuse(canon, qd, T)
    ev1.record()
    ev1.synchronize()
    fuse_ms = ev0.elapsed_time(ev1) / reps
    peak, _ = measured_hbm_peak()
    fuse_gbs = 48 * P / (fuse_ms / 1e3) / 1e9
    # many keyframes per call: the 80 maps of a 2 x 40 team at 512 x 384 (FP32, 755 MB of
    # reads and writes per call, far beyond L2), each fused with its own pose
    nk = 80
    gen = torch.Generator(device="cuda").manual_seed(7)
    bc = torch.rand((nk * P, 4), device="cuda", generator=gen) + torch.tensor([0.0, 0.0, 5.0, 1.0], device="cuda")
    bp = torch.rand((nk * P, 4), device="cuda", generator=gen) + torch.tensor([0.0, 0.0, 5.0, 0.5], device="cuda")
    rng = np.random.default_rng(8)
    bT = np.stack([random_pose(rng) for _ in range(nk)])
    boff = np.arange(nk + 1, dtype=np.int64) * P
    C.fuse_packed(bc, bp, boff, bT)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        C.fuse_packed(bc, bp, boff, bT)
    ev1.record()
    ev1.synchronize()
    packed_ms = ev0.elapsed_time(ev1) / reps
    packed_gbs = 48 * nk * P / (packed_ms / 1e3) / 1e9
    del bc, bp
    return {"pixels": P, "match_ms": match_ms, "mqueries_per_s": P / (match_ms / 1e3) / 1e6,
            "valid_fraction": float((m >= 0).float().mean().item()),
            "match_bound": "latency (a dependent walk on the ray image; the image stays in L2)",
            "fuse_ms": fuse_ms, "fuse_roofline": {"bound": "hbm", "achieved": fuse_gbs, "peak": peak,
                                                  "unit": "GB/s", "frac": fuse_gbs / peak,
                                                  "algorithmic_bytes_per_launch": 48 * P},
            "fuse_packed": {"keyframes": nk, "ms": packed_ms,
                            "roofline": {"bound": "hbm", "achieved": packed_gbs, "peak": peak, "unit": "GB/s",
                                         "frac": packed_gbs / peak, "algorithmic_bytes_per_launch": 48 * nk * P}}}


_SAMPLE = None


def _sample_init(path):
    """Worker of the oracle legs: the sampled edges and the solve's system loaded once (the
    parent spawned it with one BLAS / OpenMP thread)."""
    global _SAMPLE
    z = np.load(path, allow_pickle=True)
    _SAMPLE = (z["edges"].tolist(), z["solve"].item())


def _sample_edge(k):
    from oracle import como3r_oracle as O
    Ti, Tj, Pi, Pj, params = _SAMPLE[0][k]
    O.linearize_edge(Ti, Tj, Pi, Pj, params)
    return k


def _sample_solve(_):
    from oracle import como3r_oracle as O
    s = _SAMPLE[1]
    t = time.perf_counter()
    tau, _, _ = O.damped_solve(s["H"], s["g"], s["anchor"], s["lam"], s["eps0"], s["max_attempts"])
    O.retract(s["poses"], 1e-3 * tau)
    return time.perf_counter() - t


def _oracle_pool(n, path):
    """n spawned workers, each single-threaded (BLAS / OpenMP thread counts set in the
    environment they start with), loaded with the sample."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        pool = mp.get_context("spawn").Pool(n, initializer=_sample_init, initargs=(path,))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    pool.map(_sample_edge, [0] * n, chunksize=1)  # every worker up and loaded
    return pool


def oracle_sample(prob, n_edges: int, offset: int = 0, all_cores: bool = True):
    """Time the FP64 oracle on a bounded sample of one iteration and extrapolate.

    Sample: `n_edges` edges (evenly spread) linearised with dense per-match Jacobians,
    plus the dense damped Cholesky solve and retraction of a system of the full size 7N.
    One iteration = sampled edge time x E / n_edges + solve + retraction.  Timed on one core
    (one single-threaded spawned process runs the oracle's own serial loop) and on all of
    the host's cores (one single-threaded spawned process per core takes the sampled edges;
    the solve stays serial), the core count from os.cpu_count().
    """
    from oracle import como3r_oracle as O
    arrs = O.problem_arrays(prob)
    T = [O.pose_to_matrix(p) for p in prob.poses_init]
    sel = np.unique(np.linspace(0, prob.num_edges - 1, n_edges).astype(int) + offset) % prob.num_edges
    edges = []
    for e in sel:
        i, j, m, n, Pi, Pj = O.edge_matches(prob, arrs, int(e))
        edges.append((T[i], T[j], Pi, Pj, prob.params()))
    rng = np.random.default_rng(0)
    n7 = 7 * prob.num_kf
    B = rng.normal(size=(n7, n7))
    solve = dict(H=B @ B.T / n7 + np.eye(n7), g=rng.normal(size=n7), anchor=int(prob.anchor[0]), lam=prob.lam,
                 eps0=prob.eps0, max_attempts=prob.max_attempts, poses=prob.poses_init)
    cores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.npz")
        blob = np.empty(len(edges), dtype=object)
        blob[:] = edges
        np.savez(path, edges=blob, solve=np.array(solve, dtype=object))
        with _oracle_pool(1, path) as pool:
            t0 = time.perf_counter()
            pool.map(_sample_edge, range(len(edges)), chunksize=len(edges))
            t_edges = time.perf_counter() - t0
            t_solve = pool.map(_sample_solve, [0])[0]
        t_iter = t_edges * prob.num_edges / len(sel) + t_solve
        out = {"value": 1.0 / t_iter, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"{len(sel)} of {prob.num_edges} edges linearised + full {n7}x{n7} dense solve and "
                          f"retraction ({t_edges + t_solve:.1f} s on one core), extrapolated to one GN iteration"),
               "seconds_per_iteration": t_iter}
        if all_cores and cores > 1:
            with _oracle_pool(cores, path) as pool:
                t0 = time.perf_counter()
                pool.map(_sample_edge, range(len(edges)), chunksize=1)
                t_par = time.perf_counter() - t0
            t_iter_all = t_par * prob.num_edges / len(sel) + t_solve
            out = dict(out, value=1.0 / t_iter_all, cores=cores, seconds_per_iteration=t_iter_all,
                       sample=(f"{len(sel)} of {prob.num_edges} edges linearised on {cores} cores ({t_par:.1f} s, "
                               f"one single-threaded spawned process per core) + the full {n7}x{n7} dense solve and "
                               f"retraction on one core ({t_solve:.1f} s), extrapolated to one GN iteration"),
                       one_core={"value": 1.0 / t_iter, "unit": UNIT, "cores": 1, "seconds_per_iteration": t_iter})
    return out


def measure_small(C, torch) -> dict:
    """The oracle-sized workload (2 agents x 6 keyframes, 64x48, FP64 storage, 14 edges, 10 %
    outliers, 10 iterations, seed 0): both GPU forms (launch-bound at this size), with the
    GPU poses' error against the stored FP64 oracle golden of the same inputs.  (The
    oracle's own time on it is part of the CPU baseline.)"""
    from tests.golden import fullsize as F
    prob = F.problem("two_agent_6kf")
    iters = prob.iters
    res = {"workload": "two_agent_6kf_64x48", "edges": prob.num_edges, "valid_matches_per_iter": prob.valid_matches(),
           "iters_per_step": iters}
    poses0 = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
    work = torch.empty_like(poses0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    finals = {}
    for name, mode in (("mixed", C.MIXED), ("fp64", C.PLAIN_FP64)):
        g = C.Graph(prob, mode=mode)
        for _ in range(3):
            work.copy_(poses0)
            g.solve(work, iters, trace=False)
        torch.cuda.synchronize()
        steps = 50
        ev0.record()
        for _ in range(steps):
            work.copy_(poses0)
            g.solve(work, iters, trace=False)
        ev1.record()
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        finals[name] = work.cpu().numpy()
        g.close()
        res[name] = {"gn_iters_per_s": iters / (ms / 1e3), "ms_per_step": ms}
    if os.path.exists(F.PATHS["two_agent_6kf"]):
        gold = F.load("two_agent_6kf")
        F.check_fingerprint(prob, gold)
        from tests.gpu_helpers import pose_err
        for name in ("mixed", "fp64"):
            e = pose_err(finals[name], gold["poses"])
            res[name]["error_vs_oracle"] = {"rotation_rad": e["rot"], "translation_rel": e["trans"],
                                            "scale_rel": e["scale"]}
    return res


def small_oracle_timing(iters: int = 10) -> dict:
    """CPU baseline on the small configuration: the FP64 oracle's whole solve on one core
    (one single-threaded spawned process)."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(1) as pool:
            _, t = pool.apply(_small_oracle_solve, (iters,))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"workload": "two_agent_6kf_64x48", "gn_iters_per_s": iters / t, "seconds": t, "cores": 1,
            "kind": "oracle", "sample": f"the whole {iters}-iteration solve"}


def _small_oracle_solve(iters):
    from oracle import como3r_oracle as O
    from synth import make_workload
    prob = make_workload("two_agent_6kf_64x48", seed=0)
    t = time.perf_counter()
    po, _ = O.gn_solve(prob, prob.poses_init, iters)
    return po, time.perf_counter() - t


def error_vs_golden(C, torch, prob, gold, iters: int) -> dict:
    """Both forms against a stored FP64 oracle golden of the same inputs: the assembled H and
    g at the initial poses (when stored) and the poses and final cost after `iters`
    iterations (rotation angle, translation relative to max(|t|, trajectory RMS radius),
    scale ratio, as the parity tests measure them)."""
    from tests.gpu_helpers import pose_err
    out = {}
    N = prob.num_kf
    for name, mode in (("mixed", C.MIXED), ("fp64", C.PLAIN_FP64)):
        r = {}
        poses = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
        g = C.Graph(prob, mode=mode)
        if "H_blocks" in gold:
            H = torch.zeros((7 * N, 7 * N), dtype=torch.float64, device="cuda")
            gv = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
            g.gn_step(poses.clone(), H, gv)
            Ho = np.zeros((7 * N, 7 * N))
            for (rr, cc), blk in zip(gold["H_block_rc"].astype(int), gold["H_blocks"]):
                Ho[7 * rr:7 * rr + 7, 7 * cc:7 * cc + 7] = blk.reshape(7, 7)
                if rr != cc:
                    Ho[7 * cc:7 * cc + 7, 7 * rr:7 * rr + 7] = blk.reshape(7, 7).T
            Hg = H.cpu().numpy()
            r["hessian_rel"] = float(np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho))
            r["gradient_rel"] = float(np.linalg.norm(gv.cpu().numpy() - gold["g"]) / np.linalg.norm(gold["g"]))
        st, trace, info = g.solve(poses, iters)
        g.close()
        err = pose_err(poses.cpu().numpy(), gold["poses"])
        r.update({"rotation_rad": err["rot"], "translation_rel": err["trans"], "scale_rel": err["scale"],
                  "final_cost_rel": float(abs(trace[-1, 0] / gold["trace"][-1] - 1.0)), "iters": iters})
        out[name] = r
    return out


def measure_team(C, torch, args) -> dict:
    """The batched mixed-precision workload: 4 agents x 150 keyframes at 512x384 with FP16
    storage (points and confidence), 952 edges (60 inter-agent), each edge's valid matches
    restricted to a column band covering U[0.2, 1] of the image (uneven edge sizes), 1 %
    depth noise, 15 % outliers; one persistent residual launch per iteration, the
    iterations replayed from a CUDA graph, the residual kernel autotuned.  Inputs:
    shared-canvas generator, seed 31 (about a minute on the host)."""
    from tests.golden import fullsize as F
    t = time.time()
    prob = F.problem("team_4x150_f16")
    gen_s = time.time() - t
    iters = F.ITERS["team_4x150_f16"]
    pts = torch.from_numpy(np.ascontiguousarray(prob.points)).cuda()
    idx = torch.from_numpy(np.ascontiguousarray(prob.match_idx)).cuda()
    poses0 = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
    work = torch.empty_like(poses0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"workload": "4 agents x 150 kf, 512x384 FP16, column-band masks U[0.2,1]", "keyframes": prob.num_kf,
           "edges": prob.num_edges, "valid_matches_per_iter": prob.valid_matches(), "iters_per_step": iters,
           "generate_s": gen_s}
    for name, mode, steps in (("mixed", C.MIXED, 5), ("fp64", C.PLAIN_FP64, 1)):
        g = C.Graph(prob, mode=mode, points=pts, match_idx=idx)
        work.copy_(poses0)
        g.solve(work, 2, trace=False)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            work.copy_(poses0)
            g.solve(work, iters, trace=False)
        ev1.record()
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        st = g.time_stages(poses0, reps=3)
        stats = g.stats()
        g.close()
        v = iters / (ms / 1e3)
        res[name] = {"gn_iters_per_s": v, "mresiduals_per_s": v * prob.valid_matches() / 1e6, "ms_per_step": ms,
                     "stages_ms": st, "k1_config": stats["block"] % 100, "solve_ctas": stats["solve_ctas"]}
    res["mixed_over_fp64"] = res["mixed"]["gn_iters_per_s"] / res["fp64"]["gn_iters_per_s"]
    peak, _ = measured_hbm_peak()
    bytes_alg = algorithmic_bytes(prob)
    k1_ms = res["mixed"]["stages_ms"]["residual_reduce"]
    ach = bytes_alg / (k1_ms / 1e3) / 1e9
    res["roofline"] = {"kernel": "residual_reduce (K1, mixed, FP16 storage)", "bound": "hbm", "achieved": ach,
                       "peak": peak, "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_launch": bytes_alg,
                       "k1_ms_per_launch": k1_ms}
    if os.path.exists(F.PATHS["team_4x150_f16"]):
        gold = F.load("team_4x150_f16")
        F.check_fingerprint(prob, gold)
        res["error_vs_oracle"] = error_vs_golden(C, torch, prob, gold, iters)
    del pts, idx
    torch.cuda.empty_cache()
    return res


def measure_adjoint_4x30(C, torch) -> dict:
    """The adjoint workload: 4 agents x 30 keyframes at 512x384 FP32 (180 edges), the refined
    cost after 8 iterations differentiated w.r.t. per-pixel log-range and confidence:
    unrolled vjp timing in both forms, the per-match adjoint kernel's roofline, and the
    gradients against the stored FP64 oracle golden (complex-step directional derivatives
    along two seeded directions, envelope derivatives and central differences of 64
    seeded pixels)."""
    from tests.golden import fullsize as F
    t = time.time()
    prob = F.problem("adjoint_4x30")
    gen_s = time.time() - t
    iters = F.ITERS["adjoint_4x30"]
    poses0 = torch.tensor(prob.poses_init, dtype=torch.float64, device="cuda")
    res = {"workload": "4 agents x 30 kf, 512x384 FP32", "edges": prob.num_edges, "iters": iters,
           "valid_matches_per_iter": prob.valid_matches(), "generate_s": gen_s}
    peak, _ = measured_hbm_peak()
    valid = prob.valid_matches()
    adj_bytes = algorithmic_bytes(prob) + 16 * valid
    grads = {}
    for name, mode in (("mixed", C.MIXED), ("fp64", C.PLAIN_FP64)):
        g = C.Graph(prob, mode=mode)
        parts = g.time_vjp(poses0, iters, reps=2)
        t_fwd = g.time_stages(poses0, reps=3)["iteration"] * iters
        for vm, vname in ((C.VJP_UNROLLED, "unrolled"), (C.VJP_ENVELOPE, "envelope")):
            st, gl, gc, loss = g.vjp(poses0, iters, vm)
            grads[(name, vname)] = (gl.double().cpu().numpy(), gc.double().cpu().numpy(), float(loss.sum()))
        g.close()
        adj_ms = parts["adjoint_match"] / max(iters, 1)
        res[name] = {"vjp_ms": parts["forward"] + parts["envelope"] + parts["backward"], "parts_ms": parts,
                     "forward_iterations_ms": t_fwd,
                     "match_kernel": {"bound": "hbm", "ms_per_launch": adj_ms,
                                      "achieved": adj_bytes / (adj_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                                      "frac": adj_bytes / (adj_ms / 1e3) / 1e9 / peak,
                                      "algorithmic_bytes_per_launch": int(adj_bytes)}}
    if os.path.exists(F.PATHS["adjoint_4x30"]):
        gold = F.load("adjoint_4x30")
        F.check_fingerprint(prob, gold)
        err = {}
        pix = gold["pixels"].astype(np.int64)
        for (name, vname), (gl, gc, loss) in grads.items():
            e = {"loss_rel": abs(loss / gold["loss"][0] - 1.0)}
            ref = gold["dir_unrolled"] if vname == "unrolled" else gold["dir_envelope"]
            dirs = []
            for seed, r in zip(gold["dir_seeds"], ref):
                rng = np.random.default_rng(int(seed))
                vl, vc = rng.normal(size=gl.size), rng.normal(size=gl.size)
                got = float(gl @ vl + gc @ vc)
                mag = float(np.abs(gl * vl).sum() + np.abs(gc * vc).sum())
                dirs.append(abs(got - r) / mag)
            e["directional_rel_max"] = max(dirs)  # relative to sum |g_p v_p|
            if vname == "envelope":
                env = gold["envelope"]
                scale = np.abs(env).max(axis=0)
                e["pixels_rel_max"] = float(max(np.abs(gl[pix] - env[:, 0]).max() / scale[0],
                                                np.abs(gc[pix] - env[:, 1]).max() / scale[1]))
            else:
                g_at = np.where(gold["fd_which"] == 0, gl[pix], gc[pix])
                keep = gold["fd_excluded"] == 0
                ex = gold["exact_idx"].astype(int)
                sc = float(np.abs(g_at).max())
                e["exact_pixels_rel_max"] = float(np.max(np.abs(g_at[ex] - gold["exact"]) /
                                                         np.maximum(np.abs(gold["exact"]), 1e-3 * sc)))
                e["central_difference"] = {
                    "pixels": int(len(pix)), "excluded_huber_branch": int((~keep).sum()), "step": 1e-4,
                    "noise_rms_at_exact_pixels": float(np.sqrt(np.mean((gold["fd"][ex] - gold["exact"]) ** 2))),
                    "spread_rms_vs_gradient": float(np.sqrt(np.mean((g_at - gold["fd"])[keep] ** 2)))}
            err[f"{name}_{vname}"] = e
        err["note"] = ("8 unconverged IRLS iterations amplify rounding: the mixed form's unrolled gradient differs "
                       "from the FP64 one at O(1) here (its envelope does not); the central differences are "
                       "noise-dominated (noise_rms vs derivatives of 0.05..2000) and agree within it")
        res["error_vs_oracle"] = err
    return res


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    rank, local_rank, world = rank_info()
    if rank != 0:
        return
    from synth import make_workload
    prob = make_workload(args.workload, seed=args.seed)
    # each step: a bounded sample of one GN iteration (a few edges, rotating over the edge
    # list, plus the full dense solve), sized so that the whole run stays within minutes
    n_edges = 1 if args.steps + args.warmup > 24 else 4
    for w in range(args.warmup):
        oracle_sample(prob, n_edges, offset=w, all_cores=False)
    t0 = time.perf_counter()
    its, cores = [], []
    for k in range(args.steps):
        r = oracle_sample(prob, n_edges, offset=args.warmup + k, all_cores=False)
        its.append(r["seconds_per_iteration"])
        cores.append(r["cores"])
    wall = time.perf_counter() - t0
    value = 1.0 / float(np.mean(its))
    cb = {"value": value, "unit": UNIT, "cores": int(max(cores)), "kind": "oracle",
          "sample": (f"per step {n_edges} of {prob.num_edges} edges linearised (rotating) + the full "
                     f"{7 * prob.num_kf}x{7 * prob.num_kf} dense solve and retraction, extrapolated to one "
                     f"GN iteration; {args.steps} steps in {wall:.1f} s")}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "iters": prob.iters, "keyframes": prob.num_kf,
                      "edges": prob.num_edges, "valid_matches": prob.valid_matches(), "seed": args.seed},
           "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import torch
    rank, local_rank, world = rank_info()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local_rank))
    from paper_2605_30488_b300 import build as b
    if rank == 0 or world == 1:
        b.build()
    if dist:
        dist.barrier()
    from paper_2605_30488_b300 import como3r as C
    from synth import make_workload

    if args.only == "front":
        if rank == 0:
            print(json.dumps({"front_end": measure_front(C, torch), "note": "profiling run (--only front)"}),
                  flush=True)
        return
    if args.only == "cfg5":
        if rank == 0:
            cfg5 = measure_cfg5(C, torch, torch.device("cuda", local_rank), args.batch_reps)
            print(json.dumps({"cfg5": cfg5, "note": "profiling run (--only cfg5)"}), flush=True)
        return
    if args.only in ("team", "adjoint4"):
        if rank == 0:
            r = measure_team(C, torch, args) if args.only == "team" else measure_adjoint_4x30(C, torch)
            print(json.dumps({args.only: r, "note": f"profiling run (--only {args.only})"}), flush=True)
        return
    if args.only == "gauge":
        if rank == 0:
            gauge = measure_gauge(C, torch, torch.device("cuda", local_rank))
            print(json.dumps({"gauge_sync": gauge, "note": "profiling run (--only gauge)"}), flush=True)
        return
    prob = make_workload(args.workload, seed=args.seed)
    if args.only == "depth":
        if rank == 0:
            print(json.dumps({"depth_refine": measure_depth(C, torch, prob), "note": "profiling run (--only depth)"}),
                  flush=True)
        return
    iters = prob.iters
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id
    clocks = ClockSampler(gpu_id)
    clocks.start()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if not dist:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    poses0 = torch.tensor(prob.poses_init, dtype=torch.float64, device=dev)
    work = torch.empty_like(poses0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- mixed form, inputs resident in HBM (headline)
    g = C.Graph(prob, mode=C.MIXED)
    for _ in range(args.warmup):
        work.copy_(poses0)
        g.solve(work, iters, trace=False)
    barrier()
    launches = 0
    tw0 = time.time()
    torch.cuda.nvtx.range_push("como3r_timed")  # lets ncu select the timed launches (--nvtx-include)
    ev0.record()
    for _ in range(args.steps):
        work.copy_(poses0)
        st, _, info = g.solve(work, iters, trace=False)
        launches += g.last_launch_count()
    ev1.record()
    barrier()
    torch.cuda.nvtx.range_pop()
    tw1 = time.time()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    final_cost = info[0]["cost"]
    stages = g.time_stages(poses0, reps=20)
    stats = g.stats()
    g.close()
    value = world * args.steps * iters / (ms / 1e3)
    valid = prob.valid_matches()

    if args.only == "mixed":
        clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
                              "stages_ms": stages, "note": "profiling run (--only mixed)"}), flush=True)
        return

    # ---- plain FP64 form (same storage, same bytes)
    gp = C.Graph(prob, mode=C.PLAIN_FP64)
    work.copy_(poses0)
    gp.solve(work, iters, trace=False)
    barrier()
    psteps = max(2, min(args.steps, 5))
    ev0.record()
    for _ in range(psteps):
        work.copy_(poses0)
        gp.solve(work, iters, trace=False)
    ev1.record()
    barrier()
    pms = max_over_ranks(ev0.elapsed_time(ev1))
    pstages = gp.time_stages(poses0, reps=3)
    gp.close()
    plain_value = world * psteps * iters / (pms / 1e3)

    # ---- e2e: C ABI with pinned host buffers, uploads and readback inside the timed region
    pts_h = torch.from_numpy(np.ascontiguousarray(prob.points)).pin_memory()
    idx_h = torch.from_numpy(np.ascontiguousarray(prob.match_idx)).pin_memory()
    poses_h = torch.tensor(prob.poses_init, dtype=torch.float64).pin_memory()
    ge = C.Graph(prob, mode=C.MIXED, points=pts_h, match_idx=idx_h, copy_inputs=True)
    esteps = max(3, min(args.steps, 50))
    for _ in range(max(1, min(args.warmup, 3))):
        poses_h.copy_(torch.from_numpy(prob.poses_init))
        ge.update_inputs(pts_h, idx_h)
        ge.solve(poses_h, iters, trace=False)
    barrier()
    ev0.record()
    for _ in range(esteps):
        poses_h.copy_(torch.from_numpy(prob.poses_init))
        ge.update_inputs(pts_h, idx_h)
        ge.solve(poses_h, iters, trace=True)
    ev1.record()
    barrier()
    ems = max_over_ranks(ev0.elapsed_time(ev1))
    ge.close()
    e2e_serial = world * esteps * iters / (ems / 1e3)
    h2d = pts_h.numel() * pts_h.element_size() + idx_h.numel() * idx_h.element_size() + poses_h.numel() * 8
    d2h = poses_h.numel() * 8 + (iters + 1) * prob.num_graphs * 8
    # pipelined: two graphs on two streams, each step still uploading its inputs and reading
    # its poses and cost trace back, so that one step's upload overlaps the other's solve
    e2e_value, e2e_pipe_steps = pipelined_e2e(C, torch, prob, pts_h, idx_h, iters, esteps, args.warmup, barrier,
                                              max_over_ranks)
    e2e_value *= world

    # ---- adjoint (gradient of the refined cost w.r.t. per-pixel log-depth and confidence),
    # unrolled through the same iterations, mixed form
    ga = C.Graph(prob, mode=C.MIXED)
    vjp_parts = ga.time_vjp(poses0, iters, reps=3)
    ga.close()

    # ---- the secondary kernels; cfg5 (50 GB of device inputs) runs last: legs measured after
    # it were up to 40 % slower than on their own (the gauge kernel 0.243 vs 0.176 ms)
    gauge = None if args.no_batch else measure_gauge(C, torch, dev)
    depth = measure_depth(C, torch, prob)
    front = measure_front(C, torch)
    # the mixed and FP64 forms against the stored FP64 oracle golden of this workload
    from tests.golden import fullsize as F
    golden_err = None
    if args.workload == "two_agent_40kf_512x384" and args.seed == 0 and os.path.exists(F.PATHS["two_agent_40kf"]):
        gold = F.load("two_agent_40kf")
        F.check_fingerprint(prob, gold)
        golden_err = error_vs_golden(C, torch, prob, gold, iters)
    small = measure_small(C, torch)
    team = None if args.no_team else measure_team(C, torch, args)
    adj4 = None if args.no_team else measure_adjoint_4x30(C, torch)
    # ---- cfg5: a 64-graph batch in one launch per step, per-graph latency; the long chain
    cfg5 = None if args.no_batch else measure_cfg5(C, torch, dev, args.batch_reps)

    clocks.stop()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_src = measured_hbm_peak()
    bytes_alg = algorithmic_bytes(prob)
    k1_ms = stages["residual_reduce"]
    achieved = bytes_alg / (k1_ms / 1e3) / 1e9
    traffic = k1_traffic_from_profile()
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_sample(prob, args.cpu_sample_edges)
        cpu.pop("seconds_per_iteration", None)
        cpu["cfg1_small"] = small_oracle_timing(small["iters_per_step"])
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "agents": 2, "keyframes": prob.num_kf, "edges": prob.num_edges,
                   "pointmap": "512x384 FP32", "iters_per_step": iters, "valid_matches_per_iter": valid,
                   "seed": args.seed, "l2": "inputs larger than L2 (points+matches %.0f MB > 126 MB)"
                   % ((prob.points.nbytes + prob.match_idx.nbytes) / 1e6),
                   "parallelism": f"replicas x{world}"},
        "mresiduals_per_s": value * valid / 1e6,
        "plain_fp64": {"value": plain_value, "unit": UNIT, "ms_per_step": pms / psteps,
                       "mresiduals_per_s": plain_value * valid / 1e6,
                       "k1_ms": pstages["residual_reduce"], "stages_ms": pstages},
        "mixed_over_plain": value / plain_value,
        "stages_ms": stages,
        "final_cost": final_cost,
        "roofline": {"kernel": "residual_reduce (K1, mixed)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_source": f"{peak_src} hbm_gbs (copy)", "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_alg,
                     "k1_ms_per_launch": k1_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "pipeline": "2 graphs on 2 streams (one host thread each), %d steps" % e2e_pipe_steps,
                "serial": e2e_serial,
                "steps": esteps},
        "gpu_launches": int(launches),
        "clocks": clocks.summary(tw0, tw1),
        "plan": {k: stats[k] for k in ("items", "chunk", "block", "grid", "blocks", "updates", "levels",
                                       "smem_solve")},
    }
    # per-match adjoint kernel: K1's bytes plus four 4-byte atomic adds per valid match
    adj_bytes = bytes_alg + 16 * valid
    adj_ms = vjp_parts["adjoint_match"] / max(iters, 1)
    adj_gbs = adj_bytes / (adj_ms / 1e3) / 1e9
    out["adjoint"] = {"mode": "unrolled, mixed", "iters": iters,
                      "vjp_ms": vjp_parts["forward"] + vjp_parts["envelope"] + vjp_parts["backward"],
                      "parts_ms": vjp_parts, "forward_solve_ms": ms / args.steps,
                      "match_kernel": {"bound": "hbm", "ms_per_launch": adj_ms, "achieved": adj_gbs, "peak": peak,
                                       "unit": "GB/s", "frac": adj_gbs / peak,
                                       "algorithmic_bytes_per_launch": int(adj_bytes)}}
    # K3: FP64 operations of one factorisation + solve (from the plan) over its measured time
    flops = float(stats["solve_flops"])
    out["factor_solve"] = {"bound": "latency (dependent FP64 chains along the elimination tree)",
                           "flops_per_solve": flops, "ms": stages["factor_solve"],
                           "gflops": flops / (stages["factor_solve"] / 1e3) / 1e9,
                           "levels": stats["levels"], "ctas_per_graph": stats["solve_ctas"],
                           "fp64_nominal_tflops": 1.25}
    if cfg5 is not None:
        out["cfg5"] = cfg5
    if gauge is not None:
        out["gauge_sync"] = gauge
    out["depth_refine"] = depth
    out["front_end"] = front
    if golden_err is not None:
        out["mixed_error_vs_oracle"] = dict(golden_err, reference="FP64 oracle golden (tests/golden), same inputs",
                                            targets={"fp64": 1e-9, "mixed": 1e-5})
    out["cfg1_small"] = small
    if team is not None:
        out["cfg3_team_f16"] = team
    if adj4 is not None:
        out["cfg4_adjoint"] = adj4
    if cpu is not None:
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
