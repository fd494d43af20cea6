"""Full-size oracle goldens: the problems they are computed on, and their file format.

The FP64 oracle needs minutes to hours per full-size workload, too long to run inside a
GPU test, so `make_fullsize_goldens.py` (beside this file) runs it once and writes its
results here as text; the GPU tests and the bench regenerate the same seeded inputs and
compare against these files.  Every value in them comes from `oracle/` alone.

Workloads (all synthetic, seeded; the stand-ins for the paper's 512 x 384 pointmaps and
2-4 agent teams):
* two_agent_40kf  -- 2 agents x 40 keyframes, 512 x 384 FP32, 120 edges, 15 % outliers,
                     15 Gauss-Newton iterations (the bench workload);
* team_4x150_f16  -- 4 agents x 150 keyframes, 512 x 384 FP16 storage, 952 edges with 60
                     inter-agent ones, each edge's valid matches restricted to a column
                     band covering U[0.2, 1] of the image, 10 iterations (shared-canvas
                     generator: exact correspondences, generated in about a minute);
* adjoint_4x30    -- 4 agents x 30 keyframes, 512 x 384 FP32, 180 edges, 8 iterations,
                     the refined cost differentiated w.r.t. per-pixel log-range and
                     confidence;
* two_agent_6kf   -- the small configuration: 2 agents x 6 keyframes, 64 x 48 FP64, 14
                     edges, 10 iterations (seconds of the oracle; stored so that the bench
                     reads its errors against the oracle instead of running it).

A fingerprint of the inputs (valid match count, sum of the match indices, sums of the
stored point values) is stored with each golden, so a test can tell a changed input from
a changed result.
"""
from __future__ import annotations

import os
from typing import Dict

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

PATHS = {
    "two_agent_40kf": os.path.join(HERE, "fullsize_two_agent_40kf.txt"),
    "team_4x150_f16": os.path.join(HERE, "fullsize_team_4x150_f16.txt"),
    "adjoint_4x30": os.path.join(HERE, "fullsize_adjoint_4x30.txt"),
    "two_agent_6kf": os.path.join(HERE, "fullsize_two_agent_6kf.txt"),
}
ITERS = {"two_agent_40kf": 15, "team_4x150_f16": 10, "adjoint_4x30": 8, "two_agent_6kf": 10}


def problem(name: str):
    """The seeded inputs of a full-size golden (exactly what the script used)."""
    from synth import make_cloud_problem, make_workload
    if name == "two_agent_40kf":
        return make_workload("two_agent_40kf_512x384", seed=0)
    if name == "team_4x150_f16":
        spec = dict(agents=4, n_kf=150, H=384, W=512, period=100, shift=24, loop=0, n_inter=60, noise=0.01,
                    outlier=0.15, band=(0.2, 1.0))
        return make_cloud_problem(31, [spec], dtype=np.float16, iters=ITERS[name], name="team-4x150-f16-band")
    if name == "adjoint_4x30":
        return make_workload("four_agent_30kf_512x384", seed=0)
    if name == "two_agent_6kf":
        return make_workload("two_agent_6kf_64x48", seed=0)
    raise KeyError(name)


def fingerprint(prob) -> Dict[str, float]:
    pts = np.asarray(prob.points, dtype=np.float64)
    idx = np.asarray(prob.match_idx)
    return dict(valid=float((idx >= 0).sum()), idx_sum=float(idx.astype(np.int64).sum()),
                pts_sum=float(pts.sum()), pts_abs_sum=float(np.abs(pts).sum()))


def check_fingerprint(prob, gold: dict) -> None:
    """Raises AssertionError when the regenerated inputs are not the golden's inputs."""
    fp = fingerprint(prob)
    assert fp["valid"] == gold["fp_valid"][0] and fp["idx_sum"] == gold["fp_idx_sum"][0], \
        ("regenerated match indices differ from the golden's inputs", fp)
    for k in ("pts_sum", "pts_abs_sum"):
        assert abs(fp[k] - gold["fp_" + k][0]) <= 1e-12 * abs(gold["fp_" + k][0]) + 1e-9, \
            ("regenerated points differ from the golden's inputs", k, fp[k], gold["fp_" + k][0])


def write(path: str, header: str, entries: Dict[str, np.ndarray]) -> None:
    """One entry per line: `name d0 d1 ...: v v v ...` (values at full FP64 precision)."""
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        for name, v in entries.items():
            a = np.atleast_1d(np.asarray(v, dtype=np.float64))
            f.write(f"{name} {' '.join(str(d) for d in a.shape)}: {' '.join(repr(float(x)) for x in a.ravel())}\n")


def read(path: str) -> Dict[str, np.ndarray]:
    out = {}
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        head, vals = line.split(":", 1)
        parts = head.split()
        shape = tuple(int(d) for d in parts[1:])
        out[parts[0]] = np.array([float(x) for x in vals.split()], dtype=np.float64).reshape(shape)
    return out


def load(name: str) -> Dict[str, np.ndarray]:
    return read(PATHS[name])
