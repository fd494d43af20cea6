"""Host logic of the benchmark's roofline figures, without a GPU.

The algorithmic bytes of the residual kernel (4 B per streamed pixel for its match index,
plus the streamed and the gathered packed pixel per valid match) are recounted from a
seeded problem's own arrays, and the DRAM traffic of a committed ncu summary is used only
while the summary's recorded source hash matches the kernel source.
"""
import hashlib
import os
import shutil

import numpy as np

import bench
from synth import make_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_recounted_from_the_problem():
    for dtype, bpp in ((np.float32, 16), (np.float16, 8), (np.float64, 32)):
        prob = make_problem(4, agents=2, n_kf=4, H=12, W=16, f=10.0, n_inter=2, dtype=dtype)
        idx = np.asarray(prob.match_idx)
        expect, off = 0, 0
        for e in range(prob.num_edges):
            npix = int(prob.height[0]) * int(prob.width[0])  # one graph: every keyframe's pixel count
            rows = idx[off:off + npix]
            off += npix
            expect += 4 * npix + 2 * bpp * int((rows >= 0).sum())
        assert off == idx.size
        assert bench.algorithmic_bytes(prob) == expect, dtype


def test_profile_traffic_only_for_the_profiled_source(tmp_path):
    # the committed K1 summary matches the current source: its traffic is used
    t = bench.k1_traffic_from_profile()
    assert t is not None and t > 0
    # a summary recorded on another source hash gives none
    summary = tmp_path / "summary.txt"
    txt = open(bench.PROFILE).read()
    src_hash = hashlib.sha256(open(bench.K1_SOURCE, "rb").read()).hexdigest()
    assert src_hash in txt
    summary.write_text(txt.replace(src_hash, "0" * 64))
    assert bench.traffic_from_profile(str(summary), bench.K1_SOURCE) is None
    # the same summary against a copy of the source with one byte more gives none either
    src = tmp_path / "k.cu"
    shutil.copy(bench.K1_SOURCE, src)
    with open(src, "ab") as f:
        f.write(b"\n")
    summary.write_text(txt)
    assert bench.traffic_from_profile(str(summary), str(src)) is None
    assert bench.traffic_from_profile(str(summary), bench.K1_SOURCE) == t
