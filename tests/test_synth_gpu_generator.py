"""The device-side shared-canvas generator (used for the 64-graph batch and the long
chain at full resolution), run here on the CPU device: its pointmaps and matches are
exact (the oracle's cost vanishes at ground truth without noise), it is deterministic
in its seed, and one graph extracted from a batch is the same data as the batch holds."""
import numpy as np
import torch

from oracle import como3r_oracle as O
from synth import graph_subproblem, make_cloud_batch_gpu
from synth.cloud_gpu import batch64_specs, chain2000_spec

SPECS = [dict(agents=2, n_kf=6, H=24, W=32, period=40, shift=4, n_inter=2),
         dict(agents=3, n_kf=5, H=16, W=20, period=30, shift=3, n_inter=2, loop=2)]


def test_noise_free_batch_has_zero_cost_at_ground_truth():
    prob, pts, midx = make_cloud_batch_gpu(3, SPECS, device="cpu", storage=torch.float64)
    assert prob.num_graphs == 2 and pts.shape[0] == prob.pixels_of().sum()
    for g in range(prob.num_graphs):
        sub = graph_subproblem(prob, pts, midx, g)
        assert (sub.match_idx >= -1).all() and (sub.match_idx < sub.height[0] * sub.width[0]).all()
        assert (sub.match_idx >= 0).mean() > 0.5
        c_gt = O.total_cost(sub, sub.poses_gt)[0]
        c_init = O.total_cost(sub, sub.poses_init)[0]
        assert c_init > 1.0
        assert c_gt <= 1e-18 * c_init


def test_fp32_storage_and_outliers():
    prob, pts, midx = make_cloud_batch_gpu(4, SPECS, device="cpu", noise=0.01, outlier=0.2)
    assert pts.dtype == torch.float32
    sub = graph_subproblem(prob, pts, midx, 0)
    # outliers make the cost at ground truth large, and confidences are lognormal(1, 0.5)
    assert O.total_cost(sub, sub.poses_gt)[0] > 1.0
    c = sub.points[:, 3].astype(np.float64)
    assert abs(np.log(c).mean() - 1.0) < 0.05 and abs(np.log(c).std() - 0.5) < 0.05


def test_deterministic_in_seed_and_subproblem_is_a_slice():
    a = make_cloud_batch_gpu(7, SPECS, device="cpu", noise=0.01, outlier=0.1)
    b = make_cloud_batch_gpu(7, SPECS, device="cpu", noise=0.01, outlier=0.1)
    c = make_cloud_batch_gpu(8, SPECS, device="cpu", noise=0.01, outlier=0.1)
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert not torch.equal(a[1], c[1])
    prob, pts, midx = a
    sub = graph_subproblem(prob, pts, midx, 1)
    k0 = int(prob.kf_offset[1])
    p0 = int(prob.pixels_of()[:k0].sum())
    assert np.array_equal(sub.points, pts[p0:p0 + sub.points.shape[0]].numpy())
    assert np.array_equal(sub.edge_i + k0, prob.edge_i[prob.edge_offset[1]:])
    assert sub.match_idx.size == sub.num_edges * int(sub.height[0]) * int(sub.width[0])


def test_cfg5_specs():
    specs = batch64_specs()
    assert len(specs) == 64
    assert {(s["H"], s["W"]) for s in specs} <= {(192, 256), (288, 384), (384, 512)}
    assert all(2 <= s["agents"] <= 4 and 10 <= s["n_kf"] <= 200 for s in specs)
    (chain,) = chain2000_spec()
    assert chain["n_kf"] == 2000 and chain["loop"] == 100 and (chain["H"], chain["W"]) == (384, 512)


def test_cloud_band_masks_keep_one_column_band_per_edge():
    """band=(lo, hi): every edge keeps matches only inside one column band of i (valid columns
    span at most the band, at least lo of the width is kept wherever the unmasked edge had
    matches everywhere), the pointmaps are unchanged, and the per-edge counts become uneven."""
    from synth import make_cloud_problem
    spec = dict(agents=2, n_kf=6, H=24, W=40, period=10, shift=4, n_inter=2, noise=0.01, outlier=0.0)
    a = make_cloud_problem(3, [spec])
    b = make_cloud_problem(3, [dict(spec, band=(0.2, 1.0))])
    np.testing.assert_array_equal(a.points, b.points)
    P, W = 24 * 40, 40
    ratios = []
    for e in range(b.num_edges):
        ib = b.match_idx[e * P:(e + 1) * P].reshape(24, W)
        ia = a.match_idx[e * P:(e + 1) * P].reshape(24, W)
        assert np.all((ib == ia) | (ib == -1))  # without outliers the kept matches are the exact ones
        cols = np.nonzero((ib >= 0).any(axis=0))[0]
        if cols.size:
            assert np.all(np.diff(cols) == 1)  # one contiguous band of columns
        ratios.append((ib >= 0).sum() / max((ia >= 0).sum(), 1))
    assert min(ratios) < 0.6 and max(ratios) > 0.6
