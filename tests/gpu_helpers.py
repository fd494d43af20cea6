"""Shared helpers of the GPU parity tests (oracle side and comparisons)."""
import numpy as np

from oracle import como3r_oracle as O


def oracle_dense_without_anchor(prob, poses, graph=0):
    """The oracle's H, g of one graph with the fixed keyframes' rows/columns zeroed (as exported)."""
    H, g, E, recs = O.build_system(prob, poses, graph)
    H = H.copy(); g = g.copy()
    for a in O.component_anchors(prob, graph):
        H[7 * a:7 * a + 7, :] = 0.0
        H[:, 7 * a:7 * a + 7] = 0.0
        g[7 * a:7 * a + 7] = 0.0
    return H, g, E, recs


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def pose_err(pa, pb):
    return O.pose_errors(np.asarray(pa), np.asarray(pb))
