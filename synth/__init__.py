"""Seeded synthetic multi-agent pointmap scenes (inputs only).

This module produces the inputs both the CPU oracle and the CUDA library consume:
camera-frame pointmaps with per-pixel confidences, dense pixel correspondences per
edge, the edge list across agents, ground-truth and perturbed Sim(3) poses.  It holds
none of the refinement's arithmetic (no residual, Jacobian, Huber, solve or Sim(3)
exponential); poses are perturbed with a plain axis-angle rotation, a body-frame
offset and a scale factor.
"""
from .cloud import make_cloud_problem
from .cloud_gpu import graph_subproblem, make_cloud_batch_gpu
from .scene import (Problem, WORKLOADS, make_problem, make_workload, quat_from_matrix,
                    matrix_from_quat, pose_matrix, pose_from_matrix, random_pose)

__all__ = ["Problem", "WORKLOADS", "make_problem", "make_workload", "make_cloud_problem", "make_cloud_batch_gpu",
           "graph_subproblem", "quat_from_matrix", "matrix_from_quat", "pose_matrix", "pose_from_matrix", "random_pose"]
