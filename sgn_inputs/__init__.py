"""Seeded synthetic problem instances for the SGN hot path.

This package builds meshes, boundary conditions, loads, tracking targets and
initial design vectors.  It holds none of the method's arithmetic (no element
model, no derivatives, no linear algebra of the Gauss-Newton step); both the
CPU oracle and the CUDA path take their inputs from here.
"""
from .meshes import (grid2d, kuhn3d, Problem, problem_2d, problem_3d,
                     problem_tiny_2d, problem_tiny_3d, problem_batch2d, batch2d_instances, problem_rbf3d, draw_thetas, select_instances, PRESETS,
                     make_preset)

__all__ = ["grid2d", "kuhn3d", "Problem", "problem_2d", "problem_3d",
           "problem_tiny_2d", "problem_tiny_3d", "problem_batch2d", "batch2d_instances", "problem_rbf3d", "draw_thetas", "select_instances",
           "PRESETS", "make_preset"]
