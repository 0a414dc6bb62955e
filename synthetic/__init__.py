"""Seeded synthetic inputs for the nodal-density path.

This package produces plain arrays only (atom positions, Gaussian depths and
widths, the seeded additive noise potential, sampled nodes and their region
half-widths, solver settings).  It contains none of the method's arithmetic:
no potential sum, no stencil, no poles, no solver.  Both the oracle and the
CUDA library take their inputs from here, so that they see identical
workloads.
"""
from .rng import splitmix64, uniform01
from .workloads import Workload, make_workload, WORKLOADS

__all__ = ["splitmix64", "uniform01", "Workload", "make_workload", "WORKLOADS"]
