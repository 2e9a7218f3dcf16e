"""Seeded synthetic inputs for WCC refinement (graphs + input clusterings).

This module holds no part of the refinement's arithmetic: it only draws
random graphs and clusterings with numpy's PCG64 generator.  Both the oracle
tests and the CUDA-path tests/bench take their inputs from here.
"""
from .graphs import (Workload, planted_1k, lfr_like, dc_planted, tiny_family,  # noqa: F401
                     random_gnp, WORKLOADS)
