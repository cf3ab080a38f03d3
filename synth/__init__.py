"""Seeded synthetic correlation-function workloads.

This module only *describes* inputs: the leaf tensors (shape, kind, seed) and
the stream of binary contraction requests that form each correlation
function's contraction trees.  It holds none of the method's arithmetic: it
does not deduplicate requests, schedule, simulate memory or contract
anything.  Both the CUDA path (through the C ABI) and the CPU oracle consume
the same description, each with its own DAG builder.
"""
from .workloads import (  # noqa: F401
    Leaf, Request, Workload, CONFIGS, BATCHED, BatchedRecipe, make_workload, leaf_data,
    ring_requests,
)
