"""Seeded synthetic Ising instances shaped like the paper's workloads.

This module only draws instances: graphs, couplings and fields. It holds none
of the solver's arithmetic (no energies, no pruning, no gradients), so that the
CPU oracle and the CUDA library can both be fed from it without sharing any
method code. Every generator takes an explicit integer seed and uses numpy's
PCG64, so an instance is a pure function of its arguments.
"""

from .instances import (  # noqa: F401
    Instance,
    sk_dense,
    er_dense,
    er_graph_edges,
    regular_graph_edges,
    torus_edges,
    pendant_tree_edges,
    csr_from_edges,
    dense_from_edges,
    er_pendant_csr,
    torus_csr,
    regular_instance,
    table1_instance,
    table2_instance,
    random_sparse_instance,
    workload,
    serving_stream,
    serving_stream_pooled,
)
