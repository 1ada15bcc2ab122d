"""Seeded synthetic inputs for ProbeWalk: graphs in CSR form and query streams.

This module is shared by the oracle, the tests, the CUDA path and the bench.
It holds none of the estimator's arithmetic: it only builds undirected simple
graphs (as sorted CSR arrays) and draws query pairs, error targets, seeds and
arrival times from numpy's seeded generators.
"""

from .graphs import (  # noqa: F401
    CSRGraph,
    barabasi_albert,
    complete_graph,
    cycle_graph,
    er_cycle,
    from_edges,
    grid_deleted,
    path_graph,
    rmat,
    rmat_native,
    workload_graph,
)
from .queries import (  # noqa: F401
    eps_choice,
    eps_uniform,
    poisson_arrivals,
    query_seeds,
    uniform_pairs,
)
