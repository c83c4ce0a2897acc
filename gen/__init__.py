"""Seeded synthetic inputs for the blocked Floyd-Warshall APSP library.

This package only *shapes inputs*: point clouds, k-nearest-neighbour and
Erdos-Renyi edge lists, their dense adjacency matrices, and the serving
arrival trace.  It holds none of the shortest-path arithmetic.  Both the
CPU oracle (``oracle/``) and the CUDA path (``paper_1902_04446_gb300``) are
fed from here, and neither imports the other.

The paper measures on Erdos-Renyi graphs whose only relevant property is the
vertex count n (Sec. 5.1); the workloads below are kNN manifolds and ER
graphs of the same n range, built from a fixed seed.
"""
from .graphs import (  # noqa: F401
    INF32,
    INF16,
    swiss_roll,
    gaussian_mixture,
    knn_edges,
    int_weights,
    er_graph,
    dense_matrix,
    serving_trace,
    serving_request,
    workload,
    WORKLOADS,
)
