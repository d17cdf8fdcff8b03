"""Seeded synthetic inputs shaped like the paper's retrieval workloads.

This package only draws numbers (view features, query view counts, a codebook
fixture). It holds none of the matching method's arithmetic; the oracle tests
and the CUDA path both take their inputs from here.
"""
from .workload import (  # noqa: F401
    CONFIGS,
    Config,
    class_centres,
    shape_views,
    signed_views,
    query_views,
    kmeans_codebook,
    kmeans_init_rows,
    make_config_inputs,
    config_views,
    config_codebook,
    codebook_sample_shapes,
    second_measure,
    projection_matrix,
    upstream_grad,
    DIFF_WORKLOAD,
)
