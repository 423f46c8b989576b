"""Seeded synthetic workloads shaped like the paper's read sets and reference databases.

This package only draws random data (genomes, reads, read-versus-window pairs, arrival
times). It holds none of the classification arithmetic: no k-mers, minimizers, hashing,
clustering, edit-distance approximation or abundance maths. Both the CPU oracle and the
CUDA path consume what it produces, so it is the one module they share.
"""
from .workloads import (  # noqa: F401
    CONFIGS,
    Genomes,
    Reads,
    EdaPairs,
    config,
    make_genomes,
    make_reads,
    make_eda_pairs,
    make_arrivals,
    subsample_reads,
    Taxonomy,
    make_taxonomy,
    ascii_of,
    revcomp_ascii,
)
