"""Seeded synthetic inputs for circulant-embedding conditional simulation.

This package holds only input generation: observation sites, data values and
the problem parameters of each named workload.  It contains none of the
method's arithmetic (no circulant embedding, no Kriging, no covariance
matrices); both the CUDA path and the FP64 oracle take their inputs from here.
"""
from .synth import (  # noqa: F401
    batch_events,
    WORKLOADS,
    Workload,
    make_sites,
    se_study_sites,
    make_data,
    workload,
)
