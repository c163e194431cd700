"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This package only draws random numbers with numpy; it holds none of the
method's arithmetic (no kernel evaluation, no factorisation, no solve).  Both
the CPU oracle and the CUDA path receive exactly the arrays produced here.
"""
from .synthetic import (  # noqa: F401
    Workload,
    make_c1_plain_fp64,
    make_c2_mixed,
    make_c3_batched,
    make_c4_krill,
    make_serving_request,
    make_serving_stream,
    uniform_centers,
    WORKLOADS,
)
