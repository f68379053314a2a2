"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method (no right-hand side, no Runge-Kutta
step, no step-size control). It only builds problem inputs: the low-rank factors of
the physics kernels the paper studies, initial and sample states, and the recipe of
the batched workload. Both the CUDA path and the oracle take these as inputs.
"""
from .generators import (  # noqa: F401
    KERNELS,
    kernel_factors,
    monodisperse,
    sample_state,
    random_state,
    random_factors,
    batch_recipe,
    WORKLOADS,
)
