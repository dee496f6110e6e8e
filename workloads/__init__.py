"""Seeded synthetic workloads shared by the CUDA path, the oracle, the tests and the benchmark.

This package draws random numbers and builds problem descriptions. It holds none of the
method's arithmetic (no stencil, mapping, force or adjoint code), so the oracle and the CUDA
path can both take their inputs from here without sharing any implementation.
"""
from .synth import (  # noqa: F401
    BC_INFLOW_OUTFLOW,
    BC_PERIODIC,
    BC_PRESSURE,
    BC_WALL,
    CKPT_BF16,
    CKPT_BINOMIAL,
    CKPT_FP16,
    CKPT_FP32,
    CKPT_STORE_ALL,
    CKPT_UNIFORM,
    DOF_ROT,
    DOF_TX,
    DOF_TY,
    DOF_TZ,
    ROT_FREE,
    W_BILINEAR,
    W_COS4,
    Problem,
    config,
    config_names,
    gamma_2d,
    gamma_3d,
    inertia_tensor,
    initial_state,
    mass_properties,
    splitmix64_uniform,
    verification,
)
