"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the solver: it only draws random numbers
(numpy PCG64 via ``default_rng``) in a fixed order, so that the CUDA path and
the CPU oracle are fed the very same arrays.

HPCG generates its own operator (Section II-B), so the only drawn inputs are
right-hand sides, solution targets, the diagonal field kappa of the
differentiable form and the grid sizes of the uneven batch.
"""
import numpy as np


def normal(n, seed):
    """n draws of N(0,1)."""
    return np.random.default_rng(seed).standard_normal(n)


def uniform(n, lo, hi, seed):
    """n draws of U[lo, hi)."""
    return np.random.default_rng(seed).uniform(lo, hi, n)


def mixed_precision_xtrue(n, seed=1):
    """x_true ~ U[-1,1] for the mixed-precision workload (b = A x_true)."""
    return uniform(n, -1.0, 1.0, seed)


def multi_rhs(n, nrhs=32, seed=2):
    """nrhs right-hand sides ~ N(0,1), returned as an (nrhs, n) array, RHS-major draws."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, n))


def uneven_batch_dims(count=64, edges=(32, 48, 64, 80, 96), seed=3):
    """Grid edges for the uneven batch: 3*count draws from ``edges`` in order
    (instance-major, then x, y, z)."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(edges), size=(count, 3))


def differentiable_inputs(n, seed=4):
    """kappa ~ U[0,1], then b ~ N(0,1), then x_target ~ N(0,1), from one generator."""
    rng = np.random.default_rng(seed)
    kappa = rng.uniform(0.0, 1.0, n)
    b = rng.standard_normal(n)
    x_target = rng.standard_normal(n)
    return kappa, b, x_target
