"""Seeded synthetic matrices for GEMM tests and benchmarks.

This module only draws numbers: it holds none of the GEMM arithmetic and
none of the BF16 split, so the GPU library and the FP64 oracle can both be
fed from it without sharing any of the method's code.  Every generator is a
numpy PCG64 stream keyed by an integer seed, so the same seed gives the same
matrix on x86-64 and AArch64.

Distributions (the workloads the library is measured on):

* ``uniform``      -- i.i.d. U[lo, hi] (default U[-1, 1]).
* ``log_uniform``  -- sign-random log-uniform magnitudes: |x| = 2**u with
  u ~ U[emin, emax], sign +-1 with probability 1/2, drawn in FP64 and
  rounded to FP32 (default 2**[-10, 10]).
* ``normal``       -- i.i.d. N(0, std**2), e.g. std = 1/sqrt(K).
* ``integers``     -- integer values, i.i.d. uniform in [lo, hi]; sums of
  their products stay exact in FP32 while below 2**24.
* ``bf16_values``  -- a float32 matrix rounded to BF16-representable values
  by torch's CPU conversion (used to make native BF16 inputs).
"""
import numpy as np

DEFAULT_SEED = 0x5EED


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(shape, seed=DEFAULT_SEED, lo=-1.0, hi=1.0):
    return _rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def log_uniform(shape, seed=DEFAULT_SEED, emin=-10.0, emax=10.0):
    g = _rng(seed)
    u = g.uniform(emin, emax, size=shape)
    sign = np.where(g.random(size=shape) < 0.5, -1.0, 1.0)
    return (sign * np.exp2(u)).astype(np.float32)


def normal(shape, seed=DEFAULT_SEED, std=1.0):
    return (_rng(seed).standard_normal(size=shape) * std).astype(np.float32)


def integers(shape, seed=DEFAULT_SEED, lo=-8, hi=8):
    return _rng(seed).integers(lo, hi + 1, size=shape).astype(np.float32)


def bf16_values(x):
    """Round float32 values to the nearest BF16 values (returned as float32)
    with torch's CPU converter, and the raw BF16 bit patterns (uint16)."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    bits = t.view(torch.int16).numpy().view(np.uint16).copy()
    return t.to(torch.float32).numpy(), bits


def make(dist, shape, seed=DEFAULT_SEED, k=None):
    """Draw a matrix by distribution name ('uniform', 'log_uniform',
    'normal' (std 1/sqrt(k)), 'integers', 'ones')."""
    if dist == "uniform":
        return uniform(shape, seed)
    if dist == "log_uniform":
        return log_uniform(shape, seed)
    if dist == "normal":
        return normal(shape, seed, std=1.0 / np.sqrt(k if k else shape[-1]))
    if dist == "integers":
        return integers(shape, seed)
    if dist == "ones":
        return np.ones(shape, dtype=np.float32)
    raise ValueError("unknown distribution %r" % dist)
