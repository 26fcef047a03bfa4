"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module draws random numbers and nothing else: it holds none of the
transform's arithmetic (no DFT, no decomposition, no redistribution), so that
the CUDA path and the CPU oracle can be fed identical values without sharing
any code that computes a result.

All arrays are drawn on the host with a seeded ``torch.Generator`` in float32
(the dtype the GPU path computes in); the oracle upcasts the same float32
values to float64.  Distributions follow the workloads of the paper's
benchmarks (cubic DNS-style grids, Sec. 4): i.i.d. uniform or normal values.
"""
from __future__ import annotations

import torch

# Shapes and virtual grids of the uneven-shape batch workload (48 transforms).
BATCH_SHAPES = (
    (64, 64, 64),
    (96, 96, 96),
    (128, 128, 128),
    (64, 128, 256),
    (160, 160, 160),
    (256, 256, 256),
)
BATCH_GRIDS = ((1, 2), (2, 2), (2, 4))


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def uniform_complex(shape, seed: int = 0) -> torch.Tensor:
    """complex64 array, real and imaginary parts i.i.d. U[-1, 1) (float32)."""
    g = _gen(seed)
    ri = torch.rand(*shape, 2, generator=g, dtype=torch.float32) * 2.0 - 1.0
    return torch.view_as_complex(ri)


def normal_complex(shape, seed: int = 0) -> torch.Tensor:
    """complex64 array, real and imaginary parts i.i.d. N(0, 1) (float32)."""
    g = _gen(seed)
    ri = torch.randn(*shape, 2, generator=g, dtype=torch.float32)
    return torch.view_as_complex(ri)


def normal_real(shape, seed: int = 0) -> torch.Tensor:
    """float32 array, i.i.d. N(0, 1)."""
    return torch.randn(*shape, generator=_gen(seed), dtype=torch.float32)


def uniform01_real(shape, seed: int = 1) -> torch.Tensor:
    """float32 array, i.i.d. U[0, 1) (the spectral weight of the loss)."""
    return torch.rand(*shape, generator=_gen(seed), dtype=torch.float32)


def batch_problems(count: int = 48, seed: int = 0):
    """Draw ``count`` (shape, grid) pairs uniformly with replacement."""
    g = _gen(seed)
    si = torch.randint(0, len(BATCH_SHAPES), (count,), generator=g)
    gi = torch.randint(0, len(BATCH_GRIDS), (count,), generator=g)
    return [(BATCH_SHAPES[int(a)], BATCH_GRIDS[int(b)]) for a, b in zip(si, gi)]
