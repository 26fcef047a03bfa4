"""Spectral-weight loss and its gradient (oracle; test infrastructure only).

L(x) = sum_k |F(x)_k * w_k|^2 with F the paper-normalised forward transform
(Eq. multifft, 1/N on the forward) and w a real weight on the spectrum.

For complex x the gradient in the convention dL/dRe(x) + i dL/dIm(x) is
2 * F^H (w^2 * F x).  F = (1/N) D with D the unnormalised DFT, so the adjoint
is F^H = (1/N) D^H = (1/N) * backward (Eq. 2 has no scale on the backward).
"""
from __future__ import annotations

import math

import numpy as np

from . import dft


def loss(x: np.ndarray, w: np.ndarray) -> float:
    y = dft.fftn_forward(x)
    return float(np.sum(np.abs(y * w) ** 2))


def adjoint(y: np.ndarray) -> np.ndarray:
    """F^H y = (1/N) * backward(y)."""
    N = math.prod(y.shape)
    return dft.fftn_backward(y) / N


def grad(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dL/dRe(x) + i dL/dIm(x) = 2 F^H (w^2 F x)."""
    y = dft.fftn_forward(x)
    return 2.0 * adjoint((np.asarray(w, dtype=np.float64) ** 2) * y)


def central_difference(x, w, direction, h=1e-6) -> float:
    """(L(x + h d) - L(x - h d)) / (2 h): the directional derivative along d."""
    return (loss(x + h * direction, w) - loss(x - h * direction, w)) / (2.0 * h)
