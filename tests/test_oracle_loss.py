"""Pins for oracle.loss: finite differences and the adjoint identity (CPU only)."""
import numpy as np

from oracle import dft, loss


def _crand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def check_gradient_fd(shape=(32, 32, 32), ndirs=20, grad_fn=None):
    """Central differences in FP64, h = 1e-6, along seeded complex directions:
    (L(x + h d) - L(x - h d)) / 2h = Re <grad, d>."""
    grad_fn = grad_fn or loss.grad
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    w = rng.random(shape)
    gr = grad_fn(x, w)
    for k in range(ndirs):
        d = _crand(shape, 100 + k)
        fd = loss.central_difference(x, w, d, h=1e-6)
        an = float(np.sum(gr.real * d.real + gr.imag * d.imag))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, fd, an)


def test_gradient_central_differences_32cubed():
    check_gradient_fd()


def test_adjoint_identity():
    """<F x, y> = <x, F^H y> for random x, y."""
    shape = (6, 10, 8)
    x, y = _crand(shape, 1), _crand(shape, 2)
    lhs = np.vdot(dft.fftn_forward(x), y)
    rhs = np.vdot(x, loss.adjoint(y))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_loss_of_delta():
    """x = delta at the origin: F x = 1/N everywhere, so L = sum w^2 / N^2."""
    shape = (4, 6, 5)
    N = 4 * 6 * 5
    x = np.zeros(shape, complex)
    x[0, 0, 0] = 1
    w = np.random.default_rng(3).random(shape)
    assert np.isclose(loss.loss(x, w), np.sum(w ** 2) / N ** 2, rtol=1e-13)
