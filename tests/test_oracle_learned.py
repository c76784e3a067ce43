"""Pins of the network oracle: conv / upsample against direct definitions and
the analytic gradient against central finite differences."""
import itertools

import numpy as np
import pytest

from oracle import learned


def conv_direct(x, W, b, stride):
    Cin, Nz, Ny, Nx = x.shape
    M = [(n - 1) // stride + 1 for n in (Nz, Ny, Nx)]
    out = np.zeros((W.shape[0], *M))
    for o in range(W.shape[0]):
        for i, j, k in itertools.product(*[range(m) for m in M]):
            s = b[o]
            for kz, ky, kx in itertools.product(range(3), repeat=3):
                z, y, xx = stride * i + kz - 1, stride * j + ky - 1, stride * k + kx - 1
                if 0 <= z < Nz and 0 <= y < Ny and 0 <= xx < Nx:
                    s += np.dot(W[o, :, kz, ky, kx], x[:, z, y, xx])
            out[o, i, j, k] = s
    return out


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_matches_direct_loops(stride):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 7, 5))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    b = rng.normal(size=2)
    np.testing.assert_allclose(learned.conv3d(x, W, b, stride), conv_direct(x, W, b, stride), atol=1e-12)


def test_upsample_interpolates_linear_fields():
    z, y, x = np.meshgrid(np.arange(3.0), np.arange(4.0), np.arange(5.0), indexing="ij")
    f = (2 * x - y + 0.5 * z + 1)[None]
    up = learned.upsample(f)
    Z, Y, X = np.meshgrid(np.arange(5) / 2, np.arange(7) / 2, np.arange(9) / 2, indexing="ij")
    np.testing.assert_allclose(up[0], 2 * X - Y + 0.5 * Z + 1, atol=1e-13)
    # transpose identity <up x, y> = <x, up^T y>
    rng = np.random.default_rng(1)
    a = rng.normal(size=(2, 3, 4, 5))
    c = rng.normal(size=(2, 5, 7, 9))
    assert abs(np.sum(learned.upsample(a) * c) - np.sum(a * learned.upsample_backward(c))) < 1e-11


@pytest.mark.parametrize("levels,ch,N", [(2, (3, 4), 5), (3, (2, 3, 4), 9)])
def test_gradient_matches_central_differences(levels, ch, N):
    rng = np.random.default_rng(2)
    theta = learned.init_params(levels, ch, seed=3) + 0.05 * rng.normal(size=learned.n_params(levels, ch))
    x = rng.normal(size=(4, N, N, N))
    t = rng.normal(size=(3, N, N, N))
    g = learned.loss_grad(theta, x, t, levels, ch)
    idx = rng.choice(theta.size, size=40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (learned.loss(theta + e, x, t, levels, ch) - learned.loss(theta - e, x, t, levels, ch)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_storage_hook():
    """forward(store=...) applies the hook to every stored field: the identity
    reproduces the plain forward exactly; rounding every stored field to a 1/8 grid
    changes a random network's output, while on integer data through integer
    weights (every field already on that grid) it changes nothing."""
    levels, ch, N = 2, (4, 8), 5
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4, N, N, N))
    theta = learned.init_params(levels, ch, seed=4)
    y = learned.forward(theta, x, levels, ch)
    assert np.array_equal(learned.forward(theta, x, levels, ch, store=lambda v: v), y)
    grid = lambda v: np.round(np.asarray(v) * 8.0) / 8.0
    assert not np.array_equal(learned.forward(theta, x, levels, ch, store=grid), y)
    ti = np.zeros_like(theta)
    nz = rng.choice(theta.size, size=theta.size // 10, replace=False)
    ti[nz] = rng.choice([-1.0, 1.0], size=nz.size)
    xi = rng.integers(0, 4, size=(4, N, N, N)).astype(np.float64)
    yi = learned.forward(ti, xi, levels, ch)
    # upsampling halves odd nodes: integer fields stay on the 1/8 grid one level down
    assert np.array_equal(learned.forward(ti, xi, levels, ch, store=grid), yi)
    _, tape = learned.forward(ti, xi, levels, ch, keep=True, store=grid)
    assert all(np.array_equal(t[0], grid(t[0])) for t in tape if not isinstance(t[0], str))
