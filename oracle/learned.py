"""FP64 oracle of the learned coarse-correction network (test infrastructure only).

The paper has no learned component; this is the small 3-D convolution network
that the library trains and evaluates on the Q1 vertex grid.  Definitions:

* fields are channel-major ``[C, Nz, Ny, Nx]`` on an odd vertex grid;
* ``conv3d``: 3x3x3 taps, zero padding, stride 1 or 2, vertex-centred
  (output node i reads input nodes stride*i - 1 .. stride*i + 1), so a grid of
  N nodes goes to (N - 1) / stride + 1 nodes; weights ``[Cout, Cin, 3, 3, 3]``
  indexed (kz, ky, kx), plus a bias per output channel;
* ``upsample``: vertex-centred linear interpolation per axis, M -> 2M - 1
  nodes (even nodes copy, odd nodes average their two neighbours);
* the network (levels L, channels c_0..c_{L-1}):
      h = relu(conv(x, 4 -> c0)); s_0 = h = relu(conv(h, c0 -> c0))
      for l = 1..L-1: h = relu(conv_s2(h, c_{l-1} -> c_l)); s_l = h = relu(conv(h, c_l -> c_l))
      for l = L-2..0: h = relu(conv(up(h), c_{l+1} -> c_l)) + s_l; h = relu(conv(h, c_l -> c_l))
      y = conv(h, c0 -> 3)
* the flat parameter vector lists the layers in that order, each as W then b,
  W in the order [Cout][Cin][kz][ky][kx];
* loss per sample: ||y - t||^2 / ||t||^2.
The backward pass is written from these definitions (transposed convolution,
transposed interpolation, relu masks) and pinned against central differences.
"""
import itertools

import numpy as np


def conv3d(x, W, b, stride=1):
    Cin, Nz, Ny, Nx = x.shape
    Mz, My, Mx = (Nz - 1) // stride + 1, (Ny - 1) // stride + 1, (Nx - 1) // stride + 1
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((W.shape[0], Mz, My, Mx))
    for kz, ky, kx in itertools.product(range(3), repeat=3):
        sl = xp[:, kz:kz + stride * (Mz - 1) + 1:stride, ky:ky + stride * (My - 1) + 1:stride,
                kx:kx + stride * (Mx - 1) + 1:stride]
        out += np.einsum("oc,czyx->ozyx", W[:, :, kz, ky, kx], sl)
    return out + b[:, None, None, None]


def conv3d_backward(x, W, dy, stride=1):
    """Gradients (dx, dW, db) of conv3d for output gradient dy."""
    Cin, Nz, Ny, Nx = x.shape
    _, Mz, My, Mx = dy.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for kz, ky, kx in itertools.product(range(3), repeat=3):
        idx = (slice(None), slice(kz, kz + stride * (Mz - 1) + 1, stride), slice(ky, ky + stride * (My - 1) + 1, stride),
               slice(kx, kx + stride * (Mx - 1) + 1, stride))
        dW[:, :, kz, ky, kx] = np.einsum("ozyx,czyx->oc", dy, xp[idx])
        dxp[idx] += np.einsum("oc,ozyx->czyx", W[:, :, kz, ky, kx], dy)
    return dxp[:, 1:-1, 1:-1, 1:-1], dW, dy.sum(axis=(1, 2, 3))


def _up1(M):
    U = np.zeros((2 * M - 1, M))
    for i in range(M):
        U[2 * i, i] = 1.0
    for i in range(M - 1):
        U[2 * i + 1, i] = U[2 * i + 1, i + 1] = 0.5
    return U


def upsample(x):
    _, Mz, My, Mx = x.shape
    return np.einsum("Zz,Yy,Xx,czyx->cZYX", _up1(Mz), _up1(My), _up1(Mx), x)


def upsample_backward(dy):
    _, Nz, Ny, Nx = dy.shape
    Mz, My, Mx = (Nz + 1) // 2, (Ny + 1) // 2, (Nx + 1) // 2
    return np.einsum("Zz,Yy,Xx,cZYX->czyx", _up1(Mz), _up1(My), _up1(Mx), dy)


def layer_shapes(levels, ch, cin=4, cout=3):
    """(Cout, Cin, stride) of every convolution in network order."""
    L = [(ch[0], cin, 1), (ch[0], ch[0], 1)]
    for l in range(1, levels):
        L += [(ch[l], ch[l - 1], 2), (ch[l], ch[l], 1)]
    for l in range(levels - 2, -1, -1):
        L += [(ch[l], ch[l + 1], 1), (ch[l], ch[l], 1)]
    L.append((cout, ch[0], 1))
    return L


def unpack(theta, levels, ch):
    out, o = [], 0
    for co, ci, s in layer_shapes(levels, ch):
        W = theta[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = theta[o:o + co]
        o += co
        out.append((W, b, s))
    assert o == theta.size
    return out


def n_params(levels, ch):
    return sum(co * ci * 27 + co for co, ci, _ in layer_shapes(levels, ch))


def forward(theta, x, levels, ch, keep=False, store=None):
    """The network's output for input x.  ``store``, if given, is applied to every
    field an implementation keeps between layers -- the input, each ReLU output,
    each upsampled field and each skip sum -- to model the precision it stores
    them in (the output layer's field is not stored)."""
    P = unpack(np.asarray(theta, dtype=np.float64), levels, ch)
    keep_field = store if store is not None else (lambda v: v)
    tape = []
    k = 0

    def conv(h, relu):
        nonlocal k
        W, b, s = P[k]
        k += 1
        z = conv3d(h, W, b, s)
        y = keep_field(np.maximum(z, 0.0)) if relu else z
        tape.append((h, W, s, relu, y))
        return y
    h = conv(keep_field(x), True)
    h = conv(h, True)
    skips = [h]
    for _ in range(1, levels):
        h = conv(h, True)
        h = conv(h, True)
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        u = keep_field(upsample(h))
        tape.append(("up",))
        h = keep_field(conv(u, True) + skips[l])
        h = conv(h, True)
    y = conv(h, False)
    return (y, tape) if keep else y


def backward(theta, x, dy, levels, ch):
    """d(loss)/d(theta) for d(loss)/dy = dy (analytic, layer by layer)."""
    _, tape = forward(theta, x, levels, ch, keep=True)
    grads = [None] * sum(1 for t in tape if not isinstance(t[0], str))
    ci = len(grads) - 1
    # walk the tape backwards; skip connections need the gradient at s_l added
    skip_grad = {}
    g = dy
    ti = len(tape) - 1
    # output layer
    x_in, W, s, relu, y = tape[ti]
    gx, dW, db = conv3d_backward(x_in, W, g, s)
    grads[ci] = (dW, db)
    ci -= 1
    ti -= 1
    g = gx
    for l in range(0, levels - 1):
        # second conv of the up block (relu)
        x_in, W, s, relu, y = tape[ti]
        gz = g * (y > 0)
        gx, dW, db = conv3d_backward(x_in, W, gz, s)
        grads[ci] = (dW, db)
        ci -= 1
        ti -= 1
        # h = relu(conv(up)) + s_l : gradient goes to both
        skip_grad[l] = gx
        x_in, W, s, relu, y = tape[ti]
        gz = gx * (y > 0)
        gu, dW, db = conv3d_backward(x_in, W, gz, s)
        grads[ci] = (dW, db)
        ci -= 1
        ti -= 1
        assert isinstance(tape[ti][0], str)
        ti -= 1
        g = upsample_backward(gu)
    # encoder, deepest first
    for l in range(levels - 1, -1, -1):
        if l in skip_grad:
            g = g + skip_grad[l]
        for _ in range(2):
            x_in, W, s, relu, y = tape[ti]
            gz = g * (y > 0)
            g, dW, db = conv3d_backward(x_in, W, gz, s)
            grads[ci] = (dW, db)
            ci -= 1
            ti -= 1
    assert ti == -1 and ci == -1
    return np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


def loss(theta, x, t, levels, ch):
    y = forward(theta, x, levels, ch)
    return float(np.sum((y - t) ** 2) / np.sum(t ** 2))


def loss_grad(theta, x, t, levels, ch):
    y = forward(theta, x, levels, ch)
    dy = 2.0 * (y - t) / np.sum(t ** 2)
    return backward(theta, x, dy, levels, ch)


def init_params(levels, ch, seed=0):
    """He-normal weights, zero biases (the library draws its own with the same law)."""
    rng = np.random.default_rng(seed)
    parts = []
    for co, ci, _ in layer_shapes(levels, ch):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (ci * 27)), size=co * ci * 27))
        parts.append(np.zeros(co))
    return np.concatenate(parts)
