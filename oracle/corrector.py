"""FP64 CPU oracle of the learned coarse-step corrector (test infrastructure only).

Only the test suite may import this module; the CUDA library never does.

The corrector is a small convolutional network applied to a field after each
coarse split-step (step length 4 dz, index screen averaged over the four fine
slices it replaces): the complex field enters as two real channels (real and
imaginary part), optionally with a third channel holding the averaged index
step, and

    Z1 = conv(X;  W1, b1),  A1 = relu(Z1)          (C_in -> 32)
    Z2 = conv(A1; W2, b2),  A2 = relu(Z2)          (32 -> 32)
    Z3 = conv(A2; W3, b3),  A3 = relu(Z3)          (32 -> 32)
    Z4 = conv(A3; W4, b4)                          (32 -> 2)
    out = X[:, :2] + sigma Z4                      (residual correction)

sigma is a fixed residual scale (the RMS size of the corrections the network
is trained to make, so that its outputs are of order one).

where conv is a 3 x 3 cross-correlation with periodic (circular) padding,
matching the periodic boundaries of the propagation:

    conv(X; W, b)[o, y, x] = b[o] + sum_{c, i, j} W[o, c, i, j] X[c, y+i-1, x+j-1].

Training minimises the mean squared error between ``out`` and the fine-step
field, L = sum (out - T)^2 / numel(T), by Adam.  The paper has no network; the
corrector is an addition of this library (it only motivates ML training data,
introduction).  Everything here is written from the definitions above:
forward pass, backpropagation by the chain rule, and the Adam update rule
(Kingma & Ba, 2015).  Arrays are float64, layout [batch][channel][y][x].

Parity status: pinned by tests/test_oracle_corrector.py (brute-force
convolution on tiny arrays, finite-difference gradients of the whole network,
the first Adam step against the closed form lr * sign(g)).
"""
from __future__ import annotations

import numpy as np

CHANNELS = 32
LAYERS = 4


def layer_shapes(c_in: int):
    """(C_out, C_in) of the four convolutions."""
    return [(CHANNELS, c_in), (CHANNELS, CHANNELS), (CHANNELS, CHANNELS), (2, CHANNELS)]


def param_count(c_in: int) -> int:
    return sum(o * i * 9 + o for o, i in layer_shapes(c_in))


def unflatten(theta: np.ndarray, c_in: int):
    """Split a flat parameter vector [W1, b1, W2, b2, W3, b3, W4, b4]."""
    out, k = [], 0
    for o, i in layer_shapes(c_in):
        W = theta[k:k + o * i * 9].reshape(o, i, 3, 3)
        k += o * i * 9
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    assert k == theta.size
    return out


def conv(X: np.ndarray, W: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    """3 x 3 cross-correlation with circular padding; X [B][C][H][W]."""
    Bn, C, H, Wd = X.shape
    O = W.shape[0]
    Y = np.zeros((Bn, O, H, Wd))
    for i in range(3):
        for j in range(3):
            # Xs[..., y, x] = X[..., y + i - 1, x + j - 1]
            Xs = np.roll(X, shift=(1 - i, 1 - j), axis=(2, 3))
            Y += np.einsum("oc,bcyx->boyx", W[:, :, i, j], Xs)
    if b is not None:
        Y += b[None, :, None, None]
    return Y


def conv_transpose(dY: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv in its input: dX[c, y, x] = sum_{o,i,j} W[o,c,i,j] dY[o, y-i+1, x-j+1]."""
    Bn, O, H, Wd = dY.shape
    C = W.shape[1]
    dX = np.zeros((Bn, C, H, Wd))
    for i in range(3):
        for j in range(3):
            dYs = np.roll(dY, shift=(i - 1, j - 1), axis=(2, 3))
            dX += np.einsum("oc,boyx->bcyx", W[:, :, i, j], dYs)
    return dX


def conv_weight_grad(X: np.ndarray, dY: np.ndarray):
    """dW[o,c,i,j] = sum_{b,y,x} dY[o,y,x] X[c, y+i-1, x+j-1];  db[o] = sum dY[o]."""
    C = X.shape[1]
    O = dY.shape[1]
    dW = np.zeros((O, C, 3, 3))
    for i in range(3):
        for j in range(3):
            Xs = np.roll(X, shift=(1 - i, 1 - j), axis=(2, 3))
            dW[:, :, i, j] = np.einsum("boyx,bcyx->oc", dY, Xs)
    return dW, dY.sum(axis=(0, 2, 3))


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) after rounding to float32:
    keep the upper 16 bits of the float32 pattern, adding half of the dropped
    part plus the kept part's lowest bit (round half to even)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta: np.ndarray, X: np.ndarray, sigma: float = 1.0, act_bf16: bool = False):
    """Network output and the intermediate tensors backpropagation needs.
    With ``act_bf16`` every convolution's input (the packed field and the
    three hidden activations) is rounded to bfloat16 first, the arithmetic
    of an inference engine that keeps activations in bfloat16 and
    accumulates exactly (here in float64)."""
    c_in = X.shape[1]
    layers = unflatten(theta, c_in)
    acts, pre = [X], []
    A = X
    for k, (W, b) in enumerate(layers):
        Z = conv(round_bf16(A) if act_bf16 else A, W, b)
        pre.append(Z)
        A = np.maximum(Z, 0.0) if k < LAYERS - 1 else Z
        acts.append(A)
    out = X[:, :2] + sigma * pre[-1]
    return out, acts, pre


def loss_and_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray, sigma: float = 1.0):
    """Mean squared error and its gradient with respect to the flat parameters."""
    c_in = X.shape[1]
    layers = unflatten(theta, c_in)
    out, acts, pre = forward(theta, X, sigma)
    r = out - T
    loss = float(np.sum(r * r) / r.size)
    dZ = 2.0 * sigma * r / r.size            # d loss / d Z4 (the residual path adds X)
    grads = [None] * LAYERS
    for k in range(LAYERS - 1, -1, -1):
        W, _ = layers[k]
        dW, db = conv_weight_grad(acts[k], dZ)
        grads[k] = (dW, db)
        if k > 0:
            dA = conv_transpose(dZ, W)
            dZ = dA * (pre[k - 1] > 0)
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat


def adam_step(theta, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
