"""The learned right preconditioner's network, its loss, gradient and Adam step, in NumPy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper preconditions GMRES from the right (Sec. 5.3, Ex. 3: GMRES on A P, x = P y); it
does not learn a preconditioner.  This network is the nonlinear right preconditioner used
with flexible GMRES (z_j = M(q_j), x = x0 + Z y), defined here by plain formulas:

* six 3x3 convolutions with zero padding (cross-correlation, as in every deep-learning
  library): out[co, y, x] = b[co] + sum_{ci, dy, dx} W[co, ci, dy, dx] in[ci, y + dy - 1, x + dx - 1],
  channels 2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU after the first five;
* input channels (r / rms(r), log kappa) on the H x W grid with rms(r) = ||r|| / sqrt(H W),
  output scaled by rms(r) (the map r -> A^{-1} r it imitates is linear, so M(c r) = c M(r)
  for c > 0 by construction);
* loss over a batch: mean_b ||F_b - t_b||^2 / ||t_b||^2 with F_b = out_b, or, for the
  residual-norm loss, F_b = A_b out_b with A_b the sample's 5-point operator (its rows as
  coefficients of the centre, west, east, north and south neighbours); with t_b = r_b this is
  ||A_b (out_b - A_b^{-1} r_b)||^2 / ||r_b||^2;
* Adam (Kingma & Ba, ICLR 2015, Alg. 1): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are one flat vector: for each layer its weights W[c_out][c_in][3][3], then its
biases b[c_out].  ``bf16=True`` rounds what the GPU keeps in bfloat16 (weights, activations,
activation gradients, the packed input) to bfloat16 at the same points, so the only
remaining difference is the order of the FP32 sums.
"""
from __future__ import annotations

import numpy as np

from .rgs import round_bf16

CHANNELS = [2, 32, 32, 32, 32, 32, 1]
NUM_LAYERS = 6


def layer_shapes():
    return [(CHANNELS[l + 1], CHANNELS[l]) for l in range(NUM_LAYERS)]


def num_params():
    return sum(co * ci * 9 + co for co, ci in layer_shapes())


def unflatten(p):
    """[(W (co, ci, 3, 3), b (co,)), ...] from the flat parameter vector."""
    out, o = [], 0
    for co, ci in layer_shapes():
        W = np.asarray(p[o:o + co * ci * 9], dtype=np.float64).reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = np.asarray(p[o:o + co], dtype=np.float64)
        o += co
        out.append((W, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def conv3x3(x, W, b=None):
    """out[n, co, y, x] = b[co] + sum W[co, ci, dy, dx] x[n, ci, y + dy - 1, x + dx - 1] (zero padding)."""
    B, C, H, Wd = x.shape
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + Wd])
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv3x3_input_grad(dout, W):
    """d(sum dout * conv3x3(x, W)) / dx: the correlation of dout with the flipped, transposed taps."""
    Wt = np.transpose(W[:, :, ::-1, ::-1], (1, 0, 2, 3))
    return conv3x3(dout, Wt)


def conv3x3_weight_grad(x, dout):
    """dW[co, ci, dy, dx] = sum_{n, y, x} dout[n, co, y, x] x[n, ci, y + dy - 1, x + dx - 1]."""
    B, C, H, Wd = x.shape
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dW = np.zeros((dout.shape[1], C, 3, 3))
    for dy in range(3):
        for dx in range(3):
            dW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", dout, xp[:, :, dy:dy + H, dx:dx + Wd])
    return dW


def _r(x, bf16):
    return round_bf16(x) if bf16 else x


def forward(p, x, bf16=False):
    """Network output (B, H, W) for input x (B, 2, H, W) and the activations of every layer."""
    layers = unflatten(p)
    if bf16:
        layers = [(round_bf16(W), np.asarray(b, dtype=np.float32).astype(np.float64)) for W, b in layers]
    acts = [_r(np.asarray(x, dtype=np.float64), bf16)]
    h = acts[0]
    for l, (W, b) in enumerate(layers):
        z = conv3x3(h, W, b)
        if l < NUM_LAYERS - 1:
            h = _r(np.maximum(z, 0.0), bf16)
            acts.append(h)
        else:
            out = z[:, 0]
    return out, acts, layers


def stencil_from_csr(csr, H, W):
    """(5, H, W) coefficients of a 5-point operator on an H x W grid (x fastest) from its CSR rows:
    centre, west (x - 1), east (x + 1), north (y - 1), south (y + 1)."""
    rowptr, colind, val = csr
    S = np.zeros((5, H * W))
    for p in range(H * W):
        for q in range(rowptr[p], rowptr[p + 1]):
            d = int(colind[q]) - p
            c = {0: 0, -1: 1, 1: 2, -W: 3, W: 4}[d]
            S[c, p] += val[q]
    return S.reshape(5, H, W)


def stencil_apply(S, v):
    """(A v)[y, x] for stencils S (B, 5, H, W) and fields v (B, H, W), zero outside the grid."""
    vp = np.zeros((v.shape[0], v.shape[1] + 2, v.shape[2] + 2))
    vp[:, 1:-1, 1:-1] = v
    return (S[:, 0] * v + S[:, 1] * vp[:, 1:-1, :-2] + S[:, 2] * vp[:, 1:-1, 2:]
            + S[:, 3] * vp[:, :-2, 1:-1] + S[:, 4] * vp[:, 2:, 1:-1])


def stencil_adjoint(S, g):
    """(A^T g): every row's coefficient sent back to the column it reads."""
    B, H, W = g.shape
    out = S[:, 0] * g
    out[:, :, 1:] += (S[:, 2] * g)[:, :, :-1]      # row (y, x-1) reads (y, x) through its east coefficient
    out[:, :, :-1] += (S[:, 1] * g)[:, :, 1:]      # row (y, x+1) through its west coefficient
    out[:, 1:, :] += (S[:, 4] * g)[:, :-1, :]      # row (y-1, x) through its south coefficient
    out[:, :-1, :] += (S[:, 3] * g)[:, 1:, :]      # row (y+1, x) through its north coefficient
    return out


def loss(out, t):
    """mean_b ||out_b - t_b||^2 / ||t_b||^2."""
    B = out.shape[0]
    e2 = ((out - t) ** 2).reshape(B, -1).sum(axis=1)
    t2 = (t ** 2).reshape(B, -1).sum(axis=1)
    return float(np.mean(e2 / t2))


def loss_grad(p, x, t, bf16=False, stencil=None):
    """(loss, flat gradient) by the chain rule through the layers, last to first."""
    out, acts, layers = forward(p, x, bf16)
    B = out.shape[0]
    F = out if stencil is None else stencil_apply(stencil, out)
    t2 = (t ** 2).reshape(B, -1).sum(axis=1)
    L = loss(F, t)
    scale = 2.0 / (t2 * B)
    if bf16:
        scale = scale.astype(np.float32).astype(np.float64)
    dF = (F - t) * scale[:, None, None]
    dout = dF if stencil is None else stencil_adjoint(stencil, dF)
    d = _r(dout, bf16)[:, None]                                      # dL / d out, (B, 1, H, W)
    grads = [None] * NUM_LAYERS
    for l in range(NUM_LAYERS - 1, -1, -1):
        W, _ = layers[l]
        h = acts[l]
        grads[l] = (conv3x3_weight_grad(h, d), d.sum(axis=(0, 2, 3)))
        if l > 0:
            d = _r(conv3x3_input_grad(d, W) * (h > 0), bf16)
    return L, flatten(grads)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v


def precondition(p, r, logkappa, bf16=False):
    """z = rms(r) net(r / rms(r), log kappa) for one residual r on the H x W grid (flattened)."""
    H, Wd = logkappa.shape
    rms = np.linalg.norm(r) / np.sqrt(H * Wd)
    if rms == 0:
        return np.zeros_like(r)
    if bf16:
        rms = float(np.float32(rms))
    x = np.stack([np.asarray(r).reshape(H, Wd) / rms, logkappa])[None]
    out, _, _ = forward(p, x, bf16)
    return rms * out[0].ravel()


def init_params(seed):
    """A random parameter vector (Kaiming-uniform weights, zero biases) from NumPy's PCG64."""
    rng = np.random.default_rng(seed)
    layers = []
    for co, ci in layer_shapes():
        bound = np.sqrt(6.0 / (9 * ci))
        layers.append((rng.uniform(-bound, bound, (co, ci, 3, 3)), np.zeros(co)))
    return flatten(layers)
