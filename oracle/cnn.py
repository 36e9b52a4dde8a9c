"""FP64 CPU oracle of the coefficient network (test infrastructure).

Only tests/ and bench.py's CPU-baseline leg may import this module.  The network maps a
(R, I) stamp pair [2][64][64] to n_out local kernel coefficients a_k (the local value of
Eq. 3's polynomials at the stamp, which Eq. 2 combines with the basis stamps):

    conv 3x3 (2 -> 32, stride 2, pad 1) -> ReLU
    conv 3x3 (32 -> 32, stride 2, pad 1) -> ReLU
    conv 3x3 (32 -> 32, stride 2, pad 1) -> ReLU
    conv 3x3 (32 -> 32, stride 1, pad 1) -> ReLU
    global average pool -> linear (32 -> n_out)

Convolution is cross-correlation, out[o][y][x] = b[o] + sum w[o][c][dy][dx]
in[c][s y + dy - 1][s x + dx - 1] (zero outside).  Loss = mean over batch and outputs of
(out - target)^2.  Forward and the hand-derived backward are written out per layer.

BF16 storage (`rounding=round_bf16`): the network stores its input, every post-ReLU
activation and every pre-activation gradient in BF16 and sums in FP32 or better; with
the rounding hook the oracle rounds the same values at the same points (everything else
stays FP64), so it computes what a BF16-storage network computes up to the summation
precision.  Without the hook it is the plain FP64 network.
Pins: finite differences of the loss (FP64), scipy correlate for the convolutions, torch
autograd for the network with BF16 storage, torch's BF16 conversion for round_bf16.
"""
from __future__ import annotations

import numpy as np

import starfield


def unflatten(params, n_out):
    out, o = [], 0
    for shp in starfield.cnn_param_shapes(n_out):
        n = int(np.prod(shp))
        out.append(np.asarray(params[o:o + n], dtype=np.float64).reshape(shp))
        o += n
    return out


def flatten(arrs):
    return np.concatenate([a.reshape(-1) for a in arrs])


def conv_fwd(x, w, b, stride):
    """x [B][C][H][W] -> [B][O][H/s][W/s] (pad 1, 3x3)."""
    B, C, H, W = x.shape
    O = w.shape[0]
    Ho, Wo = (H + 2 - 3) // stride + 1, (W + 2 - 3) // stride + 1
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, O, Ho, Wo))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + stride * (Ho - 1) + 1:stride, dx:dx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("bchw,oc->bohw", patch, w[:, :, dy, dx])
    return out + b[None, :, None, None]


def conv_bwd(x, w, dz, stride):
    """Gradients of conv_fwd given dL/dz: (dx, dw, db)."""
    B, C, H, W = x.shape
    Ho, Wo = dz.shape[2], dz.shape[3]
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            sl = (slice(None), slice(None), slice(dy, dy + stride * (Ho - 1) + 1, stride),
                  slice(dx, dx + stride * (Wo - 1) + 1, stride))
            dw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", dz, xp[sl])
            dxp[sl] += np.einsum("bohw,oc->bchw", dz, w[:, :, dy, dx])
    return dxp[:, :, 1:-1, 1:-1], dw, dz.sum(axis=(0, 2, 3))


def round_bf16(a):
    """Nearest BF16 value (8 significant bits), ties to even, as float64.  Values are
    taken to lie in BF16's normal range (no overflow or gradual underflow handling)."""
    m, e = np.frexp(np.asarray(a, dtype=np.float64))  # a = m 2^e, 1/2 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)       # rint: round half to even


def _identity(a):
    return a


def forward(params, x, n_out, rounding=None):
    """x [B][2][64][64] -> (out [B][n_out], cache).  rounding: applied to the stored
    input and activations (None: plain FP64)."""
    r = rounding or _identity
    p = unflatten(params, n_out)
    acts = [r(np.asarray(x, dtype=np.float64))]
    for li, (_, stride) in enumerate(starfield.CNN_LAYERS):
        z = conv_fwd(acts[-1], p[2 * li], p[2 * li + 1], stride)
        acts.append(r(np.maximum(z, 0.0)))
    pooled = acts[-1].mean(axis=(2, 3))
    out = pooled @ p[-2].T + p[-1]
    return out, (p, acts, pooled)


def loss_and_grad(params, x, target, n_out, rounding=None):
    """(loss, flat gradient) of the mean squared error.  rounding: also applied to the
    stored pre-activation gradients dL/dz (None: plain FP64)."""
    r = rounding or _identity
    out, (p, acts, pooled) = forward(params, x, n_out, rounding)
    B = out.shape[0]
    diff = out - np.asarray(target, dtype=np.float64)
    loss = float((diff ** 2).mean())
    dout = 2.0 * diff / diff.size
    grads = [None] * len(p)
    grads[-2] = dout.T @ pooled
    grads[-1] = dout.sum(axis=0)
    dpool = dout @ p[-2]
    a = acts[-1]
    da = np.broadcast_to(dpool[:, :, None, None] / (a.shape[2] * a.shape[3]), a.shape).copy()
    for li in range(len(starfield.CNN_LAYERS) - 1, -1, -1):
        stride = starfield.CNN_LAYERS[li][1]
        dz = r(da * (acts[li + 1] > 0.0))
        da, grads[2 * li], grads[2 * li + 1] = conv_bwd(acts[li], p[2 * li], dz, stride)
    return loss, flatten(grads)
