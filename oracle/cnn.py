"""Oracle of the candidate classifier (test infrastructure only), arXiv
2606.27262 Sec. 3.2.2: two convolutional networks, one on the
frequency-time image and one on the DM-time image of a candidate, fused
multiplicatively into one probability, trained by binary cross-entropy.

Plain numpy in float64.  With ``bf16=True`` the values the GPU stores in
bfloat16 -- GEMM weights, each layer's ReLU output and each layer's output
gradient -- are rounded to bfloat16 (round to nearest even) at the same
points, so that the GPU's remaining differences are those of float32
accumulation.  Also the image features (frequency-time crop, DM-time sum
over shifted subbands, per-image standardisation) and the subband shift
table from Eq. 1.

Network per image: five 3x3 convolutions, stride 2, zero padding 1,
channels 1-16-32-64-128-256, ReLU after each; global average pooling; a
linear head to one logit.  p = sigmoid(l_ft) * sigmoid(l_dmt).
Flat parameter order: per image (frequency-time first), per layer
W[Cout][ky][kx][Cin] then b[Cout]; then head w[256] and b.
"""
from __future__ import annotations

import numpy as np

CIN = (1, 16, 32, 64, 128)
COUT = (16, 32, 64, 128, 256)
FEAT = 256
KDM = 4.148808e3


def bf16(x):
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def num_params_branch():
    return sum(co * 9 * ci + co for ci, co in zip(CIN, COUT)) + FEAT + 1


def unpack(flat):
    """Flat vector -> [branch][layer] (W [Cout][3][3][Cin], b) and heads."""
    flat = np.asarray(flat, np.float64)
    out, k = [], 0
    for _ in range(2):
        layers = []
        for ci, co in zip(CIN, COUT):
            w = flat[k:k + co * 9 * ci].reshape(co, 3, 3, ci)
            k += co * 9 * ci
            b = flat[k:k + co]
            k += co
            layers.append((w, b))
        hw = flat[k:k + FEAT]
        k += FEAT
        hb = flat[k]
        k += 1
        out.append((layers, hw, hb))
    return out


def pack(grads):
    parts = []
    for layers, hw, hb in grads:
        for w, b in layers:
            parts += [w.reshape(-1), b.reshape(-1)]
        parts += [hw.reshape(-1), np.array([hb])]
    return np.concatenate(parts)


def patches(x):
    """3x3, stride 2, padding 1 patches of x [N][H][W][C]:
    [N][Ho][Wo][3][3][C]."""
    n, h, w, c = x.shape
    xp = np.zeros((n, h + 2, w + 2, c))
    xp[:, 1:-1, 1:-1] = x
    ho, wo = h // 2, w // 2
    out = np.empty((n, ho, wo, 3, 3, c))
    for ky in range(3):
        for kx in range(3):
            out[:, :, :, ky, kx, :] = xp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :]
    return out


def conv(x, w, b):
    """Pre-activation z[n][ho][wo][co] = b[co] + sum_{ky,kx,c}
    x[n][2ho-1+ky][2wo-1+kx][c] w[co][ky][kx][c] (zero outside x)."""
    return np.einsum("nhwijc,oijc->nhwo", patches(x), w, optimize=True) + b


def conv_input_grad(dz, w, shape):
    """Adjoint of conv with respect to x."""
    n, h, wd, c = shape
    gp = np.einsum("nhwo,oijc->nhwijc", dz, w, optimize=True)
    dxp = np.zeros((n, h + 2, wd + 2, c))
    ho, wo = dz.shape[1], dz.shape[2]
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :] += gp[:, :, :, ky, kx, :]
    return dxp[:, 1:-1, 1:-1]


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def forward_backward(flat, ft, dmt, labels=None, round_bf16=True):
    """ft, dmt [N][H][W] images (the GPU's bf16 values).  Returns p [N] and,
    with labels, (loss, flat gradient)."""
    q = bf16 if round_bf16 else (lambda v: np.asarray(v, np.float64))
    params = unpack(flat)
    caches, logits = [], []
    for (layers, hw, hb), img in zip(params, (ft, dmt)):
        x = np.asarray(img, np.float64)[..., None]
        xs = []
        for w, b in layers:
            xs.append(x)
            x = q(np.maximum(conv(x, q(w), b), 0.0))
        feat = x.mean(axis=(1, 2))
        logits.append(feat @ hw + hb)
        caches.append((xs, x, feat))
    s1, s2 = sigmoid(logits[0]), sigmoid(logits[1])
    p = s1 * s2
    if labels is None:
        return p
    y = np.asarray(labels, np.float64)
    n = y.size
    pc = np.clip(p, 1e-7, 1 - 1e-7)
    loss = float(np.mean(-(y * np.log(pc) + (1 - y) * np.log(1 - pc))))
    g = (pc - y) / (1 - pc) / n
    dls = (g * (1 - s1), g * (1 - s2))
    grads = []
    for (layers, hw, hb), (xs, y5, feat), dl in zip(params, caches, dls):
        ghw = feat.T @ dl
        ghb = float(dl.sum())
        dfeat = dl[:, None] * hw[None, :]
        hh, ww = y5.shape[1], y5.shape[2]
        dz = q(np.broadcast_to(dfeat[:, None, None, :] / (hh * ww), y5.shape) * (y5 > 0))
        lg = [None] * len(layers)
        for li in range(len(layers) - 1, -1, -1):
            w, _ = layers[li]
            x_in = xs[li]
            db = dz.sum(axis=(0, 1, 2))
            dw = np.einsum("nhwo,nhwijc->oijc", dz, patches(x_in), optimize=True)
            lg[li] = (dw, db)
            if li > 0:
                dz = q(conv_input_grad(dz, q(w), x_in.shape) * (x_in > 0))
        grads.append((lg, ghw, ghb))
    return p, loss, pack(grads)


def adam(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def dmt_shifts(freqs, nsub, max_sweep, rows=256):
    """Row j: residual sweep max_sweep * (2j/(rows-1) - 1) bins across the
    band, per subband in proportion to f^-2 - f_top^-2 (Eq. 1), rounded
    half away from zero."""
    f = np.asarray(freqs, np.float64).reshape(nsub, -1).mean(axis=1)
    g = 1.0 / (f * f)
    frac = (g - g[0]) / (g[-1] - g[0])
    sweep = max_sweep * (2.0 * np.arange(rows) / (rows - 1) - 1.0)
    v = sweep[:, None] * frac[None, :]
    return (np.sign(v) * np.floor(np.abs(v) + 0.5)).astype(np.int64)


def features(sub, shifts):
    """sub [N][S][T] -> (ft, dmt) [N][256][256], each standardised (zero
    mean, unit population variance) per image."""
    n, s, t = sub.shape
    u0 = (t - 256) // 2
    ft = sub[:, :, u0:u0 + 256].astype(np.float64)
    dmt = np.zeros((n, shifts.shape[0], 256))
    u = np.arange(256)
    for j in range(shifts.shape[0]):
        for k in range(s):
            idx = u0 + u + shifts[j, k]
            ok = (idx >= 0) & (idx < t)
            dmt[:, j, ok] += sub[:, k, idx[ok]]

    def std(a):
        m = a.mean(axis=(1, 2), keepdims=True)
        sd = a.std(axis=(1, 2), keepdims=True)
        return np.where(sd > 0, (a - m) / np.where(sd > 0, sd, 1), 0.0)
    return std(ft), std(dmt)
