"""FP64 oracle of the probe denoiser (the learned form of the update).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the CUDA library never
does, and the two share no code.

The paper has no learned component; the network follows the learned form that
is specified for this project. A 32-ray probe update is noisy. A small
convolutional network over a probe's octahedral maps and those of its six grid
neighbours predicts a correction of its irradiance toward the converged value:
  input   35 channels on the 8 x 8 bordered octahedral grid of the irradiance map:
          the irradiance rgb of the probe and of its neighbours -x, +x, -y, +y, -z, +z
          (21 channels), then their depth moments (mean distance / s, mean squared
          distance / s^2), each averaged over 2 x 2 texels of the 16 x 16 depth map (14
          channels). A neighbour outside the grid, or one without history (valid 0),
          is replaced by the probe itself.
  layers  three 3 x 3 convolutions 35 -> 64 -> 48 -> 3 over the 6 x 6 interior. Each
          reads the 8 x 8 bordered grid, so the octahedral border (Sec. 3.3, the same
          mirror rule as the maps' border fixup) acts as its padding. The hidden layers
          are ReLU, and their outputs get the border fixup again before the next layer.
  output  irradiance = max(0, own interior irradiance + residual), then the border
          fixup. The alpha channel and inactive probes pass through unchanged.
  loss    mean squared error over the interior rgb texels of active probes.
  update  Adam (Kingma and Ba 2015, Algorithm 1) with bias correction.
Precision: plain FP64, or with the rounding of the deployed network emulated. In that
mode the weights and each layer's input (the features, then the two hidden
activations) are rounded to bfloat16, round-to-nearest-even. The biases and the
residual's irradiance stay unrounded. The gradient is straight-through: it is taken
at the rounded values, and the rounding itself counts as the identity.

Parameter vector (float, 49,219 entries), in this order: w1 [9][35][64], b1 [64],
w2 [9][64][48], b2 [48], w3 [9][48][3], b3 [3]. Tap k = (dy + 1) * 3 + (dx + 1)
reads the input at (row + dy, column + dx).
"""
from __future__ import annotations

import numpy as np

C_IN, C1, C2, C_OUT = 35, 64, 48, 3
SHAPES = (("w1", (9, C_IN, C1)), ("b1", (C1,)), ("w2", (9, C1, C2)), ("b2", (C2,)),
          ("w3", (9, C2, C_OUT)), ("b3", (C_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 49,219
TAPS = tuple((dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
N = 6            # interior texels per side
T = N + 2        # with the border
ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (8 significant bits), to nearest, ties to even. The value is
    taken to float32 first, as the kernels hold it."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------- octahedral border as padding
def border_sources(n: int = N):
    """(row, col) source of every texel of an (n+2)^2 map under the border fixup: the
    texel itself in the interior, its mirror image on the border."""
    t = n + 2
    rows, cols = np.meshgrid(np.arange(t), np.arange(t), indexing="ij")
    sr, sc = rows.copy(), cols.copy()
    for x in range(1, n + 1):
        sr[0, x], sc[0, x] = 1, n + 1 - x        # top
        sr[n + 1, x], sc[n + 1, x] = n, n + 1 - x  # bottom
    for y in range(1, n + 1):
        sr[y, 0], sc[y, 0] = n + 1 - y, 1        # left
        sr[y, n + 1], sc[y, n + 1] = n + 1 - y, n  # right
    sr[0, 0], sc[0, 0] = n, n
    sr[0, n + 1], sc[0, n + 1] = n, 1
    sr[n + 1, 0], sc[n + 1, 0] = 1, n
    sr[n + 1, n + 1], sc[n + 1, n + 1] = 1, 1
    return sr, sc


_SR, _SC = border_sources()


def pad(interior: np.ndarray) -> np.ndarray:
    """[..., 6, 6, C] interior -> [..., 8, 8, C] with the octahedral border filled."""
    return interior[..., _SR - 1, _SC - 1, :]


def unpad_grad(g: np.ndarray) -> np.ndarray:
    """Adjoint of pad: the gradient on a bordered map summed onto the interior texels
    each border texel copies."""
    out = np.zeros(g.shape[:-3] + (N, N, g.shape[-1]))
    for r in range(T):
        for c in range(T):
            out[..., _SR[r, c] - 1, _SC[r, c] - 1, :] += g[..., r, c, :]
    return out


# ---------------------------------------------------------------- features
def neighbours(dims, n_grids: int = 1) -> np.ndarray:
    """[P, 6] index of the -x, +x, -y, +y, -z, +z neighbour of every probe of n_grids
    stacked grids (x fastest within a grid), -1 outside the grid."""
    nx, ny, nz = (int(d) for d in dims)
    pg = nx * ny * nz
    out = np.full((n_grids * pg, 6), -1, dtype=np.int64)
    for g in range(n_grids):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    p = g * pg + (z * ny + y) * nx + x
                    for k, (ax, d) in enumerate(((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1))):
                        c = [x, y, z]
                        c[ax] += d
                        if 0 <= c[0] < nx and 0 <= c[1] < ny and 0 <= c[2] < nz:
                            out[p, k] = g * pg + (c[2] * ny + c[1]) * nx + c[0]
    return out


def features(irr: np.ndarray, depth: np.ndarray, valid: np.ndarray, dims, n_grids: int,
             depth_scale: float) -> np.ndarray:
    """[P, 8, 8, 35] network input from the maps irr [P][8][8][4], depth [P][16][16][2]."""
    P = irr.shape[0]
    nb = neighbours(dims, n_grids)
    src = np.where((nb >= 0) & (valid[np.maximum(nb, 0)] != 0), nb, np.arange(P)[:, None])
    mom = np.asarray(depth, dtype=np.float64).reshape(P, T, 2, T, 2, 2).mean(axis=(2, 4))
    mom = mom / np.array([depth_scale, depth_scale * depth_scale])
    rgb = np.asarray(irr, dtype=np.float64)[..., :3]
    chans = [rgb] + [rgb[src[:, k]] for k in range(6)] + [mom] + [mom[src[:, k]] for k in range(6)]
    return np.concatenate(chans, axis=-1)


# ---------------------------------------------------------------- network
def conv(F: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """3 x 3 convolution of a bordered [P, 8, 8, Cin] map onto its [P, 6, 6, Cout] interior."""
    out = np.broadcast_to(b, F.shape[:-3] + (N, N, w.shape[-1])).copy()
    for k, (dy, dx) in enumerate(TAPS):
        out += F[..., 1 + dy:1 + dy + N, 1 + dx:1 + dx + N, :] @ w[k]
    return out


def forward(theta: np.ndarray, X: np.ndarray, irr: np.ndarray, round_bf16: bool = False):
    """Returns (interior irradiance [P, 6, 6, 3], cache for backward)."""
    p = unpack(theta)
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    w1, w2, w3 = r(p["w1"]), r(p["w2"]), r(p["w3"])
    F0 = r(X)
    Z1 = conv(F0, w1, p["b1"])
    F1 = r(pad(np.maximum(Z1, 0.0)))
    Z2 = conv(F1, w2, p["b2"])
    F2 = r(pad(np.maximum(Z2, 0.0)))
    R = conv(F2, w3, p["b3"])
    base = np.asarray(irr, dtype=np.float64)[:, 1:1 + N, 1:1 + N, :3]
    Y = np.maximum(base + R, 0.0)
    cache = dict(F0=F0, Z1=Z1, F1=F1, Z2=Z2, F2=F2, pre=base + R, w1=w1, w2=w2, w3=w3)
    return Y, cache


def output_maps(Y: np.ndarray, irr: np.ndarray, active: np.ndarray) -> np.ndarray:
    """The denoised [P, 8, 8, 4] maps: interior rgb Y with the border fixup, alpha kept;
    inactive probes unchanged."""
    out = np.array(irr, dtype=np.float64)
    full = pad(Y)
    act = np.asarray(active, dtype=bool)
    out[act, :, :, :3] = full[act]
    return out


def loss_and_grad(Y: np.ndarray, target: np.ndarray, active: np.ndarray):
    """Mean squared error over the interior rgb of active probes and its gradient in Y."""
    act = np.asarray(active, dtype=bool)
    n = max(int(act.sum()), 1) * N * N * 3
    tgt = np.asarray(target, dtype=np.float64)[:, 1:1 + N, 1:1 + N, :3]
    d = (Y - tgt) * act[:, None, None, None]
    return float((d * d).sum() / n), 2.0 * d / n


def conv_backward(F: np.ndarray, w: np.ndarray, dZ: np.ndarray):
    """Gradients of conv in its bordered input, weights and bias."""
    dF = np.zeros(F.shape)
    dw = np.zeros(w.shape)
    for k, (dy, dx) in enumerate(TAPS):
        sl = F[..., 1 + dy:1 + dy + N, 1 + dx:1 + dx + N, :]
        dw[k] = sl.reshape(-1, sl.shape[-1]).T @ dZ.reshape(-1, dZ.shape[-1])
        dF[..., 1 + dy:1 + dy + N, 1 + dx:1 + dx + N, :] += dZ @ w[k].T
    return dF, dw, dZ.reshape(-1, dZ.shape[-1]).sum(axis=0)


def backward(theta: np.ndarray, cache: dict, dY: np.ndarray) -> np.ndarray:
    """Gradient of the loss in the parameter vector, given its gradient dY in the output."""
    dR = dY * (cache["pre"] > 0)
    dF2, dw3, db3 = conv_backward(cache["F2"], cache["w3"], dR)
    dZ2 = unpad_grad(dF2) * (cache["Z2"] > 0)
    dF1, dw2, db2 = conv_backward(cache["F1"], cache["w2"], dZ2)
    dZ1 = unpad_grad(dF1) * (cache["Z1"] > 0)
    _, dw1, db1 = conv_backward(cache["F0"], cache["w1"], dZ1)
    return pack(dict(w1=dw1, b1=db1, w2=dw2, b2=db2, w3=dw3, b3=db3))


def loss_fn(theta, X, irr, target, active, round_bf16=False) -> float:
    Y, _ = forward(theta, X, irr, round_bf16)
    return loss_and_grad(Y, target, active)[0]


def gradients(theta, X, irr, target, active, round_bf16=False):
    """(loss, gradient in theta) by the analytic backward pass."""
    Y, cache = forward(theta, X, irr, round_bf16)
    L, dY = loss_and_grad(Y, target, active)
    return L, backward(theta, cache, dY)


def adam(theta: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, step: int, lr: float):
    """One Adam step (step counts from 1); returns the new (theta, m, v)."""
    m = ADAM_BETA1 * m + (1.0 - ADAM_BETA1) * grad
    v = ADAM_BETA2 * v + (1.0 - ADAM_BETA2) * grad * grad
    mhat = m / (1.0 - ADAM_BETA1 ** step)
    vhat = v / (1.0 - ADAM_BETA2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v
