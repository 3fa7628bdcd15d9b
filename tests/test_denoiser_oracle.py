"""Pins of the FP64 denoiser oracle (CPU only).

Every test checks the oracle against something other than its own formulas: FP64
finite differences of the loss, exact adjoint identities, the separately pinned C
border fixup, torch's bfloat16 conversion, hand-built networks whose output is
known in closed form, and Adam's first step in closed form.
"""
import numpy as np
import pytest

import oracle
import oracle.denoiser as D


def _toy(P=2, seed=0, dims=(2, 1, 1)):
    rng = np.random.default_rng(seed)
    irr = rng.uniform(0.05, 1.0, (P, 8, 8, 4))
    for p in range(P):  # maps as the update leaves them: border = fixup of the interior
        irr[p] = oracle.border(irr[p])
    depth = rng.uniform(0.5, 4.0, (P, 16, 16, 2))
    depth[..., 1] = depth[..., 0] ** 2 + rng.uniform(0.0, 0.3, (P, 16, 16))
    valid = np.ones(P, np.uint8)
    target = irr + rng.normal(0.0, 0.05, irr.shape)
    X = D.features(irr, depth, valid, dims, 1, 2.0)
    return irr, depth, valid, target, X


def _theta(seed=1, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shape in D.SHAPES:
        fan = 9 * shape[1] if len(shape) == 3 else 1
        lim = np.sqrt(6.0 / fan) if len(shape) == 3 else 0.1
        parts[name] = rng.uniform(-lim, lim, shape) * scale
    return D.pack(parts)


def test_parameter_count():
    assert D.N_PARAMS == 35 * 64 * 9 + 64 + 64 * 48 * 9 + 48 + 48 * 3 * 9 + 3 == 49219


def test_pad_equals_the_c_border_fixup():
    rng = np.random.default_rng(3)
    for C in (1, 3, 7):
        m = rng.normal(size=(8, 8, C))
        assert np.array_equal(D.pad(m[1:7, 1:7]), oracle.border(m))


def test_unpad_grad_is_the_adjoint_of_pad():
    rng = np.random.default_rng(4)
    a = rng.normal(size=(3, 6, 6, 5))
    g = rng.normal(size=(3, 8, 8, 5))
    lhs = float((D.pad(a) * g).sum())
    rhs = float((a * D.unpad_grad(g)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_conv_backward_is_the_adjoint_of_conv():
    rng = np.random.default_rng(5)
    F = rng.normal(size=(2, 8, 8, 4))
    w = rng.normal(size=(9, 4, 3))
    dZ = rng.normal(size=(2, 6, 6, 3))
    dF, dw, db = D.conv_backward(F, w, dZ)
    zero_b = np.zeros(3)
    assert abs(float((D.conv(F, w, zero_b) * dZ).sum()) - float((F * dF).sum())) < 1e-10
    assert abs(float((D.conv(F, w, zero_b) * dZ).sum()) - float((w * dw).sum())) < 1e-10
    assert np.allclose(db, dZ.sum(axis=(0, 1, 2)))


def test_gradient_matches_fp64_finite_differences():
    """Central differences at h = 1e-6 on a 2-probe toy, 72 coordinates spread over
    every parameter tensor; relative error <= 1e-6 of the gradient's scale."""
    irr, depth, valid, target, X = _toy()
    theta = _theta()
    active = np.ones(2, bool)
    L, g = D.gradients(theta, X, irr, target, active)
    rng = np.random.default_rng(9)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in D.SHAPES])
    idx = np.concatenate([rng.choice(np.arange(offs[i], offs[i + 1]), min(12, offs[i + 1] - offs[i]),
                                     replace=False) for i in range(len(D.SHAPES))])
    h = 1e-6
    fd = []
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd.append((D.loss_fn(tp, X, irr, target, active) - D.loss_fn(tm, X, irr, target, active)) / (2 * h))
    fd = np.array(fd)
    scale = np.abs(g).max()
    assert scale > 0
    assert np.abs(fd - g[idx]).max() <= 1e-6 * scale, np.abs(fd - g[idx]).max() / scale


def test_inactive_probes_neither_change_nor_count():
    irr, depth, valid, target, X = _toy()
    theta = _theta()
    active = np.array([True, False])
    Y, _ = D.forward(theta, X, irr)
    out = D.output_maps(Y, irr, active)
    assert np.array_equal(out[1], irr[1])
    L1, g1 = D.gradients(theta, X, irr, target, active)
    target2 = target.copy()
    target2[1] += 5.0  # the inactive probe's target is irrelevant
    L2, g2 = D.gradients(theta, X, irr, target2, active)
    assert L1 == L2 and np.array_equal(g1, g2)


def test_zero_network_is_the_identity():
    irr, depth, valid, target, X = _toy()
    Y, _ = D.forward(np.zeros(D.N_PARAMS), X, irr)
    out = D.output_maps(Y, irr, np.ones(2, bool))
    assert np.array_equal(out, irr)


@pytest.mark.parametrize("tap", range(9))
def test_single_tap_network_reads_the_shifted_texel(tap):
    """w1 copies the own-irradiance channels through one tap, w2 and w3 through the
    centre tap: Y = x + x(shifted by the tap), indexing the bordered input map directly."""
    irr, depth, valid, target, X = _toy()
    p = {name: np.zeros(shape) for name, shape in D.SHAPES}
    for c in range(3):
        p["w1"][tap, c, c] = 1.0
        p["w2"][4, c, c] = 1.0
        p["w3"][4, c, c] = 1.0
    Y, _ = D.forward(D.pack(p), X, irr)
    dy, dx = D.TAPS[tap]
    for r in range(1, 7):
        for c in range(1, 7):
            want = irr[:, r, c, :3] + irr[:, r + dy, c + dx, :3]
            assert np.allclose(Y[:, r - 1, c - 1], want, rtol=0, atol=1e-15)


def test_features_route_neighbours_and_moments():
    dims = (3, 2, 2)
    P = 12
    irr = np.zeros((P, 8, 8, 4))
    depth = np.zeros((P, 16, 16, 2))
    for p in range(P):
        irr[p, ..., :3] = p + np.array([0.0, 0.25, 0.5])
        depth[p, ..., 0] = 1.0 + p
        depth[p, ..., 1] = (1.0 + p) ** 2 + 1.0
    valid = np.ones(P, np.uint8)
    valid[4] = 0  # probe (1, 1, 0) has no history: its neighbours see themselves instead
    s = 2.0
    X = D.features(irr, depth, valid, dims, 1, s)
    assert X.shape == (P, 8, 8, 35)
    for p in range(P):
        x, y, z = p % 3, (p // 3) % 2, p // 6
        for k, (ax, d) in enumerate(((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1))):
            c = [x, y, z]
            c[ax] += d
            inside = 0 <= c[0] < 3 and 0 <= c[1] < 2 and 0 <= c[2] < 2
            q = (c[2] * 2 + c[1]) * 3 + c[0] if inside else p
            if valid[q] == 0:
                q = p
            assert np.all(X[p, ..., 3 + 3 * k:6 + 3 * k] == irr[q, 0, 0, :3]), (p, k)
            assert np.all(X[p, ..., 23 + 2 * k] == (1.0 + q) / s), (p, k)
            assert np.all(X[p, ..., 24 + 2 * k] == ((1.0 + q) ** 2 + 1.0) / s ** 2), (p, k)
        assert np.all(X[p, ..., 0:3] == irr[p, 0, 0, :3])
    # 2 x 2 averaging of the 16 x 16 depth map onto the 8 x 8 grid
    d = np.zeros((1, 16, 16, 2))
    rr, cc = np.meshgrid(np.arange(16.0), np.arange(16.0), indexing="ij")
    d[0, ..., 0] = rr * 16 + cc
    X1 = D.features(np.zeros((1, 8, 8, 4)), d, np.ones(1, np.uint8), (1, 1, 1), 1, 1.0)
    i, j = np.meshgrid(np.arange(8.0), np.arange(8.0), indexing="ij")
    assert np.array_equal(X1[0, ..., 21], (2 * i + 0.5) * 16 + (2 * j + 0.5))


def test_bf16_rounding_matches_torch_and_ties_to_even():
    import torch
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.uniform(-6, 6, 4000),
                        [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8)]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(D.bf16(x), want)
    assert D.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0                 # tie, even mantissa below
    assert D.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6   # tie, even mantissa above


def test_adam_first_steps_closed_form():
    """With bias correction, step 1 moves each coordinate by lr * g / (|g| + eps); a
    constant gradient keeps that step size on step 2."""
    rng = np.random.default_rng(7)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    m = v = np.zeros(50)
    th1, m, v = D.adam(th, g, m, v, 1, 1e-3)
    assert np.allclose(th1, th - 1e-3 * g / (np.abs(g) + D.ADAM_EPS), rtol=0, atol=1e-15)
    th2, m, v = D.adam(th1, g, m, v, 2, 1e-3)
    assert np.allclose(th2, th1 - 1e-3 * g / (np.abs(g) + D.ADAM_EPS), rtol=0, atol=1e-14)


def test_loss_closed_form():
    irr, depth, valid, target, X = _toy()
    Y = target[:, 1:7, 1:7, :3] + 0.5
    L, dY = D.loss_and_grad(Y, target, np.ones(2, bool))
    assert abs(L - 0.25) < 1e-15
    assert np.allclose(dY, 2 * 0.5 / (2 * 108))
