"""The probe denoiser's CUDA kernels against the FP64 oracle, and what training gains
(needs a B300).

Forward: fp32 mode against the oracle in FP64. The bf16 modes (CUDA cores and tensor
cores) are checked against the oracle with the same bf16 rounding emulated. There, a
bf16 rounding of a hidden activation can land on the other side of a rounding
boundary, because the kernels accumulate in fp32 and the oracle in fp64. Such a flip
moves one activation by one bf16 unit (2^-8 relative). The tolerance therefore
bounds the fraction of outputs that move at all (observed under 2 %), and how far
any one moves (observed 3.5e-4 of the output scale).
Gradients: fp32 mode to a few fp32 roundings of the oracle's; bf16 mode (straight-
through) to 1e-3 of each parameter tensor's gradient norm.
"""
import numpy as np
import pytest

import oracle
import oracle.denoiser as D
import paper_2007_14394_b300 as S
import workloads as W
from harness import border_is_mirror

pytestmark = pytest.mark.gpu

DIMS, NG = (3, 2, 2), 2
P = NG * 12
SCALE = 2.0


def _inputs(seed=0):
    rng = np.random.default_rng(seed)
    irr = np.zeros((P, 8, 8, 4))
    irr[..., :3] = rng.uniform(0.05, 1.0, (P, 8, 8, 3))
    irr[..., 3] = 1.0
    for p in range(P):
        irr[p] = oracle.border(irr[p])
    depth = rng.uniform(0.5, 4.0, (P, 16, 16, 2))
    depth[..., 1] = depth[..., 0] ** 2 + rng.uniform(0.0, 0.3, (P, 16, 16))
    valid = (rng.random(P) > 0.2).astype(np.uint8)
    st = np.zeros(P, dtype=W.PROBE_DTYPE)
    st["flags"] = (rng.random(P) > 0.15).astype(np.uint32)
    st["flags"][0] = 1
    target = irr.copy()
    target[..., :3] += rng.normal(0.0, 0.1, (P, 8, 8, 3))
    theta = W.denoiser_init(seed + 1, last_scale=1.0).astype(np.float64)
    p = D.unpack(theta)
    for b in ("b1", "b2", "b3"):
        p[b] = rng.uniform(-0.1, 0.1, p[b].shape)
    theta = D.pack(p).astype(np.float32)
    return (irr.astype(np.float32), depth.astype(np.float32), valid, st, target.astype(np.float32), theta)


class Dev:
    def __init__(self, irr, depth, valid, st, target, theta):
        import torch
        self.torch = torch
        self.irr = torch.from_numpy(irr).cuda()
        self.depth = torch.from_numpy(depth).cuda()
        self.valid = torch.from_numpy(valid).cuda()
        self.states = torch.from_numpy(st.view(np.uint8).copy()).cuda()
        self.target = torch.from_numpy(target).cuda()
        self.maps = S.probe_maps(DIMS, NG, self.irr, self.depth, self.valid, self.states)
        self.d = S.create_denoiser(theta, SCALE)

    def denoise(self, mode):
        out = self.torch.full_like(self.irr, float("nan"))
        S.denoise(self.d, self.maps, out, mode)
        assert S.denoiser_status(self.d) == 0
        return out.cpu().numpy().astype(np.float64)

    def gradients(self, mode):
        g = self.torch.empty(S.DENOISER_PARAMS, device="cuda")
        loss = self.torch.empty(1, device="cuda")
        S.denoiser_gradients(self.d, self.maps, self.target, g, loss, mode=mode)
        self.torch.cuda.synchronize()
        return float(loss.item()), g.cpu().numpy().astype(np.float64)

    def close(self):
        S.destroy_denoiser(self.d)


def _oracle(irr, depth, valid, st, target, theta, round_bf16):
    X = D.features(irr, depth, valid, DIMS, NG, SCALE)
    act = (st["flags"] & 1).astype(bool)
    Y, _ = D.forward(theta.astype(np.float64), X, irr, round_bf16)
    L, g = D.gradients(theta.astype(np.float64), X, irr, target, act, round_bf16)
    return D.output_maps(Y, irr, act), L, g, act


@pytest.fixture(scope="module")
def case(cuda_device):
    inp = _inputs()
    dev = Dev(*inp)
    yield inp, dev
    dev.close()


def _check_common(out, irr, act):
    assert np.all(np.isfinite(out))
    assert np.array_equal(out[~act], irr[~act].astype(np.float64))        # inactive: unchanged
    assert np.array_equal(out[..., 3], irr[..., 3].astype(np.float64))    # alpha kept
    assert border_is_mirror(out[act].astype(np.float32))


def test_forward_fp32_matches_oracle(case):
    inp, dev = case
    ref, _, _, act = _oracle(*inp, round_bf16=False)
    out = dev.denoise(S.DENOISE_SIMT_FP32)
    _check_common(out, inp[0], act)
    scale = np.abs(ref).max()
    err = np.abs(out - ref).max()
    print("fp32 forward max err / scale", err / scale)
    assert err <= 2e-5 * scale


@pytest.mark.parametrize("mode", [S.DENOISE_SIMT_BF16, S.DENOISE_TENSOR])
def test_forward_bf16_matches_oracle_with_rounding(case, mode):
    inp, dev = case
    ref, _, _, act = _oracle(*inp, round_bf16=True)
    out = dev.denoise(mode)
    _check_common(out, inp[0], act)
    scale = np.abs(ref).max()
    err = np.abs(out - ref)[act][..., :3]
    frac_moved = float((err > 1e-5 * scale).mean())
    print("bf16 mode", mode, "max err / scale", err.max() / scale, "moved", frac_moved)
    assert frac_moved <= 0.05
    assert err.max() <= 2e-3 * scale


def test_tensor_core_odd_probe_count(cuda_device):
    """9 probes (one grid of 3 x 3 x 1): the tensor-core kernel's last two-probe tile holds one
    probe. Against the oracle with bf16 rounding, as above, and the inactive pass-through."""
    import torch
    dims, ng, n = (3, 3, 1), 1, 9
    rng = np.random.default_rng(7)
    irr = np.zeros((n, 8, 8, 4))
    irr[..., :3] = rng.uniform(0.05, 1.0, (n, 8, 8, 3))
    irr[..., 3] = 1.0
    for p in range(n):
        irr[p] = oracle.border(irr[p])
    depth = rng.uniform(0.5, 4.0, (n, 16, 16, 2))
    depth[..., 1] = depth[..., 0] ** 2 + rng.uniform(0.0, 0.3, (n, 16, 16))
    valid = (rng.random(n) > 0.2).astype(np.uint8)
    st = np.zeros(n, dtype=W.PROBE_DTYPE)
    st["flags"] = 1
    st["flags"][4] = 0
    theta = W.denoiser_init(3, last_scale=1.0).astype(np.float32)
    irr, depth = irr.astype(np.float32), depth.astype(np.float32)
    X = D.features(irr, depth, valid, dims, ng, SCALE)
    act = (st["flags"] & 1).astype(bool)
    Y, _ = D.forward(theta.astype(np.float64), X, irr, True)
    ref = D.output_maps(Y, irr, act)
    d = S.create_denoiser(theta, SCALE)
    try:
        # the maps view holds raw device pointers: the tensors must outlive the calls
        irr_d, depth_d = torch.from_numpy(irr).cuda(), torch.from_numpy(depth).cuda()
        valid_d, st_d = torch.from_numpy(valid).cuda(), torch.from_numpy(st.view(np.uint8).copy()).cuda()
        maps = S.probe_maps(dims, ng, irr_d, depth_d, valid_d, st_d)
        out_d = torch.full_like(irr_d, float("nan"))
        S.denoise(d, maps, out_d, S.DENOISE_TENSOR)
        assert S.denoiser_status(d) == 0
        out = out_d.cpu().numpy().astype(np.float64)
    finally:
        S.destroy_denoiser(d)
    _check_common(out, irr, act)
    scale = np.abs(ref).max()
    err = np.abs(out - ref)[act][..., :3]
    print("odd count: max err / scale", err.max() / scale, "moved", float((err > 1e-5 * scale).mean()))
    assert float((err > 1e-5 * scale).mean()) <= 0.05
    assert err.max() <= 2e-3 * scale


def test_tensor_core_matches_cuda_core_bf16(case):
    inp, dev = case
    a = dev.denoise(S.DENOISE_TENSOR)
    b = dev.denoise(S.DENOISE_SIMT_BF16)
    scale = np.abs(b).max()
    err = np.abs(a - b)
    print("tc vs simt max err / scale", err.max() / scale, "moved", float((err > 1e-5 * scale).mean()))
    assert float((err > 1e-5 * scale).mean()) <= 0.05
    assert err.max() <= 2e-3 * scale


def test_gradients_fp32_match_oracle(case):
    inp, dev = case
    _, L, g, _ = _oracle(*inp, round_bf16=False)
    Lg, gg = dev.gradients(S.DENOISE_SIMT_FP32)
    assert abs(Lg - L) <= 1e-5 * abs(L)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in D.SHAPES])
    for i, (name, _) in enumerate(D.SHAPES):
        a, b = gg[offs[i]:offs[i + 1]], g[offs[i]:offs[i + 1]]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(name, "fp32 grad rel", rel, "max", np.abs(a - b).max() / np.abs(b).max())
        assert rel <= 2e-5, name
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), name


def test_gradients_bf16_match_oracle(case):
    inp, dev = case
    _, L, g, _ = _oracle(*inp, round_bf16=True)
    Lg, gg = dev.gradients(S.DENOISE_SIMT_BF16)
    assert abs(Lg - L) <= 1e-3 * abs(L)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in D.SHAPES])
    for i, (name, _) in enumerate(D.SHAPES):
        a, b = gg[offs[i]:offs[i + 1]], g[offs[i]:offs[i + 1]]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(name, "bf16 grad rel", rel)
        assert rel <= 1e-3, name


def test_adam_matches_oracle(cuda_device):
    import torch
    rng = np.random.default_rng(11)
    th = rng.normal(0.0, 0.1, S.DENOISER_PARAMS).astype(np.float32)
    d = S.create_denoiser(th, 1.0)
    try:
        ref, m, v = th.astype(np.float64), np.zeros(S.DENOISER_PARAMS), np.zeros(S.DENOISER_PARAMS)
        for step in (1, 2, 3):
            g = rng.normal(0.0, 1e-2, S.DENOISER_PARAMS).astype(np.float32)
            S.denoiser_adam(d, torch.from_numpy(g).cuda(), 1e-3)
            ref, m, v = D.adam(ref, g.astype(np.float64), m, v, step, 1e-3)
        got = S.denoiser_params(d).astype(np.float64)
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
        # writing the parameters resets the optimiser: the next step is a first step again
        S.denoiser_params(d, write=th)
        g = np.full(S.DENOISER_PARAMS, 0.5, np.float32)
        S.denoiser_adam(d, torch.from_numpy(g).cuda(), 1e-3)
        got = S.denoiser_params(d).astype(np.float64)
        assert np.allclose(got, th.astype(np.float64) - 1e-3, rtol=0, atol=1e-6)
    finally:
        S.destroy_denoiser(d)


def test_denoise_volume_equals_denoise_of_its_maps(cuda_device):
    import torch
    pr = W.PRESETS["room64"]
    scene = pr.scene(3)
    baked = W.bake(scene, pr.sdf_dims, pr.h)
    st = W.probe_states(scene, pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.h)
    sc = S.create_scene()
    S.upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material)
    S.set_lights(sc, scene.lights, scene.sky)
    desc = S.make_desc(pr.probe_dims, 32, pr.probe_origin, pr.probe_spacing, pr.max_steps, hysteresis=0.0)
    v = S.create_volume(desc, sc)
    d = S.create_denoiser(W.denoiser_init(5, last_scale=1.0), 4.0)
    st_dev = torch.from_numpy(st.view(np.uint8).copy()).cuda()
    try:
        S.update_probes(v, 0, states=st_dev)
        n = int(np.prod(pr.probe_dims))
        irr, dep = torch.empty((n, 8, 8, 4), device="cuda"), torch.empty((n, 16, 16, 2), device="cuda")
        val = torch.empty(n, dtype=torch.uint8, device="cuda")
        S.read_state(v, irr, dep, val)
        want = torch.empty_like(irr)
        S.denoise(d, S.probe_maps(pr.probe_dims, 1, irr, dep, val, st_dev), want)
        S.denoise_volume(d, v, st_dev)
        got = torch.empty_like(irr)
        S.read_state(v, got, dep, val)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert not torch.equal(got, irr)
    finally:
        S.destroy_denoiser(d)
        S.destroy_volume(v)
        S.destroy_scene(sc)


def test_training_gains_over_the_plain_32_ray_update(cuda_device):
    """Trained on pairs the plain update makes on 24 room scenes, the network brings the
    32-ray update closer to the converged irradiance on 4 held-out scenes."""
    from paper_2007_14394_b300 import learned as L
    pr = W.PRESETS["room64"]
    train = L.make_pairs(pr, list(range(1, 25)), history_frames=16, plain_rays=(64, 256))
    held = L.make_pairs(pr, list(range(1001, 1005)), history_frames=16, plain_rays=(64, 256))
    d = S.create_denoiser(W.denoiser_init(0), 4.0)
    try:
        hist = L.train(d, train, steps=1500, batch_grids=8, lr=3e-4, log_every=300)
        print("loss", hist)
        r = L.evaluate(d, held)
        rt = L.evaluate(d, train)
        print("held-out rmse", r, "train rmse", rt)
        assert rt["denoised32"] < 0.9 * rt["plain32"]
        assert r["denoised32"] < 0.9 * r["plain32"]
        assert r["plain256"] < r["plain64"] < r["plain32"]
        rays = L.equal_error_rays(r)
        print("plain rays at the denoised error", rays)
        assert rays is not None and rays > 32
    finally:
        S.destroy_denoiser(d)
