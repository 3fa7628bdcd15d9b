"""Asynchronous reads of the maps, overlapping the next update (needs a B300).

A caller that ships every frame's maps off the GPU can copy frame f's maps on the volume's
copy stream while frame f+1 updates. Frame f+1 only reads that buffer (it is its history).
The library makes the first later call that overwrites the buffer (the update two frames
on, write_state, reset, a batch update) wait for the copy. These tests check the copied
values against a twin volume read synchronously after each update, with no host
synchronisation between the calls: plain updates with and without slab branches, a
batch, and write_state / reset after a pending read.
"""
import numpy as np
import pytest
import torch

import paper_2007_14394_b300 as S
import workloads as W
from harness import GpuVolume, make_workload

pytestmark = pytest.mark.gpu


def host_maps(P, pinned=True):
    mk = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory() if pinned else torch.empty(shape, dtype=dt)
    return mk((P, 8, 8, 4), torch.float32), mk((P, 16, 16, 2), torch.float32), mk((P,), torch.uint8)


def as_np(maps):
    return tuple(t.numpy().copy() for t in maps)


@pytest.mark.parametrize("preset,slabs", [("room64", 1), ("room64", 3), ("open256", 0)])
def test_async_reads_equal_synchronous_reads(cuda_device, preset, slabs):
    w = make_workload(W.PRESETS[preset])
    sc = S.create_scene()
    S.upload_sdf(sc, w.baked.sdf, w.baked.h, w.baked.origin, material=w.baked.material)
    S.set_lights(sc, w.lights, w.sky)
    a = GpuVolume(w, seed=2, scene=sc)   # async reads, no host synchronisation in the loop
    b = GpuVolume(w, seed=2, scene=sc)   # the twin, read synchronously after each update
    try:
        S.set_slabs(a.vol, slabs)
        S.set_slabs(b.vol, slabs)
        frames = 5
        bufs = [host_maps(w.P) for _ in range(frames)]
        done = [torch.cuda.Event() for _ in range(frames)]
        stream = torch.cuda.current_stream()
        expect = []
        for f in range(frames):
            rot = W.frame_rotation(4, f)
            a.update(rot, record=False)
            S.read_state_async(a.vol, *bufs[f], stream=stream, done_event=done[f])
            b.update(rot, record=False)
            expect.append(b.state())
        for f in range(frames):
            done[f].synchronize()
            got = as_np(bufs[f])
            for g, e, name in zip(got, expect[f], ("irr", "depth", "valid")):
                assert np.array_equal(g, e), (preset, slabs, f, name)
        assert np.abs(expect[-1][0][..., :3]).max() > 0
        assert S.volume_status(a.vol) == 0
    finally:
        a.close()
        b.close()
        S.destroy_scene(sc)


def test_async_read_then_write_state_and_reset(cuda_device):
    w = make_workload(W.PRESETS["room64"])
    gv = GpuVolume(w)
    try:
        gv.update(W.frame_rotation(1, 0), record=False)
        first = gv.state()
        out = host_maps(w.P)
        ev = torch.cuda.Event()
        S.read_state_async(gv.vol, *out, done_event=ev)
        # overwrite the buffer being read, then clear everything: both wait for the copy
        S.write_state(gv.vol, np.zeros_like(first[0]), np.zeros_like(first[1]), np.zeros_like(first[2]))
        ev.synchronize()
        for g, e in zip(as_np(out), first):
            assert np.array_equal(g, e)
        S.read_state_async(gv.vol, *out, done_event=ev)
        S.reset(gv.vol)
        ev.synchronize()
        assert not out[0].any() and not out[2].any()  # the zeros written above
        # device destinations and NULL arrays
        d_irr = torch.empty((w.P, 8, 8, 4), dtype=torch.float32, device="cuda")
        gv.update(W.frame_rotation(1, 1), record=False)
        S.read_state_async(gv.vol, d_irr, None, None, done_event=ev)
        ev.synchronize()
        assert np.array_equal(d_irr.cpu().numpy(), gv.state()[0])
    finally:
        gv.close()


def test_async_read_of_a_batched_volume(cuda_device):
    w = make_workload(W.PRESETS["room64"])
    sc = S.create_scene()
    S.upload_sdf(sc, w.baked.sdf, w.baked.h, w.baked.origin, material=w.baked.material)
    S.set_lights(sc, w.lights, w.sky)
    a = GpuVolume(w, seed=3, scene=sc)
    b = GpuVolume(w, seed=3, scene=sc)
    batch = S.create_batch([a.vol], [a.states_dev])
    try:
        bufs = [host_maps(w.P) for _ in range(4)]
        done = [torch.cuda.Event() for _ in range(4)]
        expect = []
        for f in range(4):
            S.update_batch(batch, f)
            S.read_state_async(a.vol, *bufs[f], done_event=done[f])
            S.update_probes(b.vol, f, states=b.states_dev)
            expect.append(b.state())
        for f in range(4):
            done[f].synchronize()
            for g, e in zip(as_np(bufs[f]), expect[f]):
                assert np.array_equal(g, e), f
    finally:
        S.destroy_batch(batch)
        a.close()
        b.close()
        S.destroy_scene(sc)
