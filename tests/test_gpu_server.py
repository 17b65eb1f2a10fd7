"""The render server (sdgs_server_*): continuous batching over resident scenes.

Every request's image must equal the same request rendered alone through the direct entry points
(the arithmetic does not depend on the mix, so the comparison is exact), while several requests
are in flight at once; host-side errors are reported and leave the server usable.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from paper_2503_07946_gb300 import render as prender
from paper_2503_07946_gb300 import sdgs

pytestmark = pytest.mark.gpu


def _scenes():
    return [synth.make_scene(60_000, seed=61, box=1.5, bg=synth.WHITE),
            synth.make_scene(120_000, seed=62, diag=(0.005, 0.2), clusters=16, cluster_box=2.0,
                             lambda_t=0.1, lambda_d=0.1)]


def _requests(rng, count):
    sizes = [(400, 400), (800, 800), (1352, 1014), (640, 360)]
    reqs = []
    for i in range(count):
        sid = int(rng.integers(0, 2))
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        d = rng.normal(size=3)
        eye = 4.0 * d / np.linalg.norm(d)
        cam = synth.make_camera(eye, w, h, 60.0, float(rng.uniform()), bg=(1.0, 1.0, 1.0) if sid == 0 else (0, 0, 0))
        reqs.append((sid, cam))
    return reqs


def _alone(dev, scene, cam):
    r = prender.Renderer(scene.n, cam.width, cam.height)
    img = r.forward(sdgs.scene_struct(dev, scene.lambda_t, scene.lambda_d), sdgs.view_struct(cam)).clone()
    torch.cuda.synchronize()
    return img


def test_requests_in_the_mix_equal_requests_alone():
    scenes = _scenes()
    devs = [prender.scene_to_device(s) for s in scenes]
    reqs = _requests(np.random.default_rng(7), 16)
    want = [_alone(devs[sid], scenes[sid], cam).cpu() for sid, cam in reqs]
    with sdgs.Server(budget_bytes=6 << 30, slots=4) as srv:
        ids = [srv.add_scene(d, s.lambda_t, s.lambda_d) for d, s in zip(devs, scenes)]
        outs = [torch.full((cam.height, cam.width, 3), -1.0, pin_memory=True) for _, cam in reqs]
        rids = [srv.submit(ids[sid], sdgs.view_struct(cam), out) for (sid, cam), out in zip(reqs, outs)]
        lats = [srv.wait(r, 30_000) for r in rids]
        st = srv.stats()
        for rid in rids:
            state, lat = srv.poll(rid)
            assert state == sdgs.REQ_DONE and lat > 0
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_inflight"] > 1, st  # several requests were on the device at once
    for got, exp in zip(outs, want):
        assert torch.equal(got, exp)
    assert all(l > 0 for l in lats)


def test_overflow_is_retried_transparently():
    # wide Gaussians at a small resolution need far more instances per pixel than the first guess
    scene = synth.make_scene(40_000, seed=63, box=0.5, diag=(0.2, 0.6), lambda_t=0.01, lambda_d=0.01)
    dev = prender.scene_to_device(scene)
    cam = synth.make_camera((0.0, 0.0, -2.0), 128, 128, 70.0, 0.5)
    want = _alone(dev, scene, cam).cpu()
    with sdgs.Server(budget_bytes=4 << 30, slots=2) as srv:
        sid = srv.add_scene(dev, scene.lambda_t, scene.lambda_d)
        out = torch.zeros(128, 128, 3, pin_memory=True)
        srv.wait(srv.submit(sid, sdgs.view_struct(cam), out), 30_000)
        st = srv.stats()
    assert st["retried"] >= 1
    assert torch.equal(out, want)


def test_host_side_errors_leave_the_server_usable():
    scene = synth.make_scene(20_000, seed=64, box=1.0)
    dev = prender.scene_to_device(scene)
    cam = synth.make_camera((0.0, 0.0, -3.0), 256, 256, 60.0, 0.5)
    view = sdgs.view_struct(cam)
    with sdgs.Server(budget_bytes=64 << 20, slots=1, queue_capacity=2) as srv:
        sid = srv.add_scene(dev, scene.lambda_t, scene.lambda_d)
        out = torch.zeros(256, 256, 3, pin_memory=True)
        with pytest.raises(sdgs.SdgsError) as e:
            srv.submit(sid + 5, view, out)
        assert e.value.code == 8  # NOT_FOUND
        big = sdgs.view_struct(synth.make_camera((0.0, 0.0, -3.0), 1920, 1080, 60.0, 0.5))
        with pytest.raises(sdgs.SdgsError) as e:
            srv.submit(sid, big, torch.zeros(1080, 1920, 3, pin_memory=True))
        assert e.value.code == 7  # OOM_BUDGET: more than the 64 MiB budget on its own
        with pytest.raises(sdgs.SdgsError) as e:
            srv.poll(123456789)
        assert e.value.code == 8
        # fill the queue: a submit beyond its capacity is refused, the others complete
        outs = [torch.zeros(256, 256, 3, pin_memory=True) for _ in range(8)]
        accepted, busy = [], 0
        for o in outs:
            try:
                accepted.append(srv.submit(sid, view, o))
            except sdgs.SdgsError as err:
                assert err.code == 6  # BUSY
                busy += 1
        assert busy >= 1 and accepted
        for rid in accepted:
            srv.wait(rid, 30_000)
        rid = srv.submit(sid, view, out)
        srv.wait(rid, 30_000)
        assert srv.release() >= len(accepted)
    want = _alone(dev, scene, cam).cpu()
    assert torch.equal(out, want)


def test_requests_admitted_together_share_one_slicing_launch():
    """Requests queued before the worker runs are admitted in one pass and sliced by one launch."""
    scenes = _scenes()
    devs = [prender.scene_to_device(s) for s in scenes]
    reqs = _requests(np.random.default_rng(8), 12)
    want = [_alone(devs[sid], scenes[sid], cam).cpu() for sid, cam in reqs]
    with sdgs.Server(budget_bytes=6 << 30, slots=8, batch_window_us=200_000) as srv:
        ids = [srv.add_scene(d, s.lambda_t, s.lambda_d) for d, s in zip(devs, scenes)]
        outs = [torch.zeros(cam.height, cam.width, 3, device="cuda") for _, cam in reqs]
        # submitted well within the 200 ms window: the first 8 are admitted together
        rids = [srv.submit(ids[sid], sdgs.view_struct(cam), out) for (sid, cam), out in zip(reqs, outs)]
        for r in rids:
            srv.wait(r, 30_000)
        st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["max_batch"] >= 8, st  # one launch sliced a whole wave of requests
    for got, exp in zip(outs, want):
        assert torch.equal(got.cpu(), exp)
