"""Failure detection in binning, without faulting or hanging the GPU.

The binning sort's only waits are its look-backs (a block reading the counts of the blocks before
it), each bounded.  A test entry point runs one radix pass whose block tickets start past zero, so
the blocks wait on tiles that nobody processes: each wait must give up after its round limit,
flag the error, keep every write in bounds, and leave the context usable.  A second entry point
runs the whole binning as if a pass had given up, to check what the later kernels do then."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synth
from paper_2503_07946_gb300 import sdgs
import _gpu_util as U

pytestmark = pytest.mark.gpu

SENTINEL = 0x5A5A5A5A


def _pass_inputs(n, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 3] &= 0xFFFFFF0F  # repeated digits: stability matters
    kin = torch.as_tensor(keys.view(np.int32), device="cuda")
    vin = torch.arange(n, dtype=torch.int32, device="cuda")
    pad = 4096
    kout = torch.full((n + pad,), SENTINEL, dtype=torch.int32, device="cuda")
    vout = torch.full((n + pad,), SENTINEL, dtype=torch.int32, device="cuda")
    return keys, kin, vin, kout, vout


def test_radix_pass_is_a_stable_sort_by_the_low_digit():
    n = 3 * 1024 + 17
    keys, kin, vin, kout, vout = _pass_inputs(n, 1)
    sdgs.lookback_selftest(kin, vin, kout, vout, n, first_ticket=0, spin_limit=2000)
    order = np.argsort(keys & 255, kind="stable")
    np.testing.assert_array_equal(vout[:n].cpu().numpy(), order)
    np.testing.assert_array_equal(kout[:n].cpu().numpy().view(np.uint32), keys[order])
    assert (kout[n:].cpu().numpy() == SENTINEL).all()


@pytest.mark.parametrize("first_ticket", [1, 2])
def test_lookback_wait_gives_up_reports_and_stays_in_bounds(first_ticket):
    n = 16 * 1024  # several sort tiles (1024-3072 keys each); tiles before first_ticket never run
    keys, kin, vin, kout, vout = _pass_inputs(n, 2)
    with pytest.raises(sdgs.SdgsError) as e:
        sdgs.lookback_selftest(kin, vin, kout, vout, n, first_ticket=first_ticket, spin_limit=2000)
    assert e.value.code == 5 and "gave up" in str(e.value)
    torch.cuda.synchronize()
    assert (kout[n:].cpu().numpy() == SENTINEL).all() and (vout[n:].cpu().numpy() == SENTINEL).all()
    written = vout[:n].cpu().numpy()
    written = written[written != SENTINEL]
    assert len(written) > 0 and written.min() >= 0 and written.max() < n  # only input values
    # the context is still usable: an ordinary pass right after sorts correctly
    keys, kin, vin, kout, vout = _pass_inputs(n, 3)
    sdgs.lookback_selftest(kin, vin, kout, vout, n, first_ticket=0, spin_limit=2000)
    np.testing.assert_array_equal(vout[:n].cpu().numpy(), np.argsort(keys & 255, kind="stable"))


def test_binning_failure_empties_the_lists_and_is_reported():
    scene, cam = synth.config_scene(0), synth.config_cameras(0)[0]
    got, (dev, st, view, proj) = U.gpu_project(scene, cam)
    bins = sdgs.BinBuffers(scene.n, 1 << 20, cam.width, cam.height)
    k = sdgs.bin_sort(proj, view, bins, sync=True)
    assert k > 0
    with pytest.raises(sdgs.SdgsError) as e:
        sdgs.bin_sort_failure_selftest(proj, view, bins, sync=True)
    assert e.value.code == 5
    assert int(bins.num_instances.item()) == -1
    assert int(bins.ranges.abs().sum().item()) == 0
    img, T, nc = U.gpu_render(proj, bins, view)
    np.testing.assert_array_equal(img, np.broadcast_to(np.asarray(cam.bg, np.float32), img.shape))
    assert (T == 1).all() and (nc == 0).all()
    # without a host count the call enqueues the same and returns OK; the count shows the failure
    sdgs.bin_sort_failure_selftest(proj, view, bins, sync=False)
    torch.cuda.synchronize()
    assert int(bins.num_instances.item()) == -1
    # and the next ordinary call bins the frame again
    assert sdgs.bin_sort(proj, view, bins, sync=True) == k


def test_span_walk_wait_gives_up_and_the_failure_is_reported():
    """The span walk's blocks start at ticket 1, so the block that waits on block 0 (which never
    runs) gives up after its 2000 polling rounds: the call reports SDGS_ERR_TIMEOUT, the count is
    -1, every list is empty, nothing was written outside the buffers, and the next ordinary call
    bins the frame again."""
    scene, cam = synth.config_scene(0), synth.config_cameras(0)[0]
    got, (dev, st, view, proj) = U.gpu_project(scene, cam)
    cap = 1 << 20
    bins = sdgs.BinBuffers(scene.n, cap + 4096, cam.width, cam.height)
    guard = bins.point_list[cap:]
    bins.capacity = cap  # the buffers' last 4096 entries lie past the capacity the call sees
    guard.fill_(-7)
    k = sdgs.bin_sort(proj, view, bins, sync=True)
    assert k > 0 and scene.n > 512  # several walk blocks
    with pytest.raises(sdgs.SdgsError) as e:
        sdgs.span_walk_selftest(proj, view, bins, first_ticket=1, spin_limit=2000, sync=True)
    assert e.value.code == 5
    assert int(bins.num_instances.item()) == -1
    assert int(bins.ranges.abs().sum().item()) == 0
    assert (guard == -7).all()
    assert sdgs.bin_sort(proj, view, bins, sync=True) == k

