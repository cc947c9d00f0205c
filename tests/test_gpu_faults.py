"""Failure detection of the library's error paths, without faulting the GPU.

* A device wait that gives up: the block top-K lock of the searches is
  taken at the start of the search by an injected fault, and each wait for
  it gives up after a few spins (~64 ns each) and sets the block's error
  bit; the host reads it after the stream has synchronised and returns
  MORSE_ETIMEOUT.  Nothing waits without a bound, so nothing hangs.  The
  same context then searches normally and gets the same results as before
  (single searches, the allocation-free search, the batch and a sweep).
* An allocation that fails: the next device allocation is made to fail on
  the host (as cudaMalloc does when the device is out of memory, but with
  nothing allocated); the call returns MORSE_ENOMEM and the context stays
  usable.
* Invalid arguments return MORSE_EINVAL before any GPU work (other files
  cover the method's own argument checks).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_1511_01157_gb300 as lib
    return lib


@pytest.fixture(scope="module")
def setup(m):
    ctx = m.Context(0)
    t = synth.epoch_times(500, 3)
    F, sig = synth.photometry(0.3 + 1.0 / np.sqrt(0.03 + (t / 18.0) ** 2), 3)
    ev = ctx.event(t, F, sig)
    mp = ctx.build_map(1.0, 1e-3, 2.0, 256, 1500, image_halfwidth=3.0,
                       deflect="fp32")
    # 16 warp groups per block, every one merging candidates into the block
    # list: the lock is wanted by every warp
    grid = m.Grid.make(16, 36, 10, 10, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0,
                       True, True, 64)
    yield ctx, ev, mp, grid
    ctx.inject_fault(m.FAULT_NONE, 0)
    ctx.close()


def test_lock_wait_gives_up_and_context_recovers(m, setup):
    ctx, ev, mp, grid = setup
    ref = ctx.grid_chi2(ev, mp, grid)
    # a sweep of three maps (builds on a second stream, searches on the
    # sweep's own stream) before the fault, for the comparison after it
    S, Q = np.array([0.9, 1.0, 1.1]), np.array([1e-3, 3e-3, 1e-2])
    sw_ref = ctx.sweep(ev, S, Q, 2.0, 128, 600, grid, image_halfwidth=3.0)
    ctx.inject_fault(m.FAULT_LOCK_HELD, 4)
    for call in (lambda: ctx.grid_chi2(ev, mp, grid),
                 lambda: ctx.grid_chi2_noalloc(ev, mp, grid),
                 lambda: ctx.grid_chi2_batch([ev], [mp], grid),
                 lambda: ctx.sweep(ev, S, Q, 2.0, 128, 600, grid,
                                   image_halfwidth=3.0)):
        with pytest.raises(m.MorseError) as e:
            call()
        assert e.value.status == m.ETIMEOUT
        assert "lock" in str(e.value)
    ctx.inject_fault(m.FAULT_NONE, 0)
    again = ctx.grid_chi2(ev, mp, grid)
    for f in ("idx", "chi2", "Fs", "Fb"):
        assert np.array_equal(again[f], ref[f]), f
    sw = ctx.sweep(ev, S, Q, 2.0, 128, 600, grid, image_halfwidth=3.0)
    for f in ("idx", "chi2", "Fs", "Fb"):
        assert np.array_equal(sw[f], sw_ref[f]), f
    batch = ctx.grid_chi2_batch([ev], [mp], grid)
    assert np.array_equal(batch[0, 0]["idx"], ref["idx"])


def test_failed_allocations_return_enomem(m, setup):
    ctx, ev, mp, grid = setup
    t = synth.epoch_times(200, 4)
    F, sig = synth.photometry(1.0 + 0.1 * np.cos(t), 4)
    # the map's first device buffer
    ctx.inject_fault(m.FAULT_ALLOC, 1)
    with pytest.raises(m.MorseError) as e:
        ctx.build_map(1.0, 1e-2, 2.0, 64, 200)
    assert e.value.status == m.ENOMEM
    # its third (the first two are made and released again)
    ctx.inject_fault(m.FAULT_ALLOC, 3)
    with pytest.raises(m.MorseError) as e:
        ctx.build_map(1.0, 1e-2, 2.0, 64, 200)
    assert e.value.status == m.ENOMEM
    # the event upload
    ctx.inject_fault(m.FAULT_ALLOC, 1)
    with pytest.raises(m.MorseError) as e:
        ctx.event(t, F, sig)
    assert e.value.status == m.ENOMEM
    # the search workspace when it has to grow
    bigger = m.Grid.make(40, 72, 20, 20, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0,
                         True, True, 2048)
    ctx.inject_fault(m.FAULT_ALLOC, 1)
    with pytest.raises(m.MorseError) as e:
        ctx.grid_chi2(ev, mp, bigger)
    assert e.value.status == m.ENOMEM
    # everything works again afterwards, with the same results
    ctx.inject_fault(m.FAULT_NONE, 0)
    mp2 = ctx.build_map(1.0, 1e-2, 2.0, 64, 200)
    ev2 = ctx.event(t, F, sig)
    r1 = ctx.grid_chi2(ev2, mp2, grid)
    r2 = ctx.grid_chi2(ev2, mp2, grid)
    assert np.array_equal(r1["idx"], r2["idx"])
    assert np.isfinite(ctx.grid_chi2(ev, mp, bigger)["chi2"][0])
    mp2.free()
    ev2.free()


def test_inject_fault_rejects_bad_arguments(m, setup):
    ctx, *_ = setup
    for kind, arg in ((m.FAULT_LOCK_HELD, 0), (m.FAULT_LOCK_HELD, 1 << 21),
                      (m.FAULT_ALLOC, 0), (7, 1)):
        with pytest.raises(m.MorseError) as e:
            ctx.inject_fault(kind, arg)
        assert e.value.status == m.EINVAL
    ctx.inject_fault(m.FAULT_NONE, 0)
