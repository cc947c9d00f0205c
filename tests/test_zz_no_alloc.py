"""The allocation-free search entry point (morse_grid_chi2_noalloc).

It serves callers that cannot let the library allocate device memory once
their set-up is over (cudaFree stalls the whole device; fixed memory
budgets reserved at start-up).  This file is named so that pytest collects
it last: if it fails, a run that stops at the first failure has already run
every other test.  It must also pass alone in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

CHI2_RTOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    import paper_1511_01157_gb300 as m
    ctx = m.Context(0)
    t = synth.epoch_times(700, 21)
    # a light curve with a caustic-crossing-like bump; its exact shape does
    # not matter, both entry points search the same data
    f_true = 0.3 + 1.0 / np.sqrt(0.02 + (t / 20.0) ** 2)
    F, sig = synth.photometry(f_true, 21)
    ev = ctx.event(t, F, sig)
    mp = ctx.build_map(0.95, 2e-3, 2.0, 256, 2000, image_halfwidth=3.0,
                       deflect="fp32")
    grid = m.Grid.make(12, 24, 7, 9, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0, True,
                       True, 64)
    yield m, ctx, ev, mp, grid
    mp.free()
    ev.free()
    ctx.close()


def test_noalloc_matches_allocating_search_twice(setup):
    # same kernels, same parameter set-up, same arithmetic: the records are
    # identical bit for bit, on two calls in a row that share the scratch
    m, ctx, ev, mp, grid = setup
    ref = ctx.grid_chi2(ev, mp, grid)
    for _ in range(2):
        got = ctx.grid_chi2_noalloc(ev, mp, grid)
        for f in ("idx", "chi2", "t0", "tE", "u0", "alpha", "Fs", "Fb",
                  "flags"):
            assert np.array_equal(got[f], ref[f]), f


def test_noalloc_does_not_allocate():
    # A fresh context that has only created its event and map: with the
    # next device allocation set to fail, any allocation inside the search
    # would return ENOMEM; and the device's free memory does not move.
    torch = pytest.importorskip("torch")
    import paper_1511_01157_gb300 as m
    ctx = m.Context(0)
    t = synth.epoch_times(400, 5)
    F, sig = synth.photometry(0.3 + 1.0 / np.sqrt(0.05 + (t / 15.0) ** 2), 5)
    ev = ctx.event(t, F, sig)
    mp = ctx.map_from_host(np.ones((128, 128), dtype=np.float32) +
                           np.linspace(0, 1, 128, dtype=np.float32), 2.0)
    grid = m.Grid.make(6, 12, 5, 5, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0, True,
                       True, 8)
    ctx.grid_chi2_noalloc(ev, mp, grid)       # first call: address set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    ctx.inject_fault(m.FAULT_ALLOC, 1)
    for _ in range(3):
        ctx.grid_chi2_noalloc(ev, mp, grid)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0
    # the allocation fault is still armed: the allocating search trips it
    with pytest.raises(m.MorseError) as e:
        ctx.grid_chi2(ev, mp, grid)
    assert e.value.status == m.ENOMEM
    ctx.inject_fault(m.FAULT_NONE, 0)
    mp.free()
    ev.free()
    ctx.close()


def test_noalloc_rejects_oversized_search(setup):
    m, ctx, ev, mp, grid = setup
    # enough trajectories for one block per SM, K = 4096: two per-block
    # lists of 4096 16-byte entries per block exceed the 4 MiB scratch
    big = m.Grid.make(20, 72, 12, 10, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0, True,
                      True, 4096)
    with pytest.raises(m.MorseError) as e:
        ctx.grid_chi2_noalloc(ev, mp, big)
    assert e.value.status == m.EINVAL
    assert "scratch" in str(e.value)
    # the context stays usable
    ok = ctx.grid_chi2_noalloc(ev, mp, grid)
    assert np.isfinite(ok["chi2"][0])
