"""Sharded search on one GPU: the shards of a split search, run one after
the other, merge to the unsharded result bit for bit.

* One map's grid split by trajectory index into 2, 3 or 5 ranges
  (morse_grid_chi2_range per range, morse_topk_merge of the lists) equals
  morse_grid_chi2 in every field of every record.
* A sweep's maps split into 3 blocks (morse_sweep per block, lists
  concatenated in map order) equals the whole sweep.
The same shard and merge code runs one process per GPU under
torch.distributed (tests/test_shard_gloo.py covers the gather on CPU ranks).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("idx", "chi2", "t0", "tE", "u0", "alpha", "Fs", "Fb", "flags")


@pytest.fixture(scope="module")
def m():
    import paper_1511_01157_gb300 as lib
    return lib


@pytest.fixture(scope="module")
def setup(m):
    ctx = m.Context(0)
    t = synth.epoch_times(600, 11)
    F, sig = synth.photometry(0.3 + 1.0 / np.sqrt(0.02 + (t / 25.0) ** 2),
                              11)
    ev = ctx.event(t, F, sig)
    yield ctx, ev
    ctx.close()


@pytest.mark.parametrize("world,k", [(2, 16), (3, 100), (5, 7)])
def test_trajectory_shards_merge_to_the_whole_search(m, setup, world, k):
    from paper_1511_01157_gb300 import shard
    ctx, ev = setup
    mp = ctx.build_map(0.9, 5e-3, 2.0, 256, 2000, image_halfwidth=3.0,
                       deflect="fp32")
    grid = m.Grid.make(20, 36, 10, 12, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0,
                       True, True, k)
    whole = ctx.grid_chi2(ev, mp, grid)
    gather = shard.LocalGather()
    for rank in range(world):
        merged = shard.search(ctx, ev, mp, grid, rank, world, gather)
    for f in FIELDS:
        assert np.array_equal(merged[f], whole[f]), f
    # a range shorter than K pads its list; ranges are checked
    one = ctx.grid_chi2_range(ev, mp, grid, grid.size - 3, 3)
    assert (one["idx"][:3] >= grid.size - 3).all()
    assert (one["idx"][3:] == -1).all() and np.isinf(one["chi2"][3:]).all()
    for first, count in ((-1, 5), (0, 0), (grid.size - 2, 3)):
        with pytest.raises(m.MorseError) as e:
            ctx.grid_chi2_range(ev, mp, grid, first, count)
        assert e.value.status == m.EINVAL
    mp.free()


def test_map_shards_concatenate_to_the_whole_sweep(m, setup):
    from paper_1511_01157_gb300 import shard
    ctx, ev = setup
    S = np.array([0.5, 0.8, 1.0, 1.3, 2.0, 2.6, 0.7])
    Q = np.array([1e-3, 1e-2, 3e-4, 1e-1, 1e-4, 2e-3, 5e-2])
    grid = m.Grid.make(12, 24, 8, 8, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0, True,
                       True, 12)
    whole = ctx.sweep(ev, S, Q, 2.0, 256, 1500, grid, image_halfwidth=3.0,
                      deflect="fp32")
    gather = shard.LocalGather()
    for rank in range(3):
        lists = shard.sweep(ctx, ev, S, Q, 2.0, 256, 1500, grid, rank, 3,
                            gather, image_halfwidth=3.0, deflect="fp32")
    assert lists.shape == whole.shape
    for f in FIELDS:
        assert np.array_equal(lists[f], whole[f]), f
    mi, best = shard.best_over_maps(lists, 5)
    j = int(np.argmin(whole["chi2"][:, 0]))
    assert mi[0] == j and best[0]["chi2"] == whole[j, 0]["chi2"]
