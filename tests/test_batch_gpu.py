"""Several images overfitted at once on separately loaded copies of the library: every
image's iterations are bit-identical to running it alone."""
import numpy as np
import pytest

from paper_2403_11651_gb300 import coolchic as cc
from paper_2403_11651_gb300 import synthetic as syn
from paper_2403_11651_gb300 import batch as batch_mod
from paper_2403_11651_gb300.batch import BatchOverfitter

from .helpers import config_dict

pytestmark = pytest.mark.gpu

ITEMS = [("c1", 48, 64, 1e-3), ("c2", 40, 56, 1e-2), ("t300", 64, 64, 1e-3),
         ("c1", 33, 70, 1e-4), ("c2", 96, 80, 3e-3)]


def _items():
    out = []
    for k, (arch, H, W, lam) in enumerate(ITEMS):
        d = config_dict(arch, lam=lam, total_iters=24, ste_frac=0.25)
        cfg = cc.make_config(d, seed=k)
        init = cc.flatten_params(syn.initial_parameters(syn.ArchSizes.from_config(d), k), cfg)
        out.append((syn.synthetic_image(H, W, k), d, init, k))
    return out


def test_batch_matches_single_runs():
    items = _items()
    b = BatchOverfitter(items, lanes=3, chunk=4)
    try:
        assert len({id(lib) for lib in b.libs}) == 3
        b.run(24)
        got = [b.losses(i, 0, 24) for i in range(len(items))]
        got_rd = b.rd_costs()
    finally:
        b.close()
    for i, (rgb, d, init, seed) in enumerate(items):
        cfg = cc.make_config(d, seed=seed)
        ctx = cc.cc_init_image(cfg, rgb, rgb.shape[0], rgb.shape[1], init)
        try:
            cc.cc_encode_iters(ctx, 24)
            assert np.array_equal(cc.cc_get_losses(ctx, 0, 24), got[i]), i
            assert cc.cc_rd_cost(ctx, True) == got_rd[i], i
        finally:
            cc.cc_free(ctx)


def test_autotuned_batch_matches_one_lane():
    """The autotuner measures every candidate on throwaway contexts; the configuration it
    picks gives the same results as one lane."""
    items = _items()
    best, table = batch_mod.autotune(items, lanes_options=(1, 2, 5), chunk_options=(16, 32),
                                     probe_iters=32)
    assert set(table) == {(1, 16), (1, 32), (2, 16), (2, 32), (5, 16), (5, 32)}
    assert best in table and all(t > 0 for t in table.values())
    out = []
    for lanes, chunk in ((1, 16), best):
        b = BatchOverfitter(items, lanes=lanes, chunk=chunk)
        try:
            b.run(24)
            out.append(([b.losses(i, 0, 24) for i in range(len(items))], b.rd_costs()))
        finally:
            b.close()
    assert out[0][1] == out[1][1]
    for a, c in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, c)
