"""Host logic of the warm-start experiment (no GPU): the cost checkpoints, the first
checkpoint at or below a target, and run_schedule's bookkeeping against a fake library."""
import numpy as np
import pytest

from paper_2403_11651_gb300 import warm_bench as wb


@pytest.mark.parametrize("iters,every,want", [
    (1000, 25, list(range(0, 1000, 25)) + [1000]),
    (30, 25, [0, 25, 30]),
    (50, 25, [0, 25, 50]),
    (0, 25, [0]),
])
def test_checkpoints(iters, every, want):
    assert wb.checkpoints(iters, every) == want


def test_first_at_or_below():
    assert wb.first_at_or_below([5.0, 3.0, 2.0, 1.0], 2.0) == 2
    assert wb.first_at_or_below([5.0, 3.0], 2.9) is None
    assert wb.first_at_or_below([1.0, 3.0], 2.0) == 0


def test_run_schedule_reads_cost_at_every_checkpoint(monkeypatch):
    calls = {"iters": [], "reads": 0}
    state = {"done": 0}

    def encode(ctx, n):
        calls["iters"].append(n)
        state["done"] += n

    def rd_cost(ctx, hard):
        calls["reads"] += 1
        return (0.0, 0.0, 100.0 / (1 + state["done"]))

    monkeypatch.setattr(wb.cc, "cc_init_image", lambda *a, **k: object())
    monkeypatch.setattr(wb.cc, "cc_set_latents", lambda ctx, y: None)
    monkeypatch.setattr(wb.cc, "cc_encode_iters", encode)
    monkeypatch.setattr(wb.cc, "cc_iteration", lambda ctx: state["done"])
    monkeypatch.setattr(wb.cc, "cc_rd_cost", rd_cost)
    monkeypatch.setattr(wb.cc, "cc_free", lambda ctx: None)
    rgb = np.zeros((16, 16, 3), np.uint8)
    costs, secs = wb.run_schedule(None, rgb, None, None, 60, 25)
    assert calls["iters"] == [25, 25, 10]
    assert calls["reads"] == len(wb.checkpoints(60, 25)) == len(costs) == len(secs) == 4
    np.testing.assert_allclose(costs, [100.0 / (1 + d) for d in (0, 25, 50, 60)])
    assert secs[0] == 0.0 and np.all(np.diff(secs) >= 0)
