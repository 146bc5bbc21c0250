"""The batch autotuner's choice logic, with a fake runner and a fake clock (no GPU)."""
import pytest

from paper_2403_11651_gb300 import batch


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_autotune_picks_the_fastest_and_skips_repeats(monkeypatch):
    clock = FakeClock()
    made = []
    # seconds per probe for each (lanes, chunk); 4 lanes with chunk 32 is the fastest
    cost = {(1, 16): 9.0, (1, 32): 8.0, (2, 16): 5.0, (2, 32): 4.0, (3, 16): 3.5,
            (3, 32): 3.0, (4, 16): 2.5, (4, 32): 1.0}

    class FakeRunner:
        def __init__(self, items, lanes, chunk):
            self.key = (min(lanes, len(items)), chunk)
            self.warm = True
            self.closed = False
            made.append(self)

        def run(self, n):
            if self.warm:            # the warm-up chunk is not timed
                assert n == self.key[1]
                self.warm = False
            else:
                clock.t += cost[self.key]

        def close(self):
            self.closed = True

    monkeypatch.setattr(batch, "BatchOverfitter", FakeRunner)
    items = [object()] * 3
    best, table = batch.autotune(items, lanes_options=(1, 2, 4, 8), chunk_options=(16, 32),
                                 probe_iters=64, timer=clock)
    # lanes 4 and 8 clamp to the 3 images: one candidate per chunk, measured once
    assert set(table) == {(1, 16), (1, 32), (2, 16), (2, 32), (3, 16), (3, 32)}
    assert len(made) == 6 and all(r.closed for r in made)
    assert best == (3, 32)
    assert table[best] == pytest.approx(3.0)


def test_autotune_breaks_ties_towards_fewer_lanes(monkeypatch):
    clock = FakeClock()

    class FakeRunner:
        def __init__(self, items, lanes, chunk):
            self.first = True

        def run(self, n):
            if not self.first:
                clock.t += 1.0
            self.first = False

        def close(self):
            pass

    monkeypatch.setattr(batch, "BatchOverfitter", FakeRunner)
    best, table = batch.autotune([object()] * 8, lanes_options=(8, 2), chunk_options=(32, 16),
                                 timer=clock)
    assert best == (2, 16) and len(table) == 4
