"""Host logic of the autotuner (no GPU): it times every candidate through the context,
keeps the fastest, applies it, and serves a second call from its cache."""
import pytest

from paper_2507_11603_gb300 import autotune


class FakeRun:
    def __init__(self, ms):
        self.stats = {"elapsed_ms": ms}


class FakeCtx:
    """Records the settings applied and times runs from a table keyed by the setting."""

    def __init__(self, table):
        self.table = table
        self.setting = None
        self.applied = []

    def set_launch(self, block, per_sm):
        self.setting = ("launch", block, per_sm)
        self.applied.append(self.setting)

    def set_grid_exec(self, slots, handoff):
        self.setting = ("grid", slots, handoff)
        self.applied.append(self.setting)

    def set_bursts(self, pipe, burst):
        self.setting = ("bursts", pipe, burst)
        self.applied.append(self.setting)

    def run(self, geom, n_photons, seed, **kw):
        return FakeRun(self.table[self.setting])


@pytest.fixture
def cache(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_device_name", lambda: "fake-device")


def test_tune_run_picks_and_caches(cache):
    table = {("launch", 128, 0): 5.0, ("launch", 64, 0): 3.0, ("launch", 256, 2): 4.0}
    ctx = FakeCtx(table)
    best = autotune.tune_run(ctx, None, "k", n_photons=10, candidates=[(128, 0), (64, 0), (256, 2)])
    assert (best["block"], best["blocks_per_sm"]) == (64, 0) and best["ms"] == 3.0
    assert ctx.setting == ("launch", 64, 0) and len(best["table"]) == 3
    ctx2 = FakeCtx({})  # from the cache: no run at all
    again = autotune.tune_run(ctx2, None, "k", n_photons=10, candidates=[(128, 0)])
    assert (again["block"], again["blocks_per_sm"]) == (64, 0) and ctx2.applied == [("launch", 64, 0)]


@pytest.mark.parametrize("grid,cands,fast", [
    (True, [(0, 0), (65536, 8192)], (0, 0)),
    (False, [(32, 1), (32, 4), (8, 1)], (32, 4)),
])
def test_tune_modes_picks_and_caches(cache, grid, cands, fast):
    kind = "grid" if grid else "bursts"
    table = {(kind, *c): (1.0 if tuple(c) == fast else 2.0 + i) for i, c in enumerate(cands)}
    ctx = FakeCtx(table)
    best = autotune.tune_modes(ctx, None, "m", n_photons=10, candidates=cands, grid=grid)
    assert tuple(best["mode"]) == fast and ctx.setting == (kind, *fast)
    ctx2 = FakeCtx({})
    again = autotune.tune_modes(ctx2, None, "m", n_photons=10, candidates=cands, grid=grid)
    assert tuple(again["mode"]) == fast and ctx2.applied == [(kind, *fast)]
