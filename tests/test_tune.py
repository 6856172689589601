"""Host logic of the launch autotuner (paper_2102_08756_gb300/tune.py) without
a GPU: every (variant, orbit tile, lags-per-CTA) candidate is timed through the
handle's stage events, candidates the library refuses are skipped (the
register-prefetch variant only runs the 128-record tile), the fastest is
applied and cached under a key with grid, history, precision, compensation and
GPU name, and a cache hit applies the stored launch without any trial."""
import json

import pytest

torch = pytest.importorskip("torch")


class FakeHandle:
    """Stands in for paper_2102_08756_gb300.sbim.SBIM: convolution time per launch."""

    def __init__(self, times, refuse=(), refuse_tiles=()):
        self.n1, self.n3, self.n_cut, self.precision, self.kahan = 64, 32, 1500, "fp32", True
        self.device = 0
        self.times, self.refuse, self.refuse_tiles = times, set(refuse), set(refuse_tiles)
        self.config, self.applied, self.steps, self.prof = None, [], 0, False
        self.tile = 128

    def set_conv_config(self, variant, lags_per_cta=0):
        if (variant, lags_per_cta) in self.refuse:
            raise RuntimeError("launch shape refused")
        self.config = (variant, lags_per_cta)
        self.applied.append(self.config)

    def set_conv_tile(self, tile):
        if tile in self.refuse_tiles:
            raise RuntimeError("record count not a multiple of the tile")
        self.tile = tile

    def step(self, u, v, tau=None):
        self.steps += 1
        if self.prof:
            self.prof_steps += 1

    def set_profiling(self, enable=True):
        self.prof, self.prof_steps = enable, 0

    def stage_times(self):
        t = self.times[self.config] + (0.0 if self.config[0] == 0 else TILE_COST[self.tile])
        return {"convolution": t * self.prof_steps}, self.prof_steps

    def check(self):
        pass


TILE_COST = {64: 0.25, 128: 0.0, 256: 0.5}


@pytest.fixture(autouse=True)
def fake_gpu_name(monkeypatch):
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "GB300-test")


def _times():
    t = {}
    for var in (1, 2, 3, 0):
        for lpc in (0, 256, 512, 1024):
            t[(var, lpc)] = 10.0 + var + lpc / 1000.0
    t[(3, 512)] = 7.5
    return t


def test_picks_fastest_and_skips_refused_launches(tmp_path):
    from paper_2102_08756_gb300.tune import autotune
    times = _times()
    h = FakeHandle(times, refuse={(2, 0), (2, 256)}, refuse_tiles={256})
    u = torch.zeros(3, 32, 64)
    best, table = autotune(h, u, u, steps=3, cache=str(tmp_path / "c.json"))
    assert best == {"variant": 3, "tile": 128, "lags_per_cta": 512, "conv_ms": 7.5}
    assert h.config == (3, 512) and h.tile == 128
    # every candidate but the refused ones, each timed from its own profiled steps:
    # 3 TMA variants x 2 tiles x 4 chunkings, minus 2 refused shapes x 2 tiles,
    # plus the register variant at the one tile
    assert len(table) == 3 * 2 * 4 - 2 * 2 + 4
    assert {r["tile"] for r in table} == {64, 128}
    assert all(abs(r["conv_ms"] - times[(r["variant"], r["lags_per_cta"])]
                   - (0.0 if r["variant"] == 0 else TILE_COST[r["tile"]])) < 1e-12 for r in table)
    db = json.load(open(tmp_path / "c.json"))
    assert db == {"64x32:1500:fp32:1:GB300-test": best}


def test_a_faster_tile_is_chosen():
    from paper_2102_08756_gb300.tune import autotune
    times = _times()
    h = FakeHandle(times)
    saved = dict(TILE_COST)
    try:
        TILE_COST.update({64: 0.0, 128: 0.0, 256: -1.0})
        best, table = autotune(h, torch.zeros(3, 32, 64), torch.zeros(3, 32, 64), steps=1)
    finally:
        TILE_COST.update(saved)
    assert best["tile"] == 256 and h.tile == 256 and best["variant"] == 3
    assert {r["tile"] for r in table} == {64, 128, 256}


def test_cache_hit_applies_stored_launch_without_trials(tmp_path, monkeypatch):
    from paper_2102_08756_gb300.tune import autotune
    cache = tmp_path / "c.json"
    json.dump({"64x32:1500:fp32:1:GB300-test": {"variant": 1, "lags_per_cta": 1024, "conv_ms": 3.0}},
              open(cache, "w"))
    h = FakeHandle(_times())
    u = torch.zeros(3, 32, 64)
    best, table = autotune(h, u, u, cache=str(cache))
    assert table is None and h.steps == 0
    assert h.applied == [(1, 1024)] and best["lags_per_cta"] == 1024 and h.tile == 128
    # another GPU name misses the cache and tunes
    h2 = FakeHandle(_times())
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "other")
    best2, table2 = autotune(h2, u, u, steps=1, cache=str(cache))
    assert table2 is not None and best2["variant"] == 3
    assert set(json.load(open(cache))) == {"64x32:1500:fp32:1:GB300-test", "64x32:1500:fp32:1:other"}


def test_chunkings_stop_below_the_history_length():
    from paper_2102_08756_gb300.tune import autotune
    h = FakeHandle(_times())
    h.n_cut = 600
    u = torch.zeros(3, 32, 64)
    _, table = autotune(h, u, u, steps=1)
    assert sorted({r["lags_per_cta"] for r in table}) == [0, 256, 512]
