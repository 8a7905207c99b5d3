"""Host logic of the batched solver's autotuner with the timed solves replaced
by fixed timings: the buckets of n, the rule "the largest width within 5 % of
the fastest", the per-device cache and its JSON file, the per-matrix widths,
and the strategy choice."""
import json

import numpy as np
import pytest
import torch

from paper_1401_2720_gb300 import autotune


@pytest.fixture
def fake_device(monkeypatch):
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "fake GPU")
    autotune._cache.clear()
    autotune._strategy_cache.clear()
    yield
    autotune._cache.clear()
    autotune._strategy_cache.clear()


def test_bucket_edges():
    assert [autotune.bucket_of(n) for n in (1, 32, 33, 64, 65, 128, 129, 256, 257, 512, 513, 1024)] == \
        [0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5]
    with pytest.raises(ValueError):
        autotune.bucket_of(1025)


def test_tune_keeps_the_largest_width_within_5_percent(fake_device, monkeypatch, tmp_path):
    # per bucket: b = 8 fastest; 16 within 5 % except in bucket 1; 32 always > 5 % slower
    timings = {0: {8: 1.0, 16: 1.04, 32: 1.2}, 1: {8: 1.0, 16: 1.06, 32: 1.3}, 4: {8: 2.0, 16: 1.9, 32: 1.99}}
    calls = []

    def fake_time(pick, b, device, repeats, strategy="rR"):
        k = autotune.bucket_of(pick[0].shape[1])
        assert all(autotune.bucket_of(a.shape[1]) == k for a in pick)
        calls.append((k, b))
        return timings[k][b]

    monkeypatch.setattr(autotune, "_time_batch", fake_time)
    mats = [np.zeros((40, 20)), np.zeros((64, 30)), np.zeros((80, 50)), np.zeros((400, 300))]
    path = str(tmp_path / "widths.json")
    table = autotune.tune(mats, sample=8, repeats=1, path=path, device="cpu")
    assert table == {0: 16, 1: 8, 4: 32}
    assert json.load(open(path)) == {"fake GPU": {"0": 16, "1": 8, "4": 32}}
    calls.clear()
    assert autotune.tune(mats, device="cpu") == table and calls == []     # served from the cache
    assert list(autotune.block_widths([20, 50, 300, 100], table, default=8)) == [16, 8, 32, 8]


def test_tune_strategy_picks_the_fastest(fake_device, monkeypatch):
    times = {"rR": 3.0, "rC": 2.5, "modulus": 2.7}
    seen = []

    def fake_time(pick, b, device, repeats, strategy="rR"):
        seen.append((len(pick), tuple(b), strategy))
        return times[strategy]

    monkeypatch.setattr(autotune, "_time_batch", fake_time)
    mats = [np.zeros((30, n)) for n in (8, 20, 40, 30, 12)]
    best, got = autotune.tune_strategy(mats, {0: 16, 1: 32}, sample=3, repeats=1, device="cpu")
    assert best == "rC" and got == times
    assert all(n == 3 for n, _, _ in seen) and {s for _, _, s in seen} == set(times)
    assert all(set(b) <= {8, 16, 32} for _, b, _ in seen)
