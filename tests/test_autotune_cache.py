"""Autotuner cache (host logic): jobs whose degree histograms, K and device agree share a
key; the cache survives a reload from its file."""
import numpy as np

from paper_1705_10633_gb300.autotune import TuningCache, tuning_key


def test_key_groups_alike_jobs_and_separates_others():
    rng = np.random.default_rng(0)
    du = rng.lognormal(4.5, 1.2, 200_000).astype(int) + 1
    dv = rng.lognormal(7.0, 1.0, 5_000).astype(int) + 1
    k1 = tuning_key(32, du, dv, "GPU A")
    # a resample from the same distributions bins alike
    du2 = rng.lognormal(4.5, 1.2, 200_000).astype(int) + 1
    dv2 = rng.lognormal(7.0, 1.0, 5_000).astype(int) + 1
    assert tuning_key(30, du2, dv2, "GPU A") == k1  # K 30 pads to the same width
    assert tuning_key(40, du, dv, "GPU A") != k1
    assert tuning_key(32, du, dv, "GPU B") != k1
    assert tuning_key(32, du // 8 + 1, dv, "GPU A") != k1
    assert tuning_key(32, du[:2000], dv, "GPU A") != k1  # another order of magnitude


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tuning.json")
    c = TuningCache(path)
    assert c.get("k") is None
    c.put("k", (48, 0, -1))
    c2 = TuningCache(path)
    assert c2.get("k") == (48, 0, -1)
