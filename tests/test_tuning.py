"""Host logic of the batched apply's tile autotuner (no GPU): the workload key, the cache file
and the choice between cached, measured and default shapes (the library's tuner and shape
calls are replaced by fakes here; tests/test_gpu_batch_tune.py runs them on the GPU)."""
import json

import pytest

import paper_1811_05335_gb300 as g
from paper_1811_05335_gb300 import tuning


def stats(P=4096, mean_column=38.0, max_column=780, m=6, ratio=3.0):
    M = [256 * (1 + (i % 32)) for i in range(P)]
    N = [int(ratio * v) for v in M]
    return tuning.workload_stats(M, N, m, int(mean_column * 2 * sum(M)), max_column)


def test_key_buckets_statistics():
    k = tuning.stats_key(stats(), "GPU")
    assert k == tuning.stats_key(stats(mean_column=39.0, max_column=700), "GPU")   # same buckets
    assert k != tuning.stats_key(stats(P=2048), "GPU")
    assert k != tuning.stats_key(stats(mean_column=80.0), "GPU")
    assert k != tuning.stats_key(stats(max_column=1100), "GPU")
    assert k != tuning.stats_key(stats(max_column=300), "GPU")
    assert k != tuning.stats_key(stats(m=4), "GPU")
    assert k != tuning.stats_key(stats(ratio=2.0), "GPU")
    assert k != tuning.stats_key(stats(), "OTHER")
    assert k.startswith("GPU|m6|P2^12|")


def test_cache_roundtrip_and_version(tmp_path):
    path = tmp_path / "c.json"
    assert tuning.load_cache(str(path)) == {}
    tuning.save_cache({"b": {"shape": 1}, "a": {"shape": 2}}, str(path))
    assert tuning.load_cache(str(path)) == {"a": {"shape": 2}, "b": {"shape": 1}}
    path.write_text(json.dumps({"version": 99, "entries": {}}))
    with pytest.raises(ValueError):
        tuning.load_cache(str(path))


def test_committed_cache_is_valid():
    entries = tuning.load_cache(tuning.DEFAULT_CACHE)
    shapes = g.infft_batch_tile_shapes()
    assert len(shapes) == 11 and shapes[4] == (128, 2048)         # the default: the fixed rule
    for key, e in entries.items():
        assert 0 <= e["shape"] < len(shapes)
        assert (e["cols"], e["weights"]) == shapes[e["shape"]]
        assert len(e["ms"]) == len(shapes) and min(e["ms"]) == e["ms"][e["shape"]]
        assert key.startswith(e["device"] + "|")


class FakeBatch:
    M = [256, 512, 1024]
    N = [700, 1500, 3000]


def fake_binding(monkeypatch, ms):
    calls = {"set": [], "tune": 0}
    shapes = [(64, 1024), (64, 2048), (64, 4096), (128, 1024), (128, 2048), (128, 4096), (256, 2048), (256, 4096)]
    monkeypatch.setattr(tuning.binding, "infft_batch_get_info", lambda b: {"m": 6, "nnz": 120000, "max_column": 90})
    monkeypatch.setattr(tuning.binding, "infft_batch_tile_shapes", lambda: shapes)
    monkeypatch.setattr(tuning.binding, "infft_batch_set_tile_shape", lambda b, s, st=None: calls["set"].append(s))
    monkeypatch.setattr(tuning.binding, "infft_batch_get_tile_shape", lambda b: 4)

    def tune(b, repeats, stream):
        calls["tune"] += 1
        return min(range(len(ms)), key=ms.__getitem__), list(ms)
    monkeypatch.setattr(tuning.binding, "infft_batch_tune_apply", tune)
    return calls


def test_autotune_measures_writes_then_hits_cache(monkeypatch, tmp_path):
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    ms = [0.9, 0.8, 0.85, 0.7, 0.6, 0.65, 0.75, 0.95]
    calls = fake_binding(monkeypatch, ms)
    path = str(tmp_path / "cache.json")
    r = tuning.autotune_batch(FakeBatch(), cache=path, write=path)
    assert r["source"] == "measured" and r["shape"] == 4 and calls["tune"] == 1
    entry = tuning.load_cache(path)[r["key"]]
    assert entry["shape"] == 4 and (entry["cols"], entry["weights"]) == (128, 2048) and entry["device"] == "FakeGPU"
    r2 = tuning.autotune_batch(FakeBatch(), cache=path)
    assert r2["source"] == "cache" and r2["shape"] == 4 and calls["tune"] == 1 and calls["set"] == [4]
    r3 = tuning.autotune_batch(FakeBatch(), cache=str(tmp_path / "none.json"), tune_if_missing=False)
    assert r3["source"] == "default" and calls["set"][-1] == -1 and calls["tune"] == 1
