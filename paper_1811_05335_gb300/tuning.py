"""Autotuning of the batched apply's spreading tiles, with a cache keyed by workload statistics.

The batched spreading cuts every problem's grid into tiles (grid points per tile, weights per
block: infft_batch_tile_shapes()); which shape is fastest depends on the column lengths and node
density of the batch, so the shape is chosen by measurement (infft_batch_tune_apply, CUDA events
on the batch's own B_opt) and remembered per workload class and device.  Every shape gives
bit-identical results, so a cached choice can never change an answer, only the time.

Cache file (JSON): {"version": 1, "entries": {key: {"shape": id, "cols": c, "weights": w,
"ms": [per shape], "device": name}}}.  The package ships one (tune_cache.json beside this file)
holding the measured choices of the batched workloads it has been run on.
"""
import json
import math
import os
import tempfile

from . import binding

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
CACHE_VERSION = 1


def workload_stats(M, N, m, nnz, max_column):
    """The statistics a tile shape depends on: problem count, sizes, column lengths."""
    M = [int(v) for v in M]
    N = [int(v) for v in N]
    sum_M, sum_N = sum(M), sum(N)
    return {"m": int(m), "P": len(M), "sum_M": sum_M, "sum_N": sum_N,
            "min_M": min(M), "max_M": max(M), "nodes_per_coef": sum_N / sum_M,
            "mean_column": nnz / (2.0 * sum_M), "max_column": int(max_column)}


def stats_key(st, device):
    """Bucketed key of workload statistics: P in octaves, M range in octaves, N/M in halves,
    mean column length in quarter octaves, the largest column in octaves, m and the device."""
    oct_ = lambda v: int(round(math.log2(max(v, 1))))
    return (f"{device}|m{st['m']}|P2^{oct_(st['P'])}|M2^{oct_(st['min_M'])}-2^{oct_(st['max_M'])}"
            f"|N/M{round(st['nodes_per_coef'] * 2) / 2:g}"
            f"|col2^{round(math.log2(max(st['mean_column'], 1.0)) * 4) / 4:g}"
            f"|max2^{math.ceil(math.log2(max(st['max_column'], 1)))}")


def batch_workload_key(batch, device=None):
    """Cache key of a precomputed batch (its statistics from infft_batch_get_info)."""
    info = binding.infft_batch_get_info(batch)
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    st = workload_stats(batch.M, batch.N, info["m"], info["nnz"], info["max_column"])
    return stats_key(st, device), st


def load_cache(path=DEFAULT_CACHE):
    """Entries of a cache file ({} when the file is absent)."""
    if not path or not os.path.exists(path):
        return {}
    with open(path) as fh:
        data = json.load(fh)
    if data.get("version") != CACHE_VERSION:
        raise ValueError(f"{path}: cache version {data.get('version')} (expected {CACHE_VERSION})")
    return dict(data.get("entries", {}))


def save_cache(entries, path):
    """Writes the entries atomically (temporary file in the same folder, then rename)."""
    folder = os.path.dirname(os.path.abspath(path))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=folder, suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump({"version": CACHE_VERSION, "entries": dict(sorted(entries.items()))}, fh, indent=1)
        fh.write("\n")
    os.replace(tmp, path)


def autotune_batch(batch, stream=None, cache=DEFAULT_CACHE, tune_if_missing=True, write=None, repeats=10):
    """Sets the batch's tile shape from the cache, or by measurement when the workload class is
    not cached (and tune_if_missing), else keeps the default rule.  write: a cache path that
    receives the measured entry (merged with the entries already there).  Returns
    {"key", "shape", "cols", "weights", "source": "cache" | "measured" | "default", "ms"}.
    Requires infft_batch_precompute."""
    key, st = batch_workload_key(batch)
    shapes = binding.infft_batch_tile_shapes()
    entries = load_cache(cache)
    hit = entries.get(key)
    if hit is not None and 0 <= int(hit["shape"]) < len(shapes):
        shape, source, ms = int(hit["shape"]), "cache", hit.get("ms")
        binding.infft_batch_set_tile_shape(batch, shape, stream)
    elif tune_if_missing:
        shape, ms = binding.infft_batch_tune_apply(batch, repeats, stream)
        source = "measured"
        if write:
            merged = load_cache(write)
            merged[key] = {"shape": shape, "cols": shapes[shape][0], "weights": shapes[shape][1],
                           "ms": [round(v, 5) for v in ms], "device": key.split("|", 1)[0], "stats": st}
            save_cache(merged, write)
    else:
        binding.infft_batch_set_tile_shape(batch, -1, stream)
        shape, source, ms = binding.infft_batch_get_tile_shape(batch), "default", None
    return {"key": key, "shape": shape, "cols": shapes[shape][0], "weights": shapes[shape][1],
            "source": source, "ms": ms}
