"""Autotuned tiles of the batched spreading (through the C ABI).

* Every tile shape gives a bit-identical fhat: each column is summed in one order that depends
  on its grid point only, whichever tile holds it and whether the tile's node window is staged
  in shared memory in one piece or in several (a problem of about 900 nodes per column makes
  some windows longer than the staging buffer) or the column is spread in float-float (wide
  columns) by direct loads.
* The tuner returns the shape it measured fastest and leaves the batch on it; the cache
  returns a stored choice without measuring.
The default shape's fhat is held against the FP64 oracle in test_gpu_batch.py, so equality with
it carries that parity to every shape."""
import numpy as np
import pytest

from workloads import chebyshev_jittered, jittered, iid_uniform, complex_normal, trig_poly_eval, make_batch

pytestmark = pytest.mark.gpu

# (M, N, node family, seed): clustered, uniform, jittered, non-power-of-two M, both FFT modes, and
# a dense problem (about 69 nodes per grid cell, columns of about 900 nodes)
SPECS = [(1000, 3500, "cheb", 51), (8190, 16400, "jit", 52), (256, 35000, "unif", 53), (34, 100, "jit", 54),
         (1536, 6000, "cheb", 55), (258, 700, "unif", 56), (10, 25, "unif", 57)]

_cache = {}


def nodes(fam, seed, n):
    return {"cheb": chebyshev_jittered, "jit": jittered, "unif": iid_uniform}[fam](seed, n)


def build(name):
    if name in _cache:
        return _cache[name]
    import torch
    import paper_1811_05335_gb300 as g
    dev = torch.device("cuda:0")
    if name == "mixed":
        M = [s[0] for s in SPECS]
        N = [s[1] for s in SPECS]
        x = np.concatenate([nodes(fam, sd, n) for (_, n, fam, sd) in SPECS])
        f = np.concatenate([trig_poly_eval(nodes(fam, sd, n), complex_normal(200 + sd, Mp))
                            for (Mp, n, fam, sd) in SPECS])
    else:                                   # 256 problems of the batched workload's recipe
        w = make_batch(256, seed=77)
        M, N, x = w.M, w.N, w.x_all
        f = complex_normal(78, int(np.sum(N)))
    b = g.infft_batch_create(M, N, 2.0, 6)
    g.infft_batch_set_nodes(b, torch.tensor(x, dtype=torch.float64, device=dev))
    g.infft_batch_precompute(b)
    ft = torch.tensor(np.asarray(f, np.complex64), device=dev)
    _cache[name] = (b, ft)
    return _cache[name]


@pytest.mark.parametrize("name", ["mixed", "recipe"])
def test_every_tile_shape_gives_identical_fhat(name):
    import torch
    import paper_1811_05335_gb300 as g
    b, f = build(name)
    g.infft_batch_set_tile_shape(b, -1)
    ref = g.infft_batch_apply(b, f)
    torch.cuda.synchronize()
    info = g.infft_batch_get_info(b)
    assert info["unsupported_columns"] == 0
    assert torch.isfinite(torch.view_as_real(ref)).all()
    shapes = g.infft_batch_tile_shapes()
    for sid in range(len(shapes)):
        g.infft_batch_set_tile_shape(b, sid)
        assert g.infft_batch_get_tile_shape(b) == sid
        out = g.infft_batch_apply(b, f)
        torch.cuda.synchronize()
        assert torch.equal(torch.view_as_real(out), torch.view_as_real(ref)), f"shape {sid} {shapes[sid]}"
    host = g.infft_batch_apply(b, f.cpu().numpy())            # host buffers, last shape
    assert np.array_equal(host, ref.cpu().numpy())
    g.infft_batch_set_tile_shape(b, -1)
    assert g.infft_batch_get_tile_shape(b) == 4


def test_tuner_keeps_fastest_shape():
    import torch
    import paper_1811_05335_gb300 as g
    b, f = build("recipe")
    ref = g.infft_batch_apply(b, f).clone()
    best, ms = g.infft_batch_tune_apply(b, repeats=3)
    assert len(ms) == len(g.infft_batch_tile_shapes()) and all(v > 0 for v in ms)
    assert best == int(np.argmin(ms)) and g.infft_batch_get_tile_shape(b) == best
    out = g.infft_batch_apply(b, f)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(out), torch.view_as_real(ref))


def test_autotune_cache_roundtrip(tmp_path):
    import paper_1811_05335_gb300 as g
    from paper_1811_05335_gb300 import tuning
    b, f = build("recipe")
    path = str(tmp_path / "cache.json")
    r = tuning.autotune_batch(b, cache=path, write=path, repeats=2)
    assert r["source"] == "measured" and g.infft_batch_get_tile_shape(b) == r["shape"]
    g.infft_batch_set_tile_shape(b, 0 if r["shape"] else 1)
    r2 = tuning.autotune_batch(b, cache=path)
    assert r2["source"] == "cache" and r2["shape"] == r["shape"] and r2["key"] == r["key"]
    assert g.infft_batch_get_tile_shape(b) == r["shape"]


def test_shape_set_before_precompute_and_invalid_ids():
    import torch
    import paper_1811_05335_gb300 as g
    b, f = build("mixed")
    ref = g.infft_batch_apply(b, f).clone()
    M = [s[0] for s in SPECS]
    N = [s[1] for s in SPECS]
    x = np.concatenate([nodes(fam, sd, n) for (_, n, fam, sd) in SPECS])
    b2 = g.infft_batch_create(M, N, 2.0, 6)
    g.infft_batch_set_tile_shape(b2, 0)                      # before the precompute: stored
    g.infft_batch_set_nodes(b2, torch.tensor(x, dtype=torch.float64, device="cuda:0"))
    g.infft_batch_precompute(b2)
    assert g.infft_batch_get_tile_shape(b2) == 0
    out = g.infft_batch_apply(b2, f)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(out), torch.view_as_real(ref))
    for bad in (-2, len(g.infft_batch_tile_shapes())):
        with pytest.raises(g.InfftError) as ei:
            g.infft_batch_set_tile_shape(b2, bad)
        assert ei.value.code == 1
    assert g.infft_batch_get_tile_shape(b2) == 0
    b2.close()
