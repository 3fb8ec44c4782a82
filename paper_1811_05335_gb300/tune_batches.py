"""Measures the batched spreading's tile shape for several classes of batched workloads and
writes them to a tile-shape cache (the file that paper_1811_05335_gb300.tuning reads).

    python -m paper_1811_05335_gb300.tune_batches --out paper_1811_05335_gb300/tune_cache.json

Run from the repository root on the GPU the cache is for (the entries are keyed by its name).
The classes: the batched recipe (M log-uniform in [256, 8192], N = 2-4 M, sigma = 2) with
Chebyshev-clustered nodes at m = 4, 6, 8 and with P = 512, and with i.i.d. uniform and jittered
nodes at m = 6.  Inputs are the seeded synthetic generators of workloads/.
"""
import argparse
import sys

CLASSES = [  # (P, m, node family)
    (4096, 6, "chebyshev"), (4096, 4, "chebyshev"), (4096, 8, "chebyshev"), (512, 6, "chebyshev"),
    (4096, 6, "uniform"), (4096, 6, "jittered"),
]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--repeats", type=int, default=10)
    ap.add_argument("--classes", default="all", help="comma-separated indices into CLASSES, or 'all'")
    a = ap.parse_args(argv)
    import torch
    import paper_1811_05335_gb300 as g
    from paper_1811_05335_gb300 import tuning
    from workloads import make_batch
    pick = range(len(CLASSES)) if a.classes == "all" else [int(v) for v in a.classes.split(",")]
    dev = torch.device("cuda:0")
    for i in pick:
        P, m, fam = CLASSES[i]
        w = make_batch(P, seed=1811053353 + i, m=m, nodes=fam)
        b = g.infft_batch_create(w.M, w.N, 2.0, m)
        g.infft_batch_set_nodes(b, torch.tensor(w.x_all, dtype=torch.float64, device=dev))
        g.infft_batch_precompute(b)
        r = tuning.autotune_batch(b, cache=None, write=a.out, repeats=a.repeats)
        print(f"{r['key']}: shape {r['shape']} ({r['cols']} points, {r['weights']} weights), "
              f"ms {[round(v, 3) for v in r['ms']]}", flush=True)
        b.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
