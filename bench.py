"""Benchmark of the GB300 direct inverse NFFT (overdetermined case, Sec. 3.2.2).

A step is one pass of the whole path on one synthetic problem shaped like the
paper's reconstruction experiment (Dirichlet kernel, sigma = 2, jittered nodes):
the pattern of I(l) (eq:set_l), the fp64 least-squares precompute of B_opt
(eq:opt_ansatz2 .. eq:solution_ansatz2) and the modified adjoint NFFT
fhat = D^* F^* B_opt^* f (eq:approx_ansatz2).  Workload: M = 2^16, N = 2^18,
m = 4 (override with --M/--N/--m).  Inputs live in HBM before the timed region;
the L2 cache is flushed (a 256 MiB write) before every timed step, outside the
step's CUDA events.

Output: one JSON line (rank 0).  Multi-GPU (torchrun): every rank solves its own
independent problem (replicas; the method does not shard a single problem), the
time is the max over ranks and `value` sums the nodes of all ranks.

--impl reference runs the FP64 CPU oracle instead (the only reference that exists:
the paper ships no code), on rank 0, on a bounded sample of the same workload.
"""
import os

# the CPU oracle legs are timed single-threaded; pin BLAS/OpenMP before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import make_problem, jittered  # noqa: E402

METRIC = "iNFFT nodes/s at M=2^16,N=2^18 (rel.err≤1e-5 vs FP64), % HBM roofline"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--M", type=int, default=2 ** 16)
    ap.add_argument("--N", type=int, default=2 ** 18)
    ap.add_argument("--m", type=int, default=4)
    ap.add_argument("--apply-steps", type=int, default=50)
    ap.add_argument("--rotating-reps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-under", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-problems", type=int, default=4096)
    ap.add_argument("--tune-cache-out", default=None,
                    help="write the batched workload's measured tile shape to this cache file")
    ap.add_argument("--no-2d", action="store_true")
    ap.add_argument("--no-refine", action="store_true")
    return ap.parse_args()


def workload_name(a):
    return f"1D jittered iNFFT M={a.M} N={a.N} sigma=2 m={a.m} (Dirichlet full kernel)"


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value, device, world):
    """The largest of every rank's value (the job's time is its slowest rank's).
    Replicas exchange only this scalar; there is no data-path collective."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, steps, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / seconds


# ---------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_index_for(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


# ---------------------------------------------------------------------------- roofline model


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    except (OSError, ValueError):
        return 6800.0, 2070.0, "fallback"


def sm_count():
    """Multiprocessor count of the current device (queried, not assumed)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


FP64_FLOP_PER_CLK_PER_SM = 4          # 1.25 TFLOP/s nominal at 2070 MHz over 152 SMs
KAPPA_FLOPS = 40                       # fp64 flops of one closed-form kernel value: a sincospi and a sinpi (~17 each), products, a division


def sources_sha1(paths):
    """sha1 over the concatenated contents of the kernel's source files."""
    import hashlib
    h = hashlib.sha1()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kernel`
    from the last ncu capture recorded in profiles/traffic.json, or None when one of
    the kernel's source files changed since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(kernel)
        if not rec or sources_sha1(rec["sources"]) != rec["sha1"]:
            return None
        return rec["value"] if "value" in rec else rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def lsq_flops(counts, kappa_values=None):
    """Algorithmic fp64 flops of the B_opt precompute: per column of n nodes, the
    Cholesky factorisation n^3/3, the two triangular solves 2n^2, and the
    n(n-1)/2 + n closed-form kernel values of Re G_l and Re r_l (or, when given, the
    number of kernel values the solver actually evaluates)."""
    n = counts.astype(np.float64)
    kv = float(np.sum(n * (n - 1) / 2 + n)) if kappa_values is None else float(kappa_values)
    return float(np.sum(n ** 3 / 3 + 2 * n ** 2)) + kv * KAPPA_FLOPS


def kappa_values_executed(starts, counts, N, tile=32, nmax=17):
    """Kernel values the one-thread-per-column solver evaluates: per tile of 32 consecutive
    columns it evaluates each node pair (a, b), a < b, of the tile's union of sorted nodes once
    if some column of the tile holds both (so consecutive columns share them), plus each
    column's n right-hand-side values.  Only when every column is in that tier (n <= 17)."""
    if counts.max() > nmax:
        return None
    total = 0
    for t0 in range(0, len(counts), tile):
        n = counts[t0:t0 + tile]
        live = n > 0
        if not live.any():
            continue
        s0 = starts[t0]
        rs = (starts[t0:t0 + tile] - s0) % N
        rs, n = rs[live], n[live]
        end = rs + n                       # ranges [rs, end), both non-decreasing in the column
        U = int(end.max())
        a = np.arange(U)
        last = np.searchsorted(rs, a, side="right") - 1      # last column starting at or before a
        reach = np.where(last >= 0, np.maximum.accumulate(end)[np.maximum(last, 0)], 0)
        total += int(np.sum(np.maximum(reach - a - 1, 0))) + int(n.sum())
    return total


def recorded_counter(name):
    """A counter value recorded with its capture in profiles/traffic.json (None when the
    kernel's sources changed since)."""
    return recorded_traffic(name)


KAPPA2_FLOPS = 2 * KAPPA_FLOPS + 17    # a 2-D kernel value: two 1-D Dirichlet ratios and the full kernel's cospi


def lsq_flops_2d(counts):
    """As lsq_flops for the 2-D form's columns (product-kernel entries)."""
    n = counts.astype(np.float64)
    return float(np.sum(n ** 3 / 3 + 2 * n ** 2 + (n * (n - 1) / 2 + n) * KAPPA2_FLOPS))


def apply_bytes(N, M, nnz):
    """Algorithmic HBM bytes of one modified adjoint NFFT: read f (8N), read the
    fp32 weights (4 nnz), write fhat (8M); the grid stays in L2."""
    return 8 * N + 4 * nnz + 8 * M


def rotating_applies(g, torch, a, dev, rank, stream, reps=200):
    """The apply timed over R rotating plans: R plans (seeds differ), each precomputed, their
    R applies captured back to back in one CUDA graph on one stream; the graph is replayed
    `reps` times and the per-apply time is the median replay time over R.  R is chosen so that
    R (8N + 4 nnz + 8M) >= 4 x L2.  Also timed: the same R applies issued one by one on the
    stream (no graph)."""
    L2 = torch.cuda.get_device_properties(dev).L2_cache_size
    plans, fs, outs = [], [], []
    first = make_problem(2, M=a.M, N=a.N, m=a.m, with_data=False, seed=1811053352 + 1000 * rank)
    pl = g.infft_plan_create(a.M, a.N, 2.0, a.m)
    g.infft_set_nodes(pl, torch.tensor(first.x, dtype=torch.float64, device=dev), stream)
    g.infft_precompute(pl, stream)
    torch.cuda.synchronize()
    nnz = g.infft_get_info(pl)["nnz"]
    per = apply_bytes(a.N, a.M, nnz)
    R = max(8, -(-4 * L2 // per))
    plans.append(pl)
    for r in range(1, R):
        pr = make_problem(2, M=a.M, N=a.N, m=a.m, with_data=False, seed=1811053352 + 1000 * rank + 7919 * r)
        q = g.infft_plan_create(a.M, a.N, 2.0, a.m)
        g.infft_set_nodes(q, torch.tensor(pr.x, dtype=torch.float64, device=dev), stream)
        g.infft_precompute(q, stream)
        plans.append(q)
    for r in range(R):
        gen = torch.Generator(device=dev).manual_seed(100 + r)
        fs.append(torch.randn(a.N, dtype=torch.complex64, device=dev, generator=gen))
        outs.append(torch.empty(a.M, dtype=torch.complex64, device=dev))
    for _ in range(3):
        for r in range(R):
            g.infft_apply(plans[r], fs[r], outs[r], stream)
    torch.cuda.synchronize()
    total_bytes = sum(apply_bytes(a.N, a.M, g.infft_get_info(q)["nnz"]) for q in plans)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for s0, s1 in ev:
        s0.record(stream)
        for r in range(R):
            g.infft_apply(plans[r], fs[r], outs[r], stream)
        s1.record(stream)
    torch.cuda.synchronize()
    stream_ms = statistics.median(s0.elapsed_time(s1) for s0, s1 in ev) / R
    gs = torch.cuda.Stream(dev)
    gs.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        for r in range(R):
            g.infft_apply(plans[r], fs[r], outs[r], gs)
    torch.cuda.synchronize()
    for _ in range(3):
        graph.replay()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for s0, s1 in ev:
        s0.record(stream)
        graph.replay()
        s1.record(stream)
    torch.cuda.synchronize()
    graph_ms = statistics.median(s0.elapsed_time(s1) for s0, s1 in ev) / R
    del graph
    # the same R applies of independent plans captured on S streams (apply r on stream r mod S,
    # forked from and joined to the capture stream), so that the GPU may overlap one apply's
    # tail with the next apply's start: the protocol's "keep the GPU full" reading
    concurrent = {}
    for S in (2, 4, 8):
        side = [torch.cuda.Stream(dev) for _ in range(S)]
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for q in side:
                q.wait_stream(gs)
            for r in range(R):
                g.infft_apply(plans[r], fs[r], outs[r], side[r % S])
            for q in side:
                gs.wait_stream(q)
        torch.cuda.synchronize()
        for _ in range(3):
            graph.replay()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for s0, s1 in ev:
            s0.record(stream)
            graph.replay()
            s1.record(stream)
        torch.cuda.synchronize()
        concurrent[S] = statistics.median(s0.elapsed_time(s1) for s0, s1 in ev) / R
        del graph
    launches0 = g.infft_launch_count()
    g.infft_apply(plans[0], fs[0], outs[0], stream)
    per_apply_launches = g.infft_launch_count() - launches0
    cfg = g.infft_get_apply_config(plans[0])
    for q in plans:
        q.close()
    torch.cuda.synchronize()
    return {"plans": R, "l2_bytes": L2, "bytes_per_apply": total_bytes / R, "footprint_over_l2": total_bytes / L2,
            "replays": reps, "ms_per_apply_graph": graph_ms, "ms_per_apply_stream": stream_ms,
            "ms_per_apply_graph_streams": {str(k): v for k, v in concurrent.items()},
            "launches_per_apply": per_apply_launches,
            "tile_shape": list(g.infft_apply_configs()[cfg]) if cfg >= 0 else None}


# ---------------------------------------------------------------------------- GPU arm


def run_gpu(a):
    import torch
    import torch.distributed as dist
    import paper_1811_05335_gb300 as g

    rank, local, world = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    p = make_problem(2, M=a.M, N=a.N, m=a.m, with_data=False, seed=1811053352 + 1000 * rank)
    f_host = (np.random.default_rng(7 + rank).standard_normal((a.N, 2)).astype(np.float32)
              .view(np.complex64).ravel())            # timing data: the values do not change the work
    x = torch.tensor(p.x, dtype=torch.float64, device=dev)
    f = torch.tensor(f_host, device=dev)
    fhat = torch.empty(a.M, dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    plan = g.infft_plan_create(a.M, a.N, 2.0, a.m)

    def step():
        g.infft_set_nodes(plan, x, stream)
        g.infft_precompute(plan, stream)
        g.infft_apply(plan, f, fhat, stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    info = g.infft_get_info(plan)
    pdata = g.infft_copy_plan_data(plan, weights=False)
    counts, col_starts = pdata["col_count"].astype(np.int64), pdata["col_start"].astype(np.int64)

    # ---- timed region: K whole-path steps, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index_for(local)) if rank == 0 else None
    launches0 = g.infft_launch_count()
    for i in range(a.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    launches = g.infft_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    if world > 1:
        dist.barrier()
    ms_total = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # the same K steps again with every kernel bracketed by events on its stream: the
    # per-kernel breakdown and the dominant kernel's duration (the instrumentation adds
    # a few microseconds per launch, so the step time above is taken without it)
    g.infft_profile(plan, True)
    for i in range(a.steps):
        flush.fill_(float(i))
        step()
    torch.cuda.synchronize()
    g.infft_profile(plan, False)
    kernels = g.infft_profile_read(plan)
    ms_total = max_over_ranks(ms_total, dev, world)
    ms_step = ms_total / a.steps
    value = job_rate(a.N, a.steps, world, ms_total / 1e3)

    # ---- the modified adjoint NFFT alone (the paper's "fixed nodes, several problems" regime)
    # (1) one apply at a time with the L2 cache flushed before each: single-apply latency
    k_app = a.apply_steps
    s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k_app)]
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k_app)]
    for i in range(k_app):
        flush.fill_(float(i))
        s_ev[i].record(stream)
        g.infft_apply(plan, f, fhat, stream)
        e_ev[i].record(stream)
    torch.cuda.synchronize()
    app_ms = statistics.median(s.elapsed_time(e) for s, e in zip(s_ev, e_ev))
    g.infft_profile(plan, True)
    for i in range(k_app):
        flush.fill_(float(i))
        g.infft_apply(plan, f, fhat, stream)
    torch.cuda.synchronize()
    g.infft_profile(plan, False)
    app_kernels = g.infft_profile_read(plan)
    # (2) the rotating-plan protocol: R plans of the same recipe (distinct nodes, B_opt and data)
    # whose algorithmic bytes exceed 4x the L2 cache, their applies back to back in one
    # captured CUDA graph, replayed; per-apply time = median replay time / R
    rot = rotating_applies(g, torch, a, dev, rank, stream, reps=a.rotating_reps)
    # K data vectors on the same plan in one call (infft_apply_many): the weights are read
    # once for all K; algorithmic bytes K (8N + 8M) + 4 nnz
    K_many = 16
    f_many = torch.randn((K_many, a.N), dtype=torch.complex64, device=dev)
    out_many = torch.empty((K_many, a.M), dtype=torch.complex64, device=dev)
    ws_many = torch.empty(g.infft_apply_many_workspace(plan, K_many), dtype=torch.uint8, device=dev)
    for _ in range(3):
        g.infft_apply_many(plan, f_many, out=out_many, workspace=ws_many, stream=stream)
    ms_ev = [torch.cuda.Event(enable_timing=True) for _ in range(20)]
    me_ev = [torch.cuda.Event(enable_timing=True) for _ in range(20)]
    for i in range(20):
        flush.fill_(float(i))
        ms_ev[i].record(stream)
        g.infft_apply_many(plan, f_many, out=out_many, workspace=ws_many, stream=stream)
        me_ev[i].record(stream)
    torch.cuda.synchronize()
    many_ms = sum(x.elapsed_time(y) for x, y in zip(ms_ev, me_ev)) / 20
    del f_many, out_many, ws_many

    # the own pruned FFT with fused deconvolution (D^* F^* on a grid, through the
    # allocation-free entry point) beside cuFFT's full FFT on the same grid
    grid = torch.randn(plan.M_sigma, dtype=torch.complex64, device=dev)
    out = torch.empty(a.M, dtype=torch.complex64, device=dev)

    def timed(fn, reps=50, warm=5):
        for _ in range(warm):
            fn()
        st = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for i in range(reps):
            flush.fill_(float(i))
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in zip(st, en)) / reps

    own_fft_ms = timed(lambda: g.infft_fft_deconv_noalloc(grid, a.M, out=out, stream=stream))
    cufft_ms = timed(lambda: torch.fft.fft(grid))

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not a.no_e2e:
        xh = torch.tensor(p.x, dtype=torch.float64).pin_memory().numpy()
        fh_ = torch.tensor(f_host).pin_memory().numpy()
        outh = torch.empty(a.M, dtype=torch.complex64).pin_memory().numpy()
        plan_h = g.infft_plan_create(a.M, a.N, 2.0, a.m)

        def step_host():
            g.infft_set_nodes(plan_h, xh, 0)
            g.infft_precompute(plan_h, 0)
            g.infft_apply(plan_h, fh_, outh, 0)    # returns once fhat is in host memory

        for _ in range(a.warmup):
            step_host()
        wall = 0.0
        for i in range(a.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            wall += time.perf_counter() - t0
        wall = max_over_ranks(wall, dev, world)
        e2e = {"value": job_rate(a.N, a.steps, world, wall), "unit": "nodes/s",
               "h2d_bytes_per_step": int(xh.nbytes + fh_.nbytes), "d2h_bytes_per_step": int(outh.nbytes)}
        plan_h.close()

    # ---- differentiable form (workload 5: M = 2^14, N = 2^16 i.i.d. uniform nodes, m = 4):
    # forward (the plain single-problem path) and backward (d/df and d/dx) on the same GPU
    diff = None
    if not a.no_grad:
        p5 = make_problem(5, with_data=False, seed=1811053355 + 1000 * rank)
        x5 = torch.tensor(p5.x, dtype=torch.float64, device=dev)
        f5 = torch.tensor(np.random.default_rng(11).standard_normal((p5.N, 2)).astype(np.float32)
                          .view(np.complex64).ravel(), device=dev)
        w5 = torch.tensor(np.random.default_rng(12).standard_normal((p5.M, 2)).astype(np.float32)
                          .view(np.complex64).ravel(), device=dev)
        plan5 = g.infft_plan_create(p5.M, p5.N, 2.0, 4)
        fh5 = torch.empty(p5.M, dtype=torch.complex64, device=dev)
        gf5 = torch.empty(p5.N, dtype=torch.complex64, device=dev)
        gx5 = torch.empty(p5.N, dtype=torch.float64, device=dev)

        def fwd():
            g.infft_set_nodes(plan5, x5, stream)
            g.infft_precompute(plan5, stream)
            g.infft_apply(plan5, f5, fh5, stream)

        def bwd():
            g.nfft_apply(plan5, w5, gf5, stream)
            g.infft_grad_nodes(plan5, f5, w5, gx5, stream)

        fwd()
        t_f = timed(fwd, reps=10)
        t_b = timed(bwd, reps=10)
        plan5.close()
        diff = {"workload": f"1D i.i.d. uniform nodes M={p5.M} N={p5.N} sigma=2 m=4",
                "forward_ms": t_f, "backward_ms": t_b, "backward_over_forward": t_b / t_f,
                "unit_note": "forward: pattern + fp64 B_opt + apply; backward: nfft_apply + node gradient"}

    # ---- fp64 FMA throughput of this GPU (the precompute's roofline denominator), measured
    sink = torch.empty(g.infft_fp64_fma_probe_sink_len(), dtype=torch.float64, device=dev)
    probe_iters = 4096
    g.infft_fp64_fma_probe(probe_iters, sink, stream)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for s0, s1 in pev:
        s0.record(stream)
        probe_flops = g.infft_fp64_fma_probe(probe_iters, sink, stream)
        s1.record(stream)
    torch.cuda.synchronize()
    fp64_peak = probe_flops / (statistics.median(s0.elapsed_time(s1) for s0, s1 in pev) / 1e3) / 1e12
    del sink

    # ---- underdetermined case (Sec. 3.2.1): jittered nodes, M = 4N (the ratio of the paper's
    # Example ex:trig_poly_ansatz1), N = 2^14, M = 2^16, sigma = 2, m = 4
    under = None
    if not a.no_under:
        Nu, Mu = 2 ** 14, 2 ** 16
        xu = torch.tensor(jittered(1811053360 + 1000 * rank, Nu), dtype=torch.float64, device=dev)
        fu = torch.tensor(np.random.default_rng(13).standard_normal((Nu, 2)).astype(np.float32)
                          .view(np.complex64).ravel(), device=dev)
        planu = g.infft_plan_create_ansatz(Mu, Nu, 2.0, 4, ansatz="under")
        fhu = torch.empty(Mu, dtype=torch.complex64, device=dev)

        def pre_u():
            g.infft_set_nodes(planu, xu, stream)
            g.infft_precompute(planu, stream)

        pre_u()
        t_pre = timed(pre_u, reps=5)
        t_app = timed(lambda: g.infft_apply(planu, fu, fhu, stream), reps=50)
        g.infft_profile(planu, True)
        pre_u()
        torch.cuda.synchronize()
        g.infft_profile(planu, False)
        ukern = {name: ms for name, n, ms in g.infft_profile_read(planu)}
        infou = g.infft_get_info(planu)
        planu.close()
        mom_ms = ukern.get("under_moments", float("nan"))
        # one term of a node moment: complex rotate (4 mul, 2 add) + complex accumulate (2 add)
        mom_flops = 8.0 * Nu * Mu
        peak64 = fp64_peak
        ach = mom_flops / (mom_ms / 1e3) / 1e12
        under = {"workload": f"1D jittered nodes N={Nu} M={Mu} sigma=2 m=4 (underdetermined, M = 4N)",
                 "precompute_ms": t_pre, "apply_ms": t_app, "apply_nodes_per_s": Nu / (t_app / 1e3),
                 "kernels_ms": ukern, "fallback_nodes": infou["fallback_columns"],
                 "roofline_moments": {"kernel": "k_moments (node moments, O(N M) fp64)", "bound": "alu",
                                      "achieved": ach, "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64,
                                      "algorithmic_flops": mom_flops,
                                      "peak_source": "measured in this run: fp64 FMA probe"}}

    # ---- batched form (workload 3: P problems, M log-uniform in [256, 8192], N = 2-4 M,
    # Chebyshev-clustered nodes, m = 6) against the plain single-problem form
    batched = None
    if not a.no_batch:
        from workloads import make_batch
        w = make_batch(a.batch_problems, seed=1811053353 + 1000 * rank)
        xb = torch.tensor(w.x_all, dtype=torch.float64, device=dev)
        fb = torch.tensor(np.random.default_rng(21).standard_normal((int(w.N.sum()), 2)).astype(np.float32)
                          .view(np.complex64).ravel(), device=dev)
        outb = torch.empty(int(w.M.sum()), dtype=torch.complex64, device=dev)
        bt = g.infft_batch_create(w.M, w.N, 2.0, w.m)

        def pre_b():
            g.infft_batch_set_nodes(bt, xb, stream)
            g.infft_batch_precompute(bt, stream)

        t_pre_b = timed(pre_b, reps=2, warm=1)
        # the fixed tile rule, then the autotuned shape (from the package's cache for this
        # workload class and device, else measured now); both give bit-identical fhat
        g.infft_batch_set_tile_shape(bt, -1, stream)
        t_app_fixed = timed(lambda: g.infft_batch_apply(bt, fb, out=outb, stream=stream), reps=20)
        out_fixed = outb.clone()
        from paper_1811_05335_gb300 import tuning
        tune = tuning.autotune_batch(bt, stream=stream, write=a.tune_cache_out)
        t_app_b = timed(lambda: g.infft_batch_apply(bt, fb, out=outb, stream=stream), reps=20)
        torch.cuda.synchronize()
        tuned_identical = bool(torch.equal(torch.view_as_real(outb), torch.view_as_real(out_fixed)))
        infob = g.infft_batch_get_info(bt)
        bt.close()
        nb = int(w.N.sum())
        ab_b = apply_bytes(nb, int(w.M.sum()), infob["nnz"])
        ach_b = ab_b / (t_app_b / 1e3) / 1e9
        single_rate = world * a.N / (rot["ms_per_apply_graph"] / 1e3)
        batched = {"workload": f"{w.M.size} problems, M log-uniform in [256, 8192] (sum {int(w.M.sum())}), "
                               f"N = 2-4 M (sum {nb}), Chebyshev-clustered nodes, sigma=2, m={w.m}",
                   "precompute_ms": t_pre_b, "apply_ms": t_app_b,
                   "tile_shape": {"cols": tune["cols"], "weights": tune["weights"], "source": tune["source"],
                                  "key": tune["key"], "ms_per_shape": tune["ms"]},
                   "apply_ms_fixed_rule": t_app_fixed, "tuned_vs_fixed_speedup": t_app_fixed / t_app_b,
                   "tuned_bit_identical_to_fixed": tuned_identical,
                   "apply_nodes_per_s": nb / (t_app_b / 1e3),
                   "apply_vs_single_problem_apply": (nb / (t_app_b / 1e3)) / single_rate,
                   "precompute_nodes_per_s": nb / (t_pre_b / 1e3),
                   "nnz": infob["nnz"], "large_columns": infob["large_columns"],
                   "max_column": infob["max_column"], "unsupported_columns": infob["unsupported_columns"],
                   "fallback_columns": infob["fallback_columns"],
                   "roofline_apply": {"kernel": "batched spread + chirp-convolution FFT (two launches)",
                                      "bound": "hbm", "achieved": ach_b, "peak": peaks()[0], "unit": "GB/s",
                                      "frac": ach_b / peaks()[0], "algorithmic_bytes": ab_b}}

    # ---- fp64 residual correction on the config-2 nodes: data of a trigonometric polynomial
    # (the direct fp64 sum of random coefficients), the fp64 inverse NFFT and one or two sweeps
    # fhat += D^* F^* B_opt^* (f - A fhat), errors against the true coefficients
    refine = None
    if not a.no_refine:
        gen = torch.Generator(device=dev).manual_seed(31 + rank)
        fh_true = torch.randn(a.M, dtype=torch.complex128, device=dev, generator=gen)
        plan_r = g.infft_plan_create(a.M, a.N, 2.0, a.m)
        g.infft_set_nodes(plan_r, x, stream)
        g.infft_precompute(plan_r, stream)
        f_true = g.infft_ndft_z(plan_r, fh_true, stream=stream)
        est = g.infft_apply_z(plan_r, f_true, stream=stream)

        def rel(v):
            return float(torch.linalg.norm(v - fh_true) / torch.linalg.norm(fh_true))
        errs = [rel(est)]
        for _ in range(2):
            g.infft_refine_z(plan_r, f_true, est, 1, stream)
            errs.append(rel(est))
        scratch = torch.empty_like(f_true)
        t_ndft = timed(lambda: g.infft_ndft_z(plan_r, fh_true, out=scratch, stream=stream), reps=2, warm=1)
        t_kb = timed(lambda: g.infft_nfft_kb_z(plan_r, fh_true, out=scratch, stream=stream), reps=10)
        t_sweep = timed(lambda: g.infft_refine_z(plan_r, f_true, est, 1, stream), reps=2, warm=1)
        t_apply_z = timed(lambda: g.infft_apply_z(plan_r, f_true, stream=stream), reps=10)
        plan_r.close()
        refine = {"workload": workload_name(a) + ", data f = A fhat of complex normal fhat (fp64 direct sum)",
                  "rel_err_vs_true": {"fp64_infft": errs[0], "after_1_sweep": errs[1], "after_2_sweeps": errs[2]},
                  "data": "f = A fhat by the direct fp64 sum (infft_ndft_z)",
                  "apply_z_ms": t_apply_z, "nfft_kb_z_ms": t_kb, "ndft_z_ms": t_ndft, "sweep_ms": t_sweep,
                  "note": "the sweep's A fhat by the windowed fp64 NFFT (Kaiser-Bessel, Sec. 2.1); the direct fp64 "
                          "sum (O(N M)) timed beside it"}

    # ---- 2-D tensor-product form (workload 4: radial trajectory of 512 spokes x 512
    # samples, M = 256 x 256, sigma = 2 per dimension, m = 4)
    two_d = None
    if not a.no_2d:
        from workloads import make_2d
        w2 = make_2d(seed=1811053354 + 1000 * rank)
        x2 = torch.tensor(w2.x, dtype=torch.float64, device=dev)
        f2 = torch.tensor(np.random.default_rng(22).standard_normal((w2.N, 2)).astype(np.float32)
                          .view(np.complex64).ravel(), device=dev)
        out2 = torch.empty(w2.M1 * w2.M2, dtype=torch.complex64, device=dev)
        q2 = g.infft2d_plan_create(w2.M1, w2.M2, w2.N, 2.0, w2.m)
        t_pat2 = timed(lambda: g.infft2d_set_nodes(q2, x2, stream), reps=2, warm=1)
        t_pre2 = timed(lambda: g.infft2d_precompute(q2, stream), reps=2, warm=1)
        t_app2 = timed(lambda: g.infft2d_apply(q2, f2, out=out2, stream=stream), reps=50)
        info2 = g.infft2d_get_info(q2)
        cols2 = np.diff(g.infft2d_copy_plan_data(q2, weights=False)["col_offset"].astype(np.int64))
        q2.close()
        fl2 = lsq_flops_2d(cols2)
        peak64 = fp64_peak
        ach_pre2 = fl2 / (t_pre2 / 1e3) / 1e12
        M2d = w2.M1 * w2.M2
        ab2 = 8 * w2.N + 4 * info2["nnz"] + 8 * M2d          # f, weights, fhat
        idx2 = 4 * info2["nnz"] + 4 * (4 * M2d + 1)          # node index per entry, column offsets
        ach2 = ab2 / (t_app2 / 1e3) / 1e9
        two_d = {"workload": f"2-D radial trajectory {w2.N} nodes (512 spokes x 512 samples, 1e-4 jitter), "
                             f"M = {w2.M1} x {w2.M2}, sigma = 2 per dimension, m = {w2.m}",
                 "pattern_ms": t_pat2, "precompute_ms": t_pre2, "apply_ms": t_app2,
                 "apply_nodes_per_s": w2.N / (t_app2 / 1e3),
                 "nnz": info2["nnz"], "max_column": info2["max_column"], "empty_columns": info2["empty_columns"],
                 "large_columns": info2["large_columns"], "wide_columns": info2["wide_columns"],
                 "fallback_columns": info2["fallback_columns"], "unsupported_columns": info2["unsupported_columns"],
                 "objective": info2["objective"],
                 "roofline_precompute": {"kernel": "2-D B_opt precompute, all tiers (fp64 Cholesky of every column)",
                                         "bound": "alu", "achieved": ach_pre2, "peak": peak64, "unit": "TFLOP/s",
                                         "frac": ach_pre2 / peak64, "algorithmic_flops": fl2,
                                         "peak_source": "measured in this run: fp64 FMA probe"},
                 "roofline_apply": {"kernel": "2-D spread + row and column FFT passes (one apply)", "bound": "hbm",
                                    "achieved": ach2, "peak": peaks()[0], "unit": "GB/s",
                                    "frac": ach2 / peaks()[0], "algorithmic_bytes": ab2,
                                    "index_bytes": idx2}}

    # ---- rooflines: the modified adjoint NFFT (HBM) and the B_opt precompute (fp64 ALU)
    hbm, sm_max, src = peaks()
    ktab = {name: (n, ms) for name, n, ms in kernels}
    ab = apply_bytes(a.N, a.M, info["nnz"])
    graph_ms = rot["ms_per_apply_graph"]
    ach_app = rot["bytes_per_apply"] / (graph_ms / 1e3) / 1e9
    ach_single = ab / (app_ms / 1e3) / 1e9
    traffic = recorded_traffic("apply")
    roofline = {"kernel": f"modified adjoint NFFT D^*F^*B^*f: k_apply_spread_fftA + k_fftB_r8 "
                          f"({rot['launches_per_apply']} launches per apply), {rot['plans']} applies over rotating "
                          f"plans in one CUDA graph, median of {rot['replays']} replays",
                "bound": "hbm", "achieved": ach_app, "peak": hbm, "unit": "GB/s", "frac": ach_app / hbm,
                "traffic": traffic, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_apply": rot["bytes_per_apply"],
                "algorithmic_bytes": "8N (f) + 4 nnz (fp32 weights) + 8M (fhat); the grid and the FFT "
                                     "intermediate stay in L2",
                "ms_per_apply": graph_ms, "footprint_over_l2": rot["footprint_over_l2"],
                "tile_shape": rot["tile_shape"]}
    lsq_names = [k for k in ktab if k.startswith("lsq")]
    lsq_n = ktab[lsq_names[0]][0] if lsq_names else 1
    lsq_ms = sum(ktab[k][1] for k in lsq_names) / lsq_n
    fl = lsq_flops(counts)
    ach64 = fl / (lsq_ms / 1e3) / 1e12
    executed = kappa_values_executed(col_starts, counts, a.N)
    fl_exec = None if executed is None else lsq_flops(counts, kappa_values=executed)
    roofline_precompute = {
        "kernel": "lsq (B_opt precompute, all solver tiers)", "bound": "alu", "achieved": ach64,
        "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach64 / fp64_peak,
        "peak_source": f"measured in this run: fp64 FMA probe (8 independent FMA chains per thread, 8 CTAs of "
                       f"256 threads per SM), {fp64_peak:.3f} TFLOP/s; nominal 152 SMs x 4 flop/clk x max clock = "
                       f"{sm_count() * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e12:.3f} TFLOP/s",
        "traffic": recorded_traffic("k_lsq_thread<17, 5>"),
        "flop_convention": f"per column of n nodes: n^3/3 + 2n^2 + (n(n-1)/2 + n) x {KAPPA_FLOPS} "
                           f"(one closed-form kernel value = {KAPPA_FLOPS} flop)",
        "kappa_values_per_column_definition": float(np.sum(counts * (counts - 1) / 2 + counts)),
        "kappa_values_executed": executed,
        "achieved_as_executed": None if fl_exec is None else fl_exec / (lsq_ms / 1e3) / 1e12,
        "fp64_pipe_active": recorded_counter("lsq_fp64_pipe_active"),
        "ms": lsq_ms}
    app_tab = {name: ms for name, n, ms in app_kernels}
    app_kernel_ms = sum(app_tab.values()) / k_app

    ab_many = K_many * (8 * a.N + 8 * a.M) + 4 * info["nnz"]
    ach_many = ab_many / (many_ms / 1e3) / 1e9
    apply_many = {"vectors": K_many, "ms_per_call": many_ms, "value": world * K_many * a.N / (many_ms / 1e3),
                  "unit": "nodes/s",
                  "roofline": {"kernel": "the apply's two kernels over 16 data vectors (infft_apply_many)",
                               "bound": "hbm", "achieved": ach_many, "peak": hbm, "unit": "GB/s",
                               "frac": ach_many / hbm, "algorithmic_bytes": ab_many, "peak_source": src}}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu, accuracy = cpu_baseline(a, g, torch, dev, stream)
    else:
        accuracy = None

    out = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 precompute, f32 apply", "data": "synthetic",
        "config": {"workload": workload_name(a), "M": a.M, "N": a.N, "sigma": 2.0, "m": a.m,
                   "step": "pattern + fp64 B_opt precompute + fp32 apply", "l2_flush": "256 MiB write before each step",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
        "roofline_precompute": roofline_precompute,
        "accuracy": accuracy,
        "apply_only": {"value": world * a.N / (graph_ms / 1e3), "unit": "nodes/s", "ms_per_apply": graph_ms,
                       "protocol": "rotating plans, CUDA graph (the roofline's figure)",
                       "graph_independent_streams": {
                           "ms_per_apply": rot["ms_per_apply_graph_streams"],
                           "frac": {k: rot["bytes_per_apply"] / (v / 1e3) / 1e9 / hbm
                                    for k, v in rot["ms_per_apply_graph_streams"].items()},
                           "note": "the R independent plans' applies in one graph on S capture streams "
                                   "(apply r on stream r mod S), so consecutive applies may overlap"},
                       "stream_back_to_back": {"ms_per_apply": rot["ms_per_apply_stream"],
                                               "value": world * a.N / (rot["ms_per_apply_stream"] / 1e3)},
                       "single_apply_l2_flushed": {"ms": app_ms, "achieved_gbs": ach_single,
                                                   "frac": ach_single / hbm, "kernel_ms": app_kernel_ms,
                                                   "repeats": k_app}},
        "apply_many": apply_many,
        "fft_vs_cufft": {"own_fft_deconv_ms": own_fft_ms, "cufft_ms": cufft_ms, "length": plan.M_sigma,
                         "note": "own: pruned length-M_sigma FFT with D fused (M outputs); cuFFT: full FFT"},
        "differentiable": diff,
        "underdetermined": under,
        "batched": batched,
        "two_d": two_d,
        "refine": refine,
        "kernels": {name: {"launches": n, "ms_total": ms} for name, n, ms in kernels},
        "plan": {"nnz": info["nnz"], "max_column": info["max_column"], "fallback_columns": info["fallback_columns"]},
        "cpu_baseline": cpu,
    }
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------- CPU oracle legs


def oracle_step(p, f):
    import oracle
    B = oracle.bopt.bopt_closed(p.x, p.M, 2.0, p.m)
    return oracle.infft.infft_apply(B, f)


def cpu_baseline(a, g, torch, dev, stream):
    """CPU legs on the workload of the headline (rank 0, one GPU), outside every timed GPU region:

    * the oracle as it stands (numpy, one thread): pattern, closed-form fp64 B_opt and
      D^*F^*B^*f on one full problem with data f = A fhat + 1e-8 noise;
    * the oracle's C apply (gather, radix-2 FFT, D; OpenMP on every host core), fp64 and fp32,
      with the oracle's B_opt;
    * the accuracy of the measured configuration: the GPU's fhat on the same data against the
      oracle's (on the same complex64 input) and against the true coefficients."""
    import oracle
    from oracle import capply
    p = make_problem(2, M=a.M, N=a.N, m=a.m)
    t0 = time.perf_counter()
    B = oracle.bopt.bopt_closed(p.x, p.M, 2.0, p.m)
    fhat_o = oracle.infft.infft_apply(B, p.f)
    dt = time.perf_counter() - t0
    cpu = {"value": a.N / dt, "unit": "nodes/s", "cores": 1, "kind": "oracle",
           "sample": f"one full problem of the workload (M={a.M}, N={a.N}, m={a.m}): pattern, closed-form fp64 "
                     f"B_opt and D^*F^*B^*f, {dt:.1f} s"}
    # the oracle's C apply on all host cores
    cores = os.cpu_count() or 1
    capply.set_threads(cores)
    c_apply = {}
    for prec, dt_ in (("f64", np.complex128), ("f32", np.complex64)):
        ca = capply.CApply(B, prec)
        fin = p.f.astype(dt_)
        ca(fin)
        ts = []
        for _ in range(5):
            t1 = time.perf_counter()
            ca(fin)
            ts.append(time.perf_counter() - t1)
        c_apply[prec] = {"ms_per_apply": 1e3 * statistics.median(ts), "nodes_per_s": a.N / statistics.median(ts)}
    cpu["c_apply"] = dict(c_apply, cores=capply.threads(), nproc=cores,
                          kind="oracle/capply.c: gather + radix-2 FFT + D, OpenMP, the oracle's B_opt")
    # accuracy of the measured configuration
    f32 = np.asarray(p.f, np.complex64)
    plan = g.infft_plan_create(a.M, a.N, 2.0, a.m)
    g.infft_set_nodes(plan, torch.tensor(p.x, dtype=torch.float64, device=dev), stream)
    g.infft_precompute(plan, stream)
    got = g.infft_apply(plan, torch.tensor(f32, device=dev), stream=stream).cpu().numpy().astype(np.complex128)
    plan.close()
    want = oracle.infft.infft_apply(B, f32.astype(np.complex128))
    accuracy = {"data": "f = A fhat + complex noise of 1e-8 relative level (fp64 trigonometric sum)",
                "rel_l2_vs_oracle": oracle.infft.rel_l2(got, want), "tolerance": 1e-5,
                "rel_l2_vs_true_coefficients": oracle.infft.rel_l2(got, p.fhat),
                "oracle_rel_l2_vs_true_coefficients": oracle.infft.rel_l2(fhat_o, p.fhat)}
    return cpu, accuracy


def run_reference(a):
    rank, _, world = dist_info()
    if rank != 0:
        return
    # bounded sample: the same recipe at 1/16 of the nodes and coefficients per step
    M, N = max(a.M // 16, 64), max(a.N // 16, 256)
    p = make_problem(2, M=M, N=N, m=a.m, with_data=False)
    f = np.random.default_rng(7).standard_normal(N) + 0j
    for _ in range(a.warmup):
        oracle_step(p, f)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle_step(p, f)
    dt = time.perf_counter() - t0
    v = N * a.steps / dt
    sample = f"per step the workload's recipe at M={M}, N={N}, m={a.m} (1/16 of the nodes)"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "nodes/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(a), "M": a.M, "N": a.N, "sigma": 2.0, "m": a.m},
           "cpu_baseline": {"value": v, "unit": "nodes/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)
