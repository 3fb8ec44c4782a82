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
    ap.add_argument("--apply-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-under", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-problems", type=int, default=4096)
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
        return rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def lsq_flops(counts):
    """Algorithmic fp64 flops of the B_opt precompute: per column of n nodes, the
    Cholesky factorisation n^3/3, the two triangular solves 2n^2, and the
    n(n-1)/2 + n closed-form kernel values of Re G_l and Re r_l."""
    n = counts.astype(np.float64)
    return float(np.sum(n ** 3 / 3 + 2 * n ** 2 + (n * (n - 1) / 2 + n) * KAPPA_FLOPS))


KAPPA2_FLOPS = 2 * KAPPA_FLOPS + 17    # a 2-D kernel value: two 1-D Dirichlet ratios and the full kernel's cospi


def lsq_flops_2d(counts):
    """As lsq_flops for the 2-D form's columns (product-kernel entries)."""
    n = counts.astype(np.float64)
    return float(np.sum(n ** 3 / 3 + 2 * n ** 2 + (n * (n - 1) / 2 + n) * KAPPA2_FLOPS))


def apply_bytes(N, M, nnz):
    """Algorithmic HBM bytes of one modified adjoint NFFT: read f (8N), read the
    fp32 weights (4 nnz), write fhat (8M); the grid stays in L2."""
    return 8 * N + 4 * nnz + 8 * M


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
    counts = g.infft_copy_plan_data(plan, weights=False)["col_count"]

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

    # ---- apply only (fixed plan): the paper's "fixed nodes, several problems" regime
    k_app = a.apply_steps
    s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k_app)]
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k_app)]
    for i in range(k_app):
        flush.fill_(float(i))
        s_ev[i].record(stream)
        g.infft_apply(plan, f, fhat, stream)
        e_ev[i].record(stream)
    torch.cuda.synchronize()
    app_ms = sum(s.elapsed_time(e) for s, e in zip(s_ev, e_ev)) / k_app
    g.infft_profile(plan, True)
    for i in range(k_app):
        flush.fill_(float(i))
        g.infft_apply(plan, f, fhat, stream)
    torch.cuda.synchronize()
    g.infft_profile(plan, False)
    app_kernels = g.infft_profile_read(plan)
    # the same apply replayed from a captured CUDA graph (the calls are stream-ordered
    # and allocate nothing, so they capture): the GPU time without the host's launch
    # gaps; L2 still flushed before every replay
    gstream = torch.cuda.Stream(dev)
    gstream.wait_stream(stream)
    with torch.cuda.stream(gstream):
        for _ in range(3):
            g.infft_apply(plan, f, fhat, gstream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gstream):
        g.infft_apply(plan, f, fhat, gstream)
    torch.cuda.synchronize()
    gs_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k_app)]
    ge_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k_app)]
    for _ in range(3):
        graph.replay()
    for i in range(k_app):
        flush.fill_(float(i))
        gs_ev[i].record(stream)
        graph.replay()
        ge_ev[i].record(stream)
    torch.cuda.synchronize()
    app_graph_ms = sum(s.elapsed_time(e) for s, e in zip(gs_ev, ge_ev)) / k_app
    del graph

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
        peak64 = sm_count() * FP64_FLOP_PER_CLK_PER_SM * peaks()[1] * 1e6 / 1e12
        ach = mom_flops / (mom_ms / 1e3) / 1e12
        under = {"workload": f"1D jittered nodes N={Nu} M={Mu} sigma=2 m=4 (underdetermined, M = 4N)",
                 "precompute_ms": t_pre, "apply_ms": t_app, "apply_nodes_per_s": Nu / (t_app / 1e3),
                 "kernels_ms": ukern, "fallback_nodes": infou["fallback_columns"],
                 "roofline_moments": {"kernel": "k_moments (node moments, O(N M) fp64)", "bound": "alu",
                                      "achieved": ach, "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64,
                                      "algorithmic_flops": mom_flops,
                                      "peak_source": "derived: 152 SMs x 4 fp64 flop/clk x max SM clock"}}

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
        t_app_b = timed(lambda: g.infft_batch_apply(bt, fb, out=outb, stream=stream), reps=20)
        infob = g.infft_batch_get_info(bt)
        bt.close()
        nb = int(w.N.sum())
        ab_b = apply_bytes(nb, int(w.M.sum()), infob["nnz"])
        ach_b = ab_b / (t_app_b / 1e3) / 1e9
        single_rate = world * a.N / (app_ms / 1e3)
        batched = {"workload": f"{w.M.size} problems, M log-uniform in [256, 8192] (sum {int(w.M.sum())}), "
                               f"N = 2-4 M (sum {nb}), Chebyshev-clustered nodes, sigma=2, m={w.m}",
                   "precompute_ms": t_pre_b, "apply_ms": t_app_b,
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
        peak64 = sm_count() * FP64_FLOP_PER_CLK_PER_SM * peaks()[1] * 1e6 / 1e12
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
                                         "peak_source": "derived: 152 SMs x 4 fp64 flop/clk x max SM clock"},
                 "roofline_apply": {"kernel": "2-D spread + row and column FFT passes (one apply)", "bound": "hbm",
                                    "achieved": ach2, "peak": peaks()[0], "unit": "GB/s",
                                    "frac": ach2 / peaks()[0], "algorithmic_bytes": ab2,
                                    "index_bytes": idx2}}

    # ---- roofline of the dominant kernel and of the apply
    hbm, sm_max, src = peaks()
    ktab = {name: (n, ms) for name, n, ms in kernels}
    dom = max(ktab, key=lambda k: ktab[k][1])
    dom_n, dom_ms = ktab[dom]
    dom_avg_s = dom_ms / dom_n / 1e3
    roofline = None
    if dom.startswith("lsq"):
        # all columns are solved by the warp tiers at this workload (|I(l)| <= 64)
        fl = lsq_flops(counts)
        lsq_ms = sum(ms for name, (n, ms) in ktab.items() if name.startswith("lsq")) / dom_n
        peak = sm_count() * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
        ach = fl / (lsq_ms / 1e3) / 1e12
        roofline = {"kernel": "lsq (B_opt precompute, all tiers)", "bound": "alu", "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": recorded_traffic("k_lsq_thread<17, 5>"),
                    "peak_source": "derived: 152 SMs x 4 fp64 flop/clk x max SM clock"}
    app_tab = {name: ms for name, n, ms in app_kernels}
    app_kernel_ms = sum(app_tab.values()) / k_app
    ab = apply_bytes(a.N, a.M, info["nnz"])
    ach_app = ab / (app_ms / 1e3) / 1e9
    ach_app_graph = ab / (app_graph_ms / 1e3) / 1e9
    roofline_apply = {"kernel": "spread + fft passes (one apply, event-timed as a whole)", "bound": "hbm",
                      "achieved": ach_app,
                      "peak": hbm, "unit": "GB/s", "frac": ach_app / hbm, "traffic": None,
                      "peak_source": src, "algorithmic_bytes": ab,
                      "graph_replay": {"ms_per_apply": app_graph_ms, "achieved": ach_app_graph,
                                       "frac": ach_app_graph / hbm}}

    ab_many = K_many * (8 * a.N + 8 * a.M) + 4 * info["nnz"]
    ach_many = ab_many / (many_ms / 1e3) / 1e9
    apply_many = {"vectors": K_many, "ms_per_call": many_ms, "value": world * K_many * a.N / (many_ms / 1e3),
                  "unit": "nodes/s",
                  "roofline": {"kernel": "spread + fft passes of 16 data vectors (infft_apply_many)", "bound": "hbm",
                               "achieved": ach_many, "peak": hbm, "unit": "GB/s", "frac": ach_many / hbm,
                               "algorithmic_bytes": ab_many, "peak_source": src}}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a)

    out = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "M": a.M, "N": a.N, "sigma": 2.0, "m": a.m,
                   "step": "pattern + fp64 B_opt precompute + fp32 apply", "l2_flush": "256 MiB write before each step",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
        "roofline_apply": roofline_apply,
        "apply_only": {"value": world * a.N / (app_ms / 1e3), "unit": "nodes/s", "ms_per_apply": app_ms,
                       "kernel_ms_per_apply": app_kernel_ms, "steps": k_app,
                       "graph_replay": {"value": world * a.N / (app_graph_ms / 1e3), "ms_per_apply": app_graph_ms}},
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


def cpu_baseline(a):
    """The oracle as it stands, single-threaded, on one full problem of the workload."""
    p = make_problem(2, M=a.M, N=a.N, m=a.m, with_data=False)
    f = np.random.default_rng(7).standard_normal(a.N) + 0j
    t0 = time.perf_counter()
    oracle_step(p, f)
    dt = time.perf_counter() - t0
    return {"value": a.N / dt, "unit": "nodes/s", "cores": 1, "kind": "oracle",
            "sample": f"one full problem of the workload (M={a.M}, N={a.N}, m={a.m}): pattern, closed-form "
                      f"fp64 B_opt and D^*F^*B^*f, {dt:.1f} s"}


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
