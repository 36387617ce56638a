"""Benchmark of the MAPI hot path on GB300 (prints one JSON line).

Workload (one step): MAPI-PCA top-8 principal vectors with deflation on a
zero-mean X of D = 1024 by N = 65536 (spiked covariance 50, 30, 20, 10, 5, 4,
3, 2 then 1, plus 1% Laplace(0, 20) outliers; seeded synthetic data), FP32
storage, min1 product, 100 iterations per vector, matrix-free pair mode:
pack X, then for each component 100 x (pair step over X, reduction, deflation,
l1 normalisation), then the l2 step.  value = MAPI iterations per second over
all ranks (800 per step per rank).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank solves its own seeded instance (weak scaling, no
collective on the data path).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MAPI iterations/s and matrix GB/s (% of HBM / ALU peak); "
          "served p50/p99 latency vs plain")
UNIT = "MAPI iterations/s"
D, N, K_COMP, ITERS = 1024, 65536, 8, 100
WORKLOAD = ("MAPI-PCA top-8 with deflation, pair mode, D=1024 x N=65536 spiked covariance "
            "(50,30,20,10,5,4,3,2 then 1) + 1% Laplace(0,20) outliers, FP32 storage, min1, "
            "100 iterations per vector")


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def source_digest(*names) -> str:
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2110_12065_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(summary: str, digest: str):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    summary is missing or was taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_digest") != digest:
        return None
    try:
        return float(vals["dram_bytes_per_launch"].replace(",", ""))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"mapi_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- GPU arm

def make_inputs(rank: int):
    import datagen
    X = datagen.spiked_pca_data(D, N, seed=rank)
    W0 = np.stack([datagen.start_vector(D, seed=1000 + 17 * rank + c) for c in range(K_COMP)])
    return X, W0


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (the job's time is its slowest rank)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args, rank, world, local_rank, dist):
    import torch

    import paper_2110_12065_gb300 as M
    from paper_2110_12065_gb300 import build as B

    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = M.mapi_create(local_rank)
    stream = torch.cuda.current_stream(dev)

    X, W0 = make_inputs(rank)
    Xd = torch.from_numpy(X).to(dev)
    W0d = torch.from_numpy(W0).to(dev)
    P = torch.empty_like(W0d)

    def step(xsrc, storage="f32", mode="pair", op="min1"):
        mat = M.mapi_matrix_upload(ctx, xsrc, storage)
        try:
            M.mapi_pca_topk(ctx, mat, K_COMP, mode, op, ITERS, float(N), W0d, P_out=P)
        finally:
            M.mapi_matrix_free(ctx, mat)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step(Xd)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    # timed region: the K steps, no per-kernel instrumentation
    sampler = ClockSampler(local_rank)
    sampler.start()
    M.mapi_get_stats(ctx, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(Xd)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = M.mapi_get_stats(ctx, reset=True)["launches"]
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(ms, dist, dev)
    # kernel durations: the same K steps again with CUDA events recorded on
    # the launching stream around every launch of the timed kernel classes
    M.mapi_profile(ctx, True)
    step(Xd)  # capture the instrumented graph outside the measurement
    torch.cuda.synchronize()
    M.mapi_get_stats(ctx, reset=True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step(Xd)
    p1.record(stream)
    torch.cuda.synchronize()
    stats = M.mapi_get_stats(ctx, reset=True)
    M.mapi_profile(ctx, False)
    ms_prof = p0.elapsed_time(p1)
    iters = K_COMP * ITERS * args.steps
    value = iters * world / (t_max / 1e3)
    xbytes = D * N * 4

    peaks = measured_peaks()
    pair = stats["pair"]
    achieved = (pair["bytes"] / pair["launches"]) / (pair["ms"] / pair["launches"] / 1e3) / 1e9
    # no DRAM counters for this kernel: an ncu capture of its cooperative
    # cluster launch failed at launch, so traffic stays null
    traffic = None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": traffic,
                "kernel": "k_pair_solve (persistent: all pair steps of a component)",
                "peak_source": peaks["source"],
                "algorithmic_bytes_per_launch": pair["bytes"] / pair["launches"],
                "avg_launch_us": round(pair["ms"] / pair["launches"] * 1e3, 3),
                "timing": "CUDA events on the launching stream around each persistent "
                          "launch (100 steps), second pass of the K steps",
                "instrumented_ms_per_step": round(ms_prof / args.steps, 3)}
    kernels = {name: {"launches": st["launches"],
                      "avg_us": round(st["ms"] / st["launches"] * 1e3, 3) if st["launches"] else None}
               for name, st in stats.items() if isinstance(st, dict) and st["launches"]}

    # ---- end to end: host (pinned) X -> library upload -> solve -> host P
    Xh = torch.from_numpy(X).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    step(Xh)
    P.cpu()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(Xh)
        _ = P.cpu()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": round(K_COMP * ITERS * e2e_steps * world / e2e_s, 1), "unit": UNIT,
           "h2d_bytes_per_step": xbytes, "d2h_bytes_per_step": K_COMP * D * 4}

    variants = {} if args.no_variants or rank != 0 else run_variants(M, ctx, torch, dev, X, W0d,
                                                                   peaks)
    torch.cuda.synchronize()
    M.mapi_destroy(ctx)

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "D": D, "N": N, "k": K_COMP, "iters_per_vec": ITERS,
                   "mode": "pair", "op": "min1", "storage": "f32", "parallelism":
                   f"replicas x{world}",
                   "l2": "inputs larger than L2 (X = 268 MB FP32 vs 126 MB L2)"},
        "matrix_gbs": round(value / world * xbytes / 1e9 * world, 1),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "kernels": kernels,
        "clocks": clocks,
        "variants": variants,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(X, W0, seconds=args.cpu_seconds)
    return line


def batched_leg(M, ctx, torch, dev, probe, hbm, stg, n_inst=4096, steps=100):
    """The batched workload: Wishart instances A = W W^T / k (n log-uniform in
    [64, 2048], k = n/2), 4 start vectors each, 100 steps, one persistent
    launch; ALU fraction against the probe's rate of the kernel's mix."""
    import datagen
    sizes = datagen.wishart_sizes(n_inst, seed=0)
    mats, items = [], []
    for k, n in enumerate(sizes):
        mats.append(M.mapi_matrix_upload(ctx, datagen.wishart_instance_device(int(n), k), stg))
        w0 = torch.from_numpy(np.stack([datagen.start_vector(int(n), seed=10 * k + v)
                                        for v in range(4)])).to(dev)
        items.append((mats[-1], w0, torch.empty_like(w0)))
    try:
        r = M.mapi_autotune_batched(ctx, items, "min1", 4, iters=2)
        run = lambda: M.mapi_iterate_batched(ctx, items, "min1", 4, steps)
        ms = timed(torch, run, 1)
    finally:
        for m in mats:
            M.mapi_matrix_free(ctx, m)
    elems = float((sizes.astype(np.float64) ** 2).sum())
    terms = elems * 4 * steps
    eb = 4 if stg == "f32" else 2
    # each BF16 element is widened once for the four vectors
    peak_terms = alu_peak_terms(probe["min1_term_f32"] if stg == "f32"
                                else probe["min1_term_bf16_x4"])
    return {"instances": n_inst, "steps": steps,
            "instance_steps_per_s": round(n_inst * steps / (ms / 1e3), 1),
            "ms_per_launch": round(ms, 3), "rows_per_warp": r,
            "terms_per_s": round(terms / (ms / 1e3), 1),
            "alu_frac": round(terms / (ms / 1e3) / peak_terms, 4),
            "matrix_gbs": round(elems * eb * steps / (ms / 1e3) / 1e9, 1),
            "hbm_frac": round(elems * eb * steps / (ms / 1e3) / 1e9 / hbm, 4)}


def pair_phases(M, ctx, Xd, W0d, P, storage="f32"):
    """Where the time of a pair step goes: the headline solve run once with
    the kernel's %globaltimer phase stamps on (microseconds per step,
    averaged over its 800 steps), and each streaming cluster's loop time.  The
    stamps run in a separate instantiation of the kernel and cost about 1 us
    per step themselves."""
    mat = M.mapi_matrix_upload(ctx, Xd, storage)
    try:
        M.mapi_pair_phases(ctx, True)
        M.mapi_pca_topk(ctx, mat, K_COMP, "pair", "min1", ITERS, float(N), W0d, P_out=P)
        M.mapi_pair_phases(ctx, True)  # the first run captured the graph: start again
        M.mapi_pca_topk(ctx, mat, K_COMP, "pair", "min1", ITERS, float(N), W0d, P_out=P)
        ph = M.mapi_pair_phases(ctx, False)
        cl = M.mapi_pair_cluster_times(ctx)
    finally:
        M.mapi_matrix_free(ctx, mat)
    out = {k: round(v, 3) for k, v in ph.items()}
    # how evenly the tile loop is spread: each streaming cluster's loop time
    if cl:
        srt = sorted(cl)
        out["cluster_loop_us"] = {"clusters": len(cl), "min": round(srt[0], 2),
                                  "median": round(srt[len(srt) // 2], 2),
                                  "max": round(srt[-1], 2),
                                  "by_cluster": [round(v, 1) for v in cl]}
    return out


def alu_probe(M, ctx) -> dict:
    """Per-SM, per-clock issue rates of the MAVP term's instruction mixes,
    measured by the library's probe kernel (SM cycles inside the kernel)."""
    return {m: round(M.mapi_alu_probe(ctx, m), 2) for m in M.ALU_MIXES}


def alu_peak_terms(terms_per_clk_sm: float, sm_mhz: float = 2070.0, sms: int = 152) -> float:
    """ALU roofline of the float MAVP term: the measured FP32 min1 terms per
    clock per SM (alu_probe) x SMs x the maximum SM clock."""
    return terms_per_clk_sm * sms * sm_mhz * 1e6


def timed(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_variants(M, ctx, torch, dev, X, W0d, peaks):
    """Short measurements of the other workloads (not the headline)."""
    import datagen
    out = {}
    Xd = torch.from_numpy(X).to(dev)
    P = torch.empty_like(W0d)
    hbm = peaks["hbm_gbs"]

    def instrumented(fn):
        M.mapi_profile(ctx, True)
        fn()  # capture the instrumented graph first
        torch.cuda.synchronize()
        M.mapi_get_stats(ctx, reset=True)
        fn()
        torch.cuda.synchronize()
        st = M.mapi_get_stats(ctx, reset=True)
        M.mapi_profile(ctx, False)
        return st

    def pca(storage, mode):
        mat = M.mapi_matrix_upload(ctx, Xd, storage)
        try:
            run = lambda: M.mapi_pca_topk(ctx, mat, K_COMP, mode, "min1", ITERS, float(N), W0d,
                                          P_out=P)
            ms = timed(torch, run, 2)
            st = instrumented(run)
        finally:
            M.mapi_matrix_free(ctx, mat)
        return ms, st

    probe = alu_probe(M, ctx)
    out["alu_probe_per_clk_per_sm"] = probe
    out["pca_pair_f32_phases_us"] = pair_phases(M, ctx, Xd, W0d, P)
    ms, st = pca("bf16", "pair")
    pr = st["pair"]
    gbs = pr["bytes"] / (pr["ms"] / 1e3) / 1e9
    out["pca_pair_bf16"] = {"iters_per_s": round(K_COMP * ITERS / (ms / 1e3), 1),
                            "ms_per_solve": round(ms, 3), "pair_kernel_gbs": round(gbs, 1),
                            "hbm_frac": round(gbs / hbm, 4)}
    for stg in ("f32", "bf16"):
        ms, st = pca(stg, "mincov")
        mc, gv = st["mincov"], st["gemv"]
        out[f"pca_mincov_{stg}"] = {
            "ms_per_solve": round(ms, 3), "iters_per_s": round(K_COMP * ITERS / (ms / 1e3), 1),
            "build_ms": round(mc["ms"] / max(1, mc["launches"]), 3),
            "build_terms_per_s": round(mc["terms"] / (mc["ms"] / 1e3), 1) if mc["ms"] else None,
            # the build widens BF16 while staging: its inner loop is the FP32 term
            "build_alu_frac": round(mc["terms"] / (mc["ms"] / 1e3) / alu_peak_terms(
                probe["min1_term_f32"]), 4)
            if mc["ms"] else None,
            "iterate_us_per_step": round(gv["ms"] / max(1, gv["launches"]) * 1e3, 3)}

    for stg in ("f32", "bf16"):
        out[f"batched_4096x4_{stg}"] = batched_leg(M, ctx, torch, dev, probe, hbm, stg)

    # plain MAPI / RPI on the n = 512 symmetric Gaussian, 200 steps
    A = datagen.symmetric_gaussian(512, seed=0).astype(np.float32)
    w0 = torch.from_numpy(datagen.start_vector(512, seed=0)).to(dev)
    mat = M.mapi_matrix_upload(ctx, torch.from_numpy(A).to(dev), "f32")
    for op in ("min1", "min2", "dot"):
        ms = timed(torch, lambda: M.mapi_iterate(ctx, mat, op, w0, 200), 5)
        out[f"plain_n512_{op}"] = {"iters_per_s": round(200 / (ms / 1e3), 1),
                                   "us_per_iter": round(ms / 200 * 1e3, 3)}
    M.mapi_matrix_free(ctx, mat)

    # PageRank on a dense Google matrix, n = 16384, 100 steps per storage
    n = 16384
    ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=0)
    dip, dix = torch.from_numpy(ip).to(dev), torch.from_numpy(ix).to(dev)
    w0 = torch.from_numpy(datagen.start_vector(n, seed=0, low=0.0, high=1.0)).to(dev)
    for stg in ("f32", "bf16", "fp8", "i16"):
        G = M.mapi_google_matrix(ctx, dip, dix, n, 0.85, stg)
        try:
            run = lambda: M.mapi_iterate(ctx, G, "min1", w0, 100)
            ms = timed(torch, run, 2)
            st = instrumented(run)
        finally:
            M.mapi_matrix_free(ctx, G)
        gv = st["gemv"]
        gbs = gv["bytes"] / (gv["ms"] / 1e3) / 1e9
        out[f"pagerank_n16384_{stg}"] = {"iters_per_s": round(100 / (ms / 1e3), 1),
                                         "gemv_gbs": round(gbs, 1),
                                         "hbm_frac": round(gbs / hbm, 4)}
    # sparse exact MAPI-PageRank: 2^20 nodes, 8 out-links each, 100 steps
    n = 1 << 20
    ip, ix = datagen.barabasi_albert_digraph_fast(n, m=8, seed=0)
    dip, dix = torch.from_numpy(ip).to(dev), torch.from_numpy(ix).to(dev)
    w0 = torch.from_numpy(datagen.start_vector(n, seed=0, low=0.0, high=1.0)).to(dev)
    run = lambda: M.mapi_pagerank_sparse(ctx, dip, dix, n, w0, 100)
    ms = timed(torch, run, 2)
    st = instrumented(run)
    gv = st["gemv"]
    nnz = int(ip[-1])
    out["pagerank_sparse_n1M"] = {
        "n": n, "links": nnz, "ms_per_solve": round(ms, 3),
        "iters_per_s": round(100 / (ms / 1e3), 1),
        "row_step_us": round(gv["ms"] / max(1, gv["launches"]) * 1e3, 3),
        "row_step_gbs": round(gv["bytes"] / (gv["ms"] / 1e3) / 1e9, 1) if gv["ms"] else None,
        "row_step_hbm_frac": round(gv["bytes"] / (gv["ms"] / 1e3) / 1e9 / hbm, 4)
        if gv["ms"] else None,
        "algorithmic_bytes_per_row_step": 16 * nnz + 8 * n}
    out["rpi_plain_gemv"] = run_rpi_gemv(torch, dev, hbm, Xd)
    out["image_reconstruct_128"] = run_image(M, ctx, torch, dev, hbm)
    out["minibatch_momentum_1e6x10"] = run_minibatch(M, ctx, torch, dev)
    out["serve_config5"] = run_serving_config5(M, torch, dev)
    return out


def run_rpi_gemv(torch, dev, hbm, Xd):
    """The comparison baseline: regular power iteration (Eq. (1)) through a
    plain vendor GEMV (torch.mv, i.e. cuBLAS) on the same matrices, with the
    same number of steps.  Not the product path: it only shows how the MAVP
    kernels compare with a library GEMV that streams the same bytes.
      * PageRank: the dense n = 16384 Google matrix (Eq. (11), formed here
        with torch), b <- G b / ||G b||_2, FP32 and BF16;
      * pair PCA: b <- X (X^T b) / N / ||.||_2 on the D = 1024 x N = 65536 X,
        two GEMVs (two reads of X) per step, FP32 and BF16."""
    import datagen
    res = {}
    n, alpha, T = 16384, 0.85, 100
    ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=0)
    ipd = torch.from_numpy(ip.astype(np.int64)).to(dev)
    ixd = torch.from_numpy(ix.astype(np.int64)).to(dev)
    deg = ipd[1:] - ipd[:-1]
    src = torch.repeat_interleave(torch.arange(n, device=dev), deg)
    G = torch.full((n, n), (1.0 - alpha) / n, dtype=torch.float32, device=dev)
    G.index_put_((ixd, src), (alpha / deg[src].to(torch.float64)).to(torch.float32),
                 accumulate=True)
    dang = torch.nonzero(deg == 0).flatten()
    G[:, dang] += alpha / n
    w0 = torch.from_numpy(datagen.start_vector(n, seed=0, low=0.0, high=1.0)).to(dev)

    def rpi(mv, b, steps):
        for _ in range(steps):
            y = mv(b)
            b = y / torch.linalg.vector_norm(y)
        return b

    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        Gt = G.to(dt)
        b0 = (w0 / torch.linalg.vector_norm(w0)).to(dt)
        ms = timed(torch, lambda: rpi(lambda b: torch.mv(Gt, b), b0, T), 2)
        gms = timed(torch, lambda: [torch.mv(Gt, b0) for _ in range(T)], 2)
        eb = Gt.element_size()
        gbs = n * n * eb / (gms / T / 1e3) / 1e9
        res[f"pagerank_n16384_{name}"] = {
            "iters_per_s": round(T / (ms / 1e3), 1), "us_per_iter": round(ms / T * 1e3, 2),
            "gemv_us": round(gms / T * 1e3, 2), "gemv_gbs": round(gbs, 1),
            "hbm_frac": round(gbs / hbm, 4)}
        del Gt
    del G
    Dd, Nn = Xd.shape
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        Xt = Xd.to(dt)
        b0 = torch.ones(Dd, dtype=dt, device=dev) / float(np.sqrt(Dd))
        step = lambda b: torch.mv(Xt, torch.mv(Xt.t(), b)) / Nn
        ms = timed(torch, lambda: rpi(step, b0, T), 2)
        gbs = 2.0 * Dd * Nn * Xt.element_size() / (ms / T / 1e3) / 1e9
        res[f"pca_pair_d1024_n65536_{name}"] = {
            "iters_per_s": round(T / (ms / 1e3), 1), "us_per_iter": round(ms / T * 1e3, 2),
            "gbs_two_reads_of_X": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
        del Xt
    res["note"] = ("torch.mv (cuBLAS GEMV) RPI with l2 normalisation; pair PCA reads X twice "
                   "per step (X^T b, then X t), the MAVP pair kernel once")
    return res


def psnr(a, b) -> float:
    return float(10.0 * np.log10(1.0 / np.mean((np.asarray(a, np.float64) - b) ** 2)))


def run_image(M, ctx, torch, dev, hbm):
    """Alg. 2 on ten occluded 128 x 128 images (3 of 16 tiles noise): 2
    components x 50 steps on the 16384 x 16384 min-covariance, every image
    reconstructed; PSNR of the reconstructions against the clean image."""
    import datagen
    side, N, k, T = 128, 10, 2, 50
    P = side * side
    clean, imgs = datagen.occluded_images(side, N, grid=4, n_occ=3, seed=0)
    dimg = torch.from_numpy(imgs.reshape(N, P)).to(dev)
    W0 = torch.from_numpy(np.stack([datagen.start_vector(P, seed=50 + c)
                                    for c in range(k)])).to(dev)
    res = {"images": N, "pixels": P, "components": k, "steps": T,
           "psnr_corrupted_mean": round(float(np.mean([psnr(im, clean) for im in imgs])), 2)}
    for op in ("min2", "min1", "dot"):
        run = lambda: M.mapi_image_reconstruct(ctx, dimg, k, op, T, W0)
        ms = timed(torch, run, 2)
        _, R, its = run()
        R = R.cpu().numpy().reshape(N, side, side)
        res[op] = {"ms_per_reconstruction": round(ms, 3), "iters": its,
                   "psnr_mean": round(float(np.mean([psnr(r, clean) for r in R])), 2)}
    # the parts: Eq. (5) build and the steps (instrumented), and one step-6
    # deflation's row pass over the 1 GiB C (read C rows, write the product)
    M.mapi_profile(ctx, True)
    M.mapi_image_reconstruct(ctx, dimg, k, "min2", T, W0)
    torch.cuda.synchronize()
    M.mapi_get_stats(ctx, reset=True)
    M.mapi_image_reconstruct(ctx, dimg, k, "min2", T, W0)
    torch.cuda.synchronize()
    st = M.mapi_get_stats(ctx, reset=True)
    M.mapi_profile(ctx, False)
    mc, gv = st["mincov"], st["gemv"]
    gbs = gv["bytes"] / (gv["ms"] / 1e3) / 1e9 if gv["ms"] else 0.0
    res["build_ms"] = round(mc["ms"] / max(1, mc["launches"]), 3)
    res["step_us"] = round(gv["ms"] / max(1, gv["launches"]) * 1e3, 2)
    res["step_gbs"] = round(gbs, 1)
    res["step_hbm_frac"] = round(gbs / hbm, 4)
    Cbig = torch.rand((P, P), device=dev)
    out = torch.empty_like(Cbig)
    ms = timed(torch, lambda: M.mapi_mavp_project(ctx, "min2", W0, Cbig, out=out), 3)
    res["deflation_row_pass_ms"] = round(ms, 3)
    res["deflation_row_pass_gbs"] = round(2.0 * P * P * 4 / (ms / 1e3) / 1e9, 1)
    del Cbig, out
    return res


def run_minibatch(M, ctx, torch, dev):
    """Alg. 3 on the 10^6 x 10 synthetic set: 100 steps of 1000 draws."""
    import datagen
    Nn, Dd, T, s = 10 ** 6, 10, 100, 1000
    X = datagen.stochastic_pca_data(Nn, Dd, seed=0)
    b = datagen.minibatches(Nn, T, s, seed=1)
    Xd, bd = torch.from_numpy(X).to(dev), torch.from_numpy(b).to(dev)
    w0 = torch.from_numpy(datagen.start_vector(Dd, seed=2)).to(dev)
    res = {"N": Nn, "D": Dd, "steps": T, "batch": s, "beta": 0.2025}
    for op in ("min1", "dot"):
        ms = timed(torch, lambda: M.mapi_minibatch_momentum(ctx, Xd, bd, 0.2025, op, w0,
                                                           M.FLAG_FINAL_L2), 5)
        terms = float(T) * Dd * Dd * s
        res[op] = {"ms_per_solve": round(ms, 3), "steps_per_s": round(T / (ms / 1e3), 1),
                   "terms_per_s": round(terms / (ms / 1e3), 1)}
    return res


def serving_workload(count: int, seed: int = 0):
    """Mixed served requests: 60 % PCA (min-covariance route; D in {256, 512,
    1024}, N log-uniform in [4096, 65536], k uniform in 1..8, 100 steps per
    component), 40 % PageRank (n log-uniform in [256, 8192], Barabasi-Albert
    m = 8, alpha 0.85, 100 steps or delta < 1e-8).  Inputs come from a seeded
    pool of 6 data sets and 6 graphs (drawing a fresh 1024 x 65536 data set
    per request would take the host longer than the GPU needs to serve it)."""
    import datagen
    r = datagen.rng(seed)
    pca_pool, pr_pool = [], []
    for j in range(6):
        D = (256, 512, 1024)[j % 3]
        N = int(np.exp(r.uniform(np.log(4096), np.log(65536))))
        pca_pool.append(datagen.spiked_pca_data(D, N, seed=100 + j))
        n = int(np.exp(r.uniform(np.log(256), np.log(8192))))
        pr_pool.append(datagen.barabasi_albert_digraph(n, m=8, seed=200 + j))
    reqs = []
    for i in range(count):
        if r.random() < 0.6:
            X = pca_pool[int(r.integers(0, 6))]
            k = int(r.integers(1, 9))
            W0 = np.stack([datagen.start_vector(X.shape[0], seed=10 * i + c) for c in range(k)])
            reqs.append(("pca", X, k, W0))
        else:
            ip, ix = pr_pool[int(r.integers(0, 6))]
            n = ip.shape[0] - 1
            reqs.append(("pagerank", ip, ix, datagen.start_vector(n, seed=i, low=0.0, high=1.0)))
    return reqs


def run_serving(M, torch, dev, count: int = 48, seed: int = 0):
    """Served (BF16, one batched launch per round) against plain (FP32, one
    request at a time through mapi_pca_topk / mapi_pagerank).  Latency is
    submit -> result in host memory, input upload included.  Saturation: all
    requests submitted at once.  Poisson run: arrivals at half the served
    saturation rate; the plain latencies at those arrivals come from a
    single FIFO server with the measured plain service times."""
    import datagen
    reqs = serving_workload(count, seed)

    def submit(ctx, q):
        if q[0] == "pca":
            _, X, k, W0 = q
            return M.mapi_submit(ctx, "pca", W0, op="min1", storage="bf16", max_iters=100, X=X,
                                 k=k, cov_denom=X.shape[1])
        _, ip, ix, w0 = q
        return M.mapi_submit(ctx, "pagerank", w0, op="min1", storage="bf16", max_iters=100,
                             tol_l1=1e-8, indptr=ip, indices=ix)

    def served(arrivals):
        ctx = M.mapi_create(0, hbm_budget_bytes=40 << 30)
        try:
            # warm the loop (thread, child context, kernels) on the first request
            t = submit(ctx, reqs[0])
            while M.mapi_poll(ctx, t) is None:
                time.sleep(0.001)
            pending, lat, build, t0 = {}, [], [], time.perf_counter()
            i = 0
            while i < len(reqs) or pending:
                now = time.perf_counter() - t0
                while i < len(reqs) and arrivals[i] <= now:
                    pending[submit(ctx, reqs[i])] = i
                    i += 1
                for t in list(pending):
                    res = M.mapi_poll(ctx, t)
                    if res is not None:
                        assert res["status"] == 0, res
                        lat.append(res["latency_ms"])
                        build.append(res["build_ms"])
                        del pending[t]
                time.sleep(0.0005)
            makespan = time.perf_counter() - t0
        finally:
            M.mapi_destroy(ctx)
        return np.asarray(lat), makespan, np.asarray(build)

    def plain_service():
        ctx = M.mapi_create(0)
        svc = []
        try:
            for q in reqs:
                t0 = time.perf_counter()
                if q[0] == "pca":
                    _, X, k, W0 = q
                    Xm = M.mapi_matrix_upload(ctx, torch.from_numpy(X).to(dev), "f32")
                    P, _ = M.mapi_pca_topk(ctx, Xm, k, "mincov", "min1", 100, X.shape[1],
                                           torch.from_numpy(W0).to(dev))
                    P.cpu()
                    M.mapi_matrix_free(ctx, Xm)
                else:
                    _, ip, ix, w0 = q
                    rk, _, _ = M.mapi_pagerank(ctx, torch.from_numpy(ip).to(dev),
                                               torch.from_numpy(ix).to(dev), ip.shape[0] - 1,
                                               torch.from_numpy(w0).to(dev), 100, tol_l1=1e-8)
                    rk.cpu()
                torch.cuda.synchronize()
                svc.append((time.perf_counter() - t0) * 1e3)
        finally:
            M.mapi_destroy(ctx)
        return np.asarray(svc)

    def fifo(arrivals_s, svc_ms):
        done, lat = 0.0, []
        for a, s in zip(arrivals_s * 1e3, svc_ms):
            done = max(done, a) + s
            lat.append(done - a)
        return np.asarray(lat)

    pct = lambda x, q: round(float(np.percentile(x, q)), 3)
    zero = np.zeros(len(reqs))
    lat_sat, span_sat, _ = served(zero)
    svc = plain_service()
    cap_served = len(reqs) / span_sat
    lam = 0.5 * cap_served
    arr = np.cumsum(datagen.rng(seed + 1).exponential(1.0 / lam, size=len(reqs)))
    lat_p, span_p, build_p = served(arr)
    lat_plain = fifo(arr, svc)
    return {
        "requests": len(reqs), "mix": "60% PCA mincov k<=8 x 100 steps, 40% PageRank 100 steps",
        "served_dtype": "bf16 storage, f32 arithmetic", "plain_dtype": "f32",
        "saturation": {"served_solves_per_s": round(cap_served, 2),
                       "plain_solves_per_s": round(len(reqs) / (svc.sum() / 1e3), 2),
                       "served_p50_ms": pct(lat_sat, 50), "served_p99_ms": pct(lat_sat, 99)},
        "poisson": {"lambda_per_s": round(lam, 2),
                    "served_p50_ms": pct(lat_p, 50), "served_p99_ms": pct(lat_p, 99),
                    "served_solves_per_s": round(len(reqs) / span_p, 2),
                    "served_build_p50_ms": pct(build_p, 50),
                    "plain_p50_ms": pct(lat_plain, 50), "plain_p99_ms": pct(lat_plain, 99)},
        "plain_service_ms": {"p50": pct(svc, 50), "p99": pct(svc, 99)},
    }


class ServePool:
    """The served workload as a stream of requests drawn on demand: 60 % PCA
    (min-covariance route; D in {256, 512, 1024}, N log-uniform in [4096,
    65536], k uniform in 1..8, 100 steps per component), 40 % PageRank (n
    log-uniform in [256, 8192], Barabasi-Albert m = 8, alpha 0.85, 100 steps
    or delta < 1e-8), BF16 storage.  The data sets and graphs come from a
    seeded pool of 6 each (drawing a fresh 1024 x 65536 data set per request
    would take the host longer than the GPU needs to serve it); the kind,
    the pool entry, k and the start vectors are drawn per request."""

    def __init__(self, seed: int = 0):
        import datagen
        r = datagen.rng(seed)
        self.pca, self.pr = [], []
        for j in range(6):
            D = (256, 512, 1024)[j % 3]
            N = int(np.exp(r.uniform(np.log(4096), np.log(65536))))
            self.pca.append(datagen.spiked_pca_data(D, N, seed=100 + j))
            n = int(np.exp(r.uniform(np.log(256), np.log(8192))))
            self.pr.append(datagen.barabasi_albert_digraph(n, m=8, seed=200 + j))
        self.seed = seed

    def request(self, i: int):
        import datagen
        r = datagen.rng(10_000 + 7919 * self.seed + i)
        if r.random() < 0.6:
            X = self.pca[int(r.integers(0, 6))]
            k = int(r.integers(1, 9))
            W0 = r.uniform(-1, 1, size=(k, X.shape[0])).astype(np.float32)
            return ("pca", X, k, W0)
        ip, ix = self.pr[int(r.integers(0, 6))]
        return ("pagerank", ip, ix, r.uniform(0, 1, size=ip.shape[0] - 1).astype(np.float32))


def serve_submit(M, ctx, q):
    if q[0] == "pca":
        _, X, k, W0 = q
        return M.mapi_submit(ctx, "pca", W0, op="min1", storage="bf16", max_iters=100, X=X,
                             k=k, cov_denom=X.shape[1])
    _, ip, ix, w0 = q
    return M.mapi_submit(ctx, "pagerank", w0, op="min1", storage="bf16", max_iters=100,
                         tol_l1=1e-8, indptr=ip, indices=ix)


def serve_window(M, pool, lam: float, window_s: float, drain_s: float, seed: int):
    """Poisson arrivals at rate lam for window_s seconds on a fresh serving
    context (40 GB admission budget); requests still open drain_s after the
    window are cancelled.  Returns latencies of the completed requests (ms),
    completions inside the window, and counts."""
    import datagen
    arr = np.cumsum(datagen.rng(seed).exponential(1.0 / lam, size=int(lam * window_s * 2) + 16))
    arr = arr[arr < window_s]
    ctx = M.mapi_create(0, hbm_budget_bytes=40 << 30)
    try:
        t = serve_submit(M, ctx, pool.request(0))  # warm the loop, its threads and kernels
        while M.mapi_poll(ctx, t) is None:
            time.sleep(0.001)
        pending, lat, done_in_window = {}, [], 0
        i, t0 = 0, time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while i < len(arr) and arr[i] <= now:
                pending[serve_submit(M, ctx, pool.request(1 + i))] = arr[i]
                i += 1
            for tk in list(pending):
                res = M.mapi_poll(ctx, tk)
                if res is not None:
                    if res["status"] == 0:
                        lat.append(res["latency_ms"])
                        if now <= window_s:
                            done_in_window += 1
                    del pending[tk]
            if i >= len(arr) and (not pending or now > window_s + drain_s):
                break
            time.sleep(0.0005)
        for tk in list(pending):
            M.mapi_cancel(ctx, tk)
        open_left = len(pending)
        for tk in list(pending):
            while M.mapi_poll(ctx, tk) is None:
                time.sleep(0.001)
    finally:
        M.mapi_destroy(ctx)
    return np.asarray(lat), done_in_window, len(arr), open_left


def plain_service_ms(M, torch, dev, pool, count: int, seed_base: int = 50_000):
    """Plain one-at-a-time FP32 service times (ms) of `count` requests of the
    same mix: upload, mapi_pca_topk (min-covariance route) or mapi_pagerank,
    result back on the host."""
    ctx = M.mapi_create(0)
    svc = []
    try:
        for i in range(count + 2):
            q = pool.request(seed_base + i)
            t0 = time.perf_counter()
            if q[0] == "pca":
                _, X, k, W0 = q
                Xm = M.mapi_matrix_upload(ctx, torch.from_numpy(X).to(dev), "f32")
                P, _ = M.mapi_pca_topk(ctx, Xm, k, "mincov", "min1", 100, X.shape[1],
                                       torch.from_numpy(W0).to(dev))
                P.cpu()
                M.mapi_matrix_free(ctx, Xm)
            else:
                _, ip, ix, w0 = q
                rk, _, _ = M.mapi_pagerank(ctx, torch.from_numpy(ip).to(dev),
                                           torch.from_numpy(ix).to(dev), ip.shape[0] - 1,
                                           torch.from_numpy(w0).to(dev), 100, tol_l1=1e-8)
                rk.cpu()
            torch.cuda.synchronize()
            if i >= 2:  # the first two warm the kernels and graphs
                svc.append((time.perf_counter() - t0) * 1e3)
    finally:
        M.mapi_destroy(ctx)
    return np.asarray(svc)


def fifo_latency_ms(arrivals_s, svc_ms):
    """Latencies of a single FIFO server with these service times (cycled)."""
    done, lat = 0.0, []
    for i, a in enumerate(np.asarray(arrivals_s) * 1e3):
        done = max(done, a) + svc_ms[i % len(svc_ms)]
        lat.append(done - a)
    return np.asarray(lat)


def run_serving_config5(M, torch, dev, lam: float = 2000.0, window_s: float = 3.0):
    """The served workload at the stated offered load (Poisson, lam = 2000
    requests/s, 40 GB budget) over a bounded window (the stated 60 s would
    queue about 120k requests at a saturated server: the window shows the
    saturated throughput and the latencies there), then a sweep of offered
    loads up to the measured capacity, served BF16 against plain FP32 one at
    a time (a FIFO server with measured service times)."""
    import datagen
    pool = ServePool(0)
    pct = lambda x, q: round(float(np.percentile(x, q)), 3) if len(x) else None
    lat, done, offered, left = serve_window(M, pool, lam, window_s, 2.0, seed=1)
    cap = done / window_s
    svc = plain_service_ms(M, torch, dev, pool, 120)
    plain_cap = 1e3 / float(svc.mean())
    res = {"mix": "60% PCA mincov k<=8 x 100 steps, 40% PageRank 100 steps (BF16 served, "
                  "FP32 plain)", "budget_gb": 40,
           "saturated": {"offered_per_s": lam, "window_s": window_s, "offered": offered,
                         "completed_in_window": done, "served_solves_per_s": round(cap, 2),
                         "cancelled_after_drain": left, "served_p50_ms": pct(lat, 50),
                         "served_p99_ms": pct(lat, 99)},
           "plain_solves_per_s": round(plain_cap, 2),
           "plain_service_ms": {"p50": pct(svc, 50), "p99": pct(svc, 99)}, "sweep": []}
    for f in (0.25, 0.5, 0.75, 0.9):
        lam_f = f * cap
        lat, done, offered, left = serve_window(M, pool, lam_f, 4.0, 6.0, seed=2 + int(f * 100))
        arr = np.cumsum(datagen.rng(2 + int(f * 100)).exponential(1.0 / lam_f, size=offered))
        pl = fifo_latency_ms(arr, svc)
        res["sweep"].append({"fraction_of_capacity": f, "offered_per_s": round(lam_f, 2),
                             "requests": offered, "open_after_drain": left,
                             "served_p50_ms": pct(lat, 50), "served_p99_ms": pct(lat, 99),
                             "plain_p50_ms": pct(pl, 50), "plain_p99_ms": pct(pl, 99)})
    return res


# --------------------------------------------------------------- CPU arm

def cpu_baseline(X, W0, seconds: float = 10.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    pair steps of the second component (one earlier component to deflate) on
    the full X, timed on the host cores."""
    import oracle
    Xf = np.ascontiguousarray(X, dtype=np.float64)
    w = W0[1].astype(np.float64)
    w /= np.linalg.norm(w)
    prev = W0[0].astype(np.float64)
    prev /= np.linalg.norm(prev)

    def one():
        nonlocal w
        y = oracle.pair_step("min1", Xf, w, float(N))
        y = oracle.deflate_vec("min1", y, prev[:, None])
        w = y / np.abs(y).sum()

    t0 = time.perf_counter()
    one()
    first = time.perf_counter() - t0
    reps = max(1, int(seconds / max(first, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(reps):
        one()
    dt = time.perf_counter() - t0
    cores = oracle.max_threads()
    # the same step on one host thread (a shorter sample)
    oracle.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        one()
        first1 = time.perf_counter() - t1
        reps1 = max(1, int(0.25 * seconds / max(first1, 1e-3)))
        t1 = time.perf_counter()
        for _ in range(reps1):
            one()
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(cores)
    return {"value": round(reps / dt, 4), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{reps} pair steps (component 2, one deflation) on the full "
                      f"D=1024 x N=65536 X, FP64, {dt:.1f} s",
            "value_1_thread": round(reps1 / dt1, 4),
            "sample_1_thread": f"{reps1} pair steps on 1 thread, {dt1:.1f} s"}


def oracle_times():
    """The FP64 oracle on bounded samples of each workload, on one host thread
    and on all of them (seconds per unit stated in each entry)."""
    import datagen
    import oracle
    cores = oracle.max_threads()

    def timed_both(fn, reps=1):
        out = {}
        for name, th in (("1_thread", 1), (f"{cores}_threads", cores)):
            oracle.set_num_threads(th)
            fn()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            out[name] = (time.perf_counter() - t0) / reps
        oracle.set_num_threads(cores)
        return out

    res = {"cores": cores}
    A = datagen.symmetric_gaussian(512, seed=0)
    w0 = datagen.start_vector(512, seed=0).astype(np.float64)
    t = timed_both(lambda: oracle.mapi("min1", A, w0, 200), reps=3)
    res["plain_n512_min1_s_per_iter"] = {k: v / 200 for k, v in t.items()}
    X = datagen.spiked_pca_data(1024, 65536, seed=0).astype(np.float64)
    w = datagen.start_vector(1024, seed=1).astype(np.float64)
    w /= np.linalg.norm(w)
    res["pca_pair_s_per_step"] = timed_both(lambda: oracle.pair_step("min1", X, w, 65536.0))
    Xs = np.ascontiguousarray(X[:, :2048])
    t = timed_both(lambda: oracle.mincov("min1", Xs, 2048.0))
    res["pca_mincov_build_s_full_size"] = {k: v * 32 for k, v in t.items()}
    del X, Xs
    n = 16384
    ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=0)
    G = oracle.google_matrix(n, ip, ix, 0.85)
    p0 = datagen.start_vector(n, seed=0, low=0.0, high=1.0).astype(np.float64)
    res["pagerank_n16384_f64_s_per_step"] = timed_both(lambda: oracle.mapi("min1", G, p0, 1))
    G32 = G.astype(np.float32)
    del G
    q = oracle.int_scale(G32, 16)
    Gq = oracle.quant_int(G32, q)
    res["pagerank_n16384_int16_s_per_step"] = timed_both(
        lambda: oracle.mapi_int("min1", Gq, q, p0.astype(np.float32), 1))
    del Gq, G32
    sizes = datagen.wishart_sizes(4096, seed=0)
    sub = [int(x) for x in sizes[:64]]
    mats = [datagen.wishart_instance(nn, k, dtype=np.float64) for k, nn in enumerate(sub)]
    vecs = [datagen.start_vector(nn, seed=k) for k, nn in enumerate(sub)]

    def batch_step():
        for Am, v in zip(mats, vecs):
            for _ in range(4):
                oracle.matvec("min1", Am, v)
    t = timed_both(batch_step)
    frac = float((sizes[:64].astype(np.float64) ** 2).sum() / (sizes.astype(np.float64) ** 2).sum())
    res["batched_4096x4_s_per_step_scaled"] = {k: v / frac for k, v in t.items()}
    res["batched_sample"] = "64 of the 4096 instances, 4 vectors, one product each, scaled by n^2"
    return res


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same metric."""
    if rank != 0:
        return None
    X, W0 = make_inputs(0)
    import oracle
    per_step = 2
    Xf = np.ascontiguousarray(X, dtype=np.float64)
    w = W0[1].astype(np.float64)
    w /= np.linalg.norm(w)
    prev = W0[0].astype(np.float64)
    prev /= np.linalg.norm(prev)

    def step():
        nonlocal w
        for _ in range(per_step):
            y = oracle.pair_step("min1", Xf, w, float(N))
            y = oracle.deflate_vec("min1", y, prev[:, None])
            w = y / np.abs(y).sum()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "D": D, "N": N, "k": K_COMP, "iters_per_vec": ITERS,
                   "mode": "pair", "op": "min1"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"{per_step} pair steps per step (component 2, one "
                                   f"deflation) on the full X, FP64"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def run_case(case: str):
    """One short solve of a named workload, for profilers (prints a line)."""
    import torch

    import datagen
    import paper_2110_12065_gb300 as M
    from paper_2110_12065_gb300 import build as B
    B.build()
    ctx = M.mapi_create(0)
    if case in ("pair-phases", "pair-phases-bf16"):
        X, W0 = make_inputs(0)
        W0d = torch.from_numpy(W0).cuda()
        P = torch.empty_like(W0d)
        ph = pair_phases(M, ctx, torch.from_numpy(X).cuda(), W0d, P,
                         "bf16" if case.endswith("bf16") else "f32")
        out = json.dumps({"case": case, "us_per_step": ph})
    elif case in ("pair-f32", "pair-bf16", "mincov-f32", "mincov-bf16"):
        mode, st = case.split("-")
        X = datagen.spiked_pca_data(D, N, seed=0)
        mat = M.mapi_matrix_upload(ctx, torch.from_numpy(X).cuda(), st)
        W0 = torch.from_numpy(np.stack([datagen.start_vector(D, seed=1 + c)
                                        for c in range(2)])).cuda()
        _, its = M.mapi_pca_topk(ctx, mat, 2, mode, "min1", 6, float(N), W0)
        M.mapi_matrix_free(ctx, mat)
        out = f"{case}: 2 components x 6 steps, iters {its}"
    elif case == "pagerank-sparse":
        n = 1 << 20
        ip, ix = datagen.barabasi_albert_digraph_fast(n, m=8, seed=0)
        w0 = torch.from_numpy(datagen.start_vector(n, seed=0, low=0.0, high=1.0)).cuda()
        _, it, _ = M.mapi_pagerank_sparse(ctx, torch.from_numpy(ip).cuda(),
                                          torch.from_numpy(ix).cuda(), n, w0, 6)
        out = f"{case}: n={n}, {it} steps"
    elif case.startswith("pagerank-"):
        st = case.split("-")[1]
        n = 16384
        ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=0)
        w0 = torch.from_numpy(datagen.start_vector(n, seed=0, low=0.0, high=1.0)).cuda()
        _, it, _ = M.mapi_pagerank(ctx, torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda(),
                                   n, w0, 6, storage=st)
        out = f"{case}: n={n}, {it} steps"
    elif case == "image":
        side, Nn, k = 128, 10, 2
        _, imgs = datagen.occluded_images(side, Nn, grid=4, n_occ=3, seed=0)
        W0 = torch.from_numpy(np.stack([datagen.start_vector(side * side, seed=50 + c)
                                        for c in range(k)])).cuda()
        _, _, its = M.mapi_image_reconstruct(ctx, torch.from_numpy(imgs.reshape(Nn, -1)).cuda(),
                                             k, "min2", 6, W0)
        out = f"{case}: {Nn} images of {side}x{side}, {k} components, iters {its}"
    elif case == "oracle-times":
        out = json.dumps({"case": case, "oracle": oracle_times()})
    elif case == "gemv":
        hbm = measured_peaks()["hbm_gbs"]
        n = 16384
        ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=0)
        dip, dix = torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda()
        w0 = torch.from_numpy(datagen.start_vector(n, seed=0, low=0.0, high=1.0)).cuda()
        res = {}
        for stg in ("f32", "bf16", "fp8", "i16"):
            G = M.mapi_google_matrix(ctx, dip, dix, n, 0.85, stg)
            run = lambda: M.mapi_iterate(ctx, G, "min1", w0, 100)
            M.mapi_profile(ctx, True)
            run()
            torch.cuda.synchronize()
            M.mapi_get_stats(ctx, reset=True)
            run()
            torch.cuda.synchronize()
            gv = M.mapi_get_stats(ctx, reset=True)["gemv"]
            M.mapi_profile(ctx, False)
            M.mapi_matrix_free(ctx, G)
            gbs = gv["bytes"] / (gv["ms"] / 1e3) / 1e9
            res[stg] = {"us_per_step": round(gv["ms"] / gv["launches"] * 1e3, 2),
                        "gemv_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
        out = json.dumps({"case": case, "pagerank_n16384": res})
    elif case == "batched":
        probe = alu_probe(M, ctx)
        hbm = measured_peaks()["hbm_gbs"]
        out = json.dumps({"case": case, **{stg: batched_leg(M, ctx, torch, "cuda", probe, hbm, stg)
                                           for stg in ("f32", "bf16")}})
    elif case == "alu-peak":
        out = json.dumps({"case": case, "per_clk_per_sm": alu_probe(M, ctx)})
    elif case == "minibatch":
        X = datagen.stochastic_pca_data(10 ** 6, 10, seed=0)
        b = datagen.minibatches(10 ** 6, 100, 1000, seed=1)
        w0 = torch.from_numpy(datagen.start_vector(10, seed=2)).cuda()
        M.mapi_minibatch_momentum(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(b).cuda(),
                                  0.2025, "min1", w0)
        out = f"{case}: 10^6 x 10, 100 steps of 1000"
    elif case == "serve":
        out = json.dumps(run_serving_config5(M, torch, "cuda"))
    elif case in ("batched-f32", "batched-bf16"):
        # 512 instances of the batched workload, autotuned as the benchmark
        # is; only the measured launch lies inside the profiler range
        stg = case.split("-")[1]
        sizes = datagen.wishart_sizes(512, seed=0)
        items, mats = [], []
        for k, n in enumerate(sizes):
            mats.append(M.mapi_matrix_upload(ctx, datagen.wishart_instance_device(int(n), k), stg))
            w0 = torch.rand(4, int(n), device="cuda") * 2 - 1
            items.append((mats[-1], w0, torch.empty_like(w0)))
        r = M.mapi_autotune_batched(ctx, items, "min1", 4, iters=2)
        M.mapi_iterate_batched(ctx, items, "min1", 4, 3)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        M.mapi_iterate_batched(ctx, items, "min1", 4, 3)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        for m in mats:
            M.mapi_matrix_free(ctx, m)
        out = f"{case}: 512 instances x 4 vectors, 3 steps, rows per warp {r}"
    else:
        raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize()
    M.mapi_destroy(ctx)
    print(out, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--case", default=None,
                    help="run one short solve of a workload for a profiler and exit: "
                         "pair-f32, pair-bf16, pair-phases, pair-phases-bf16, "
                         "mincov-f32, mincov-bf16, pagerank-f32, "
                         "pagerank-bf16, pagerank-fp8, pagerank-i16, pagerank-sparse, batched-f32, serve, "
                         "image, minibatch, alu-peak")
    args = ap.parse_args()
    if args.case:
        run_case(args.case)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", rank=rank, world_size=world)
        dist = tdist
    line = run_gpu(args, rank, world, local_rank, dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
