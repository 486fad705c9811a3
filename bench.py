#!/usr/bin/env python3
"""Throughput of the spatial-spectral classification hot path on GB300.

One step = one hsc_classify call (PCA one-band, SVM probabilities, KNN
filter, labels) on a 416 x 512 x 128 float32 neurosurgery-scale frame,
K = 40, 14-row window, lambda = 1, with the library's default (pruned, exact)
KNN search. The steps are a stream of frames: step i runs on context i % F
(--frames-in-flight F, default 8; each context has its own CUDA stream,
scratch and outputs), so while one frame's eigensolver occupies one SM the
other frames' GPU-wide stages run beside it; "value" is pixels/s over the K
steps, "latency_ms" the per-frame latency in that stream, and
"one_in_flight" the same steps on one context, one frame at a time. The full-window KNN (every window candidate, the paper's
procedure; same neighbour sets) is timed on the same maps afterwards and
reported with its FP32-pipe roofline under "knn_full_window". Prints one
JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only). Under torchrun each rank runs an
independent replica on its own GPU (frames are independent: weak scaling).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

CFG = 2
METRIC = "KNN-filtered pixels/s (whole classification path) on 1 GB300"
UNIT = "pixels/s"
N_ROTATING = 4  # distinct cube copies (4 x 109 MB > 129 MB L2)


def workload_config(f, extra=None):
    B, H, W = f.cube.shape
    cfg = {"workload": "neurosurgery-scale frame %dx%dx%d float32, 4 classes, K=%d, %d-row "
                       "window, lambda=%g" % (H, W, B, f.K, f.window_rows, f.lam),
           "H": H, "W": W, "B": B, "classes": f.model.n_classes, "K": f.K,
           "window_rows": f.window_rows, "lambda": f.lam,
           "l2": "%d rotating cube copies (%.0f MB) > 129 MB L2" % (
               N_ROTATING, N_ROTATING * f.cube.nbytes / 1e6),
           "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline --
def knn_pairs(H, W, R):
    """(pixel, window candidate) pairs: each of the W pixels of row r has
    W * (rows of its window) candidates."""
    rows = 0
    for r in range(H):
        lo = max(0, r - R // 2)
        hi = min(H - 1, r + (R + 1) // 2 - 1)
        rows += hi - lo + 1
    return rows * W * W


def jacobi_lane_ops(B, refine_iters, basis=16):
    """FP32 lane-operations (an FMA counts once) of one Jacobi launch: one
    sweep of (n-1) rounds, each rotating P(P-1)/2 off-diagonal 2x2 blocks (16
    ops) and P diagonal blocks with their angles (~12 ops); the rebuild of the
    basis columns (4 ops per logged rotation and column); the Rayleigh-Ritz
    step on them (C X, X^T (C X), two sweeps of the 16 x 16 problem, X W; B
    <= 128); and the double-float refinement, ~12 ops per term of C v."""
    n = B + (B & 1)
    P = n // 2
    m = min(basis, B)
    sweep = (n - 1) * (P * (P - 1) // 2 * 16 + P * 12)
    rebuild = m * (n - 1) * P * 4
    rr = (m * B * B + m * (m + 1) // 2 * B + 2 * 15 * 8 * 16 * 12 + m * m * B) if B <= 128 else 0
    refine = refine_iters * B * B * 12
    return float(sweep + rebuild + rr + refine)


def stage_work(f, knn_pairs_per_launch=None, refine_iters=13):
    """Algorithmic work per launch of each stage (bytes for HBM-bound stages,
    FP32 lane-ops for the KNN and the one-CTA Jacobi) and its bound. The KNN
    counts 4 ops per (pixel, candidate) pair it evaluates: the whole window
    for the full scan, the measured count for the pruned walk."""
    B, H, W = f.cube.shape
    N = H * W
    k = f.model.n_classes
    if knn_pairs_per_launch is None:
        knn_pairs_per_launch = knn_pairs(H, W, f.window_rows)
    return {
        # one read of the cube (the partial Gram outputs are a few MB)
        "moments": ("hbm", 4.0 * B * N),
        # cube read + I (4 B) and P (4k B) written
        "project_svm": ("hbm", 4.0 * B * N + 4.0 * N + 4.0 * k * N),
        # I read + written
        "normalize": ("hbm", 8.0 * N),
        # 4 FP32-pipe ops per (pixel, candidate) pair evaluated
        "knn": ("alu", 4.0 * knn_pairs_per_launch),
        # one CTA on one SM: its bound is that SM's FP32 pipe
        "jacobi": ("alu_sm", jacobi_lane_ops(B, refine_iters)),
    }


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_pipe_peak_tops(sm_count, mhz):
    """FP32 pipe lane-operations per second: 128 FP32 lanes per SM."""
    return sm_count * 128 * mhz * 1e6 / 1e12


def kernel_source_sha(stage):
    from paper_2404_10631_gb300.ncu_summary import source_sha
    return source_sha(stage)


def traffic_from_profiles(stage):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(stage)
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 3 and parts[0] == stage and parts[1] == sha:
            return float(parts[2])
    return None


# ----------------------------------------------------------------- oracle --
def oracle_sample(f, rows, state=None):
    """FP64 oracle on a row sample of the frame; returns (seconds per frame,
    description). Per-pixel stages are timed on the sampled rows and scaled
    by H / len(rows); the per-frame Jacobi is timed whole."""
    import oracle
    B, H, W = f.cube.shape
    if state is None:
        state = {}
    if "C" not in state:  # full-frame inputs of the per-frame / later stages
        mu = oracle.band_means(f.cube)
        state["C"] = oracle.covariance(f.cube, mu)
        pca = oracle.pca_one_band(f.cube)
        P, _, _ = oracle.svm_probs(f.cube, f.model)
        state.update(mu=mu, v1=pca["v1"], I32=pca["I_norm"].astype(np.float32),
                     P32=P.astype(np.float32))
    sub = np.ascontiguousarray(f.cube[:, rows, :])
    t0 = time.perf_counter()
    mu_s = oracle.band_means(sub)
    oracle.covariance(sub, mu_s)
    t1 = time.perf_counter()
    oracle.jacobi(state["C"])
    t2 = time.perf_counter()
    oracle.project(sub, state["mu"], state["v1"])
    oracle.svm_probs(sub, f.model)
    t3 = time.perf_counter()
    for r in rows:
        oracle.knn(state["I32"], state["P32"], f.K, f.window_rows, f.lam, r * W, (r + 1) * W)
    t4 = time.perf_counter()
    scale = H / float(len(rows))
    per_frame = (t1 - t0 + t3 - t2 + t4 - t3) * scale + (t2 - t1)
    desc = ("oracle (single-threaded C, FP64) on %d of %d rows: band means + covariance, "
            "projection, SVM + coupling and KNN timed on the rows and scaled by %.1f; "
            "full-frame Jacobi timed whole" % (len(rows), H, scale))
    return per_frame, desc, state


# ------------------------------------------------ oracle on all host cores --
_ORACLE_STATE = {}


def _oracle_init(state):
    """Worker initializer (spawned process): the frame-wide inputs of the
    per-pixel stages, sent once."""
    _ORACLE_STATE.update(state)


def _oracle_rows(payload):
    """Worker: the oracle's per-pixel stages on one block of rows; seconds."""
    import oracle
    sub, rows = payload
    st = _ORACLE_STATE
    t0 = time.perf_counter()
    mu_s = oracle.band_means(sub)
    oracle.covariance(sub, mu_s)
    oracle.project(sub, st["mu"], st["v1"])
    oracle.svm_probs(sub, st["model"])
    W = st["W"]
    for r in rows:
        oracle.knn(st["I32"], st["P32"], st["K"], st["R"], st["lam"], r * W, (r + 1) * W)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(f, state, rows_per_core=4, rounds=2, warmup=1):
    """The oracle as it stands, on every host core at once: one spawned
    process per core, each running the per-pixel stages (band means +
    covariance, projection, SVM + coupling, KNN) on its own block of rows;
    the per-frame Jacobi is timed whole on one core. Returns (seconds per
    frame, cores, description)."""
    import multiprocessing as mp
    import oracle
    B, H, W = f.cube.shape
    cores = host_cores()
    init = {"mu": state["mu"], "v1": state["v1"], "model": f.model, "I32": state["I32"],
            "P32": state["P32"], "K": f.K, "R": f.window_rows, "lam": f.lam, "W": W}
    rng = np.random.default_rng(1)
    t0 = time.perf_counter()
    oracle.jacobi(state["C"])
    t_jac = time.perf_counter() - t0
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(init,)) as pool:
        walls = []
        for rnd in range(warmup + rounds):  # the first rounds warm the workers up
            blocks = []
            for c in range(cores):
                rows = np.sort(rng.choice(H, rows_per_core, replace=False))
                blocks.append((np.ascontiguousarray(f.cube[:, rows, :]), rows))
            t0 = time.perf_counter()
            pool.map(_oracle_rows, blocks, chunksize=1)
            if rnd >= warmup:
                walls.append(time.perf_counter() - t0)
    wall = float(np.median(walls))
    per_frame = wall * H / float(cores * rows_per_core) + t_jac
    desc = ("oracle (C, FP64) as it stands on %d host cores at once: %d spawned processes, each "
            "running band means + covariance, projection, SVM + coupling and KNN on %d random rows "
            "(median wall time of %d rounds, scaled to %d rows); the full-frame Jacobi timed whole "
            "on one core (%.2f s)" % (cores, cores, rows_per_core, rounds, H, t_jac))
    return per_frame, cores, desc


def run_reference(args, f):
    """The oracle arm: the FP64 oracle as it stands, on every host core (one
    spawned process per core on its own rows; each step one round of that,
    scaled to the frame; the per-frame Jacobi timed whole)."""
    from paper_2404_10631_gb300 import replicas
    _, rank, _ = replicas.env_ranks()
    if not replicas.reports(rank):  # under torchrun rank 0 alone times the oracle
        return
    B, H, W = f.cube.shape
    N = H * W
    rows = np.linspace(0, H - 1, 2).astype(int)
    _, _, state = oracle_sample(f, rows)  # frame-wide inputs (untimed here)
    t_frame, cores, desc = oracle_parallel(f, state, rows_per_core=2, rounds=max(1, args.steps),
                                           warmup=max(1, min(args.warmup, 3)))
    value = N / t_frame
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_frame, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(f),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours --
def run_ours(args, f):
    import torch

    import paper_2404_10631_gb300 as hsc
    from paper_2404_10631_gb300 import replicas
    from paper_2404_10631_gb300 import build as hbuild

    world, rank, local = replicas.env_ranks()
    torch.cuda.set_device(local)
    replicas.init(world, local, "nccl")
    if rank == 0:
        hbuild.build()
    replicas.barrier(world)

    dev = torch.device("cuda", local)
    B, H, W = f.cube.shape
    N = H * W
    k = f.model.n_classes
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = hsc.Context(local, stream=stream)
    ctx.reserve(B, H, W, k)
    cubes = [torch.as_tensor(f.cube, device=dev).clone() for _ in range(N_ROTATING)]
    model = hsc.Model.from_host(f.model, device=dev)
    # launch shapes for this frame shape, picked by the library's autotuner
    t0 = time.perf_counter()
    tune_cfg = ctx.autotune(cubes[0], model)
    tune = {"config": tune_cfg, "seconds": time.perf_counter() - t0,
            "how": "hsc_autotune on the first cube: Gram TMA staging depth {3, 4} x projection/SVM "
                   "{1, 4} pixels per thread x {2, 4, 8, 16} CTAs per SM, median of 3 runs each; "
                   "results do not depend on them"}
    # frames in flight: F contexts, each with its own stream, scratch and
    # outputs; step i runs on context i % F, so one frame's single-SM Jacobi
    # overlaps the other frames' GPU-wide stages
    F = max(1, args.frames_in_flight)
    streams = [stream] + [torch.cuda.Stream(dev) for _ in range(F - 1)]
    ctxs = [ctx] + [hsc.Context(local, stream=s) for s in streams[1:]]
    for c in ctxs[1:]:
        c.reserve(B, H, W, k)
        c.set_tuning(B, H, W, k, (tune_cfg["gram_stages"], tune_cfg["svm_px"],
                                  tune_cfg["svm_blocks_per_sm"]))  # the same launch shapes
    outs = [(torch.empty((H, W), dtype=torch.float32, device=dev),
             torch.empty((k, H, W), dtype=torch.float32, device=dev),
             torch.empty((k, H, W), dtype=torch.float32, device=dev),
             torch.empty((H, W), dtype=torch.int32, device=dev)) for _ in range(F)]
    I, P, O, lab = outs[0]

    def step(i, nf=F):
        j = i % nf
        Ij, Pj, Oj, labj = outs[j]
        hsc.hsc_classify(ctxs[j], cubes[i % N_ROTATING], model, f.K, f.window_rows, f.lam,
                         labels=labj, out_probs=Oj, one_band=Ij, probs=Pj)

    tstream = torch.cuda.Stream(dev)  # brackets the timed region across the F streams

    def timed(nf, clocks=None):
        """K steps with nf frames in flight: (elapsed ms, per-frame latencies)."""
        for i in range(args.warmup):
            step(i, nf)
        for c in ctxs[:nf]:
            c.sync()
        replicas.barrier(world)
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e0.record(tstream)
        for s in streams[:nf]:
            s.wait_event(e0)
        for i in range(args.steps):
            st[i].record(streams[i % nf])
            step(i, nf)
            en[i].record(streams[i % nf])
        for s in streams[:nf]:
            ev_s = torch.cuda.Event()
            ev_s.record(s)
            tstream.wait_event(ev_s)
        e1.record(tstream)
        torch.cuda.synchronize(dev)
        replicas.barrier(world)
        clk = clocks.stop() if clocks else None
        return e0.elapsed_time(e1), [st[i].elapsed_time(en[i]) for i in range(args.steps)], clk

    # ---- device-resident timed region: F frames in flight, then one at a time
    clocks = ClockSampler(local)
    elapsed, per_step, clk = timed(F, clocks)
    elapsed1, per_step1, _ = timed(1) if F > 1 else (elapsed, per_step, None)
    ctx.sync()
    sweeps, refine_iters, sweep_cyc, refine_cyc = ctx.pca_diagnostics(cycles=True)
    # ---- per-stage times: the same steps again on the first context, one
    # frame at a time, with CUDA events around each stage
    for c in ctxs:
        c.sync()
    ctx.knn_candidates_evaluated()  # reset the pruned walk's counter
    ctx.profile(True)
    ctx.profile_read()
    for i in range(args.steps):
        step(i, 1)
    ctx.sync()
    stage_ms, stage_kernels, dropped = ctx.profile_read()
    ctx.profile(False)
    knn_evals = ctx.knn_candidates_evaluated()  # the profiled steps
    knn_evals_per_launch = knn_evals / float(args.steps)

    # ---- the paper's full-window KNN on the same maps (timed on its own)
    ctx.profile(True)
    ctx.profile_read()
    for i in range(args.steps):
        hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, f.lam, out_probs=O, labels=lab,
                           search=hsc.HSC_KNN_SEARCH_FULL)
    full_ms, _, _ = ctx.profile_read()
    # the paper's heap selection (partial heapsort) on the same maps: an A/B point
    n_heap = min(args.steps, 3)
    for i in range(n_heap):
        hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, f.lam, out_probs=O, labels=lab,
                           search=hsc.HSC_KNN_SEARCH_HEAP)
    heap_ms, _, _ = ctx.profile_read()
    ctx.profile(False)
    full_ms_launch = full_ms["knn"] / args.steps
    heap_ms_launch = heap_ms["knn"] / n_heap
    elapsed_max, elapsed1_max = replicas.max_over_ranks([elapsed, elapsed1], world, dev)
    value = replicas.whole_job_rate(N * args.steps, world, elapsed_max / 1e3)
    value1 = replicas.whole_job_rate(N * args.steps, world, elapsed1_max / 1e3)

    # ---- end to end through the public API with host buffers
    host_cube = torch.empty((B, H, W), dtype=torch.float32).pin_memory()
    host_cube.copy_(torch.from_numpy(f.cube))
    host_labs = [torch.empty((H, W), dtype=torch.int32).pin_memory() for _ in range(F)]
    host_model = [torch.from_numpy(a).pin_memory() for a in
                  (f.model.w, f.model.b, f.model.platt_a, f.model.platt_b)]
    # per context: its device cube and its own model copy (the copies of one
    # step and the kernels of another never share a buffer)
    e2e_models = [hsc.Model.from_host(f.model, device=dev) for _ in range(F)]
    e2e_cubes = [torch.empty((B, H, W), dtype=torch.float32, device=dev) for _ in range(F)]
    h2d = host_cube.numel() * 4 + sum(a.numel() * 4 for a in host_model)
    d2h = host_labs[0].numel() * 4
    # the host link's own rate for this copy (pinned cube -> device, CUDA
    # events), the ceiling of the end-to-end number
    for r in range(8):
        if r == 3:
            l0 = torch.cuda.Event(enable_timing=True)
            l0.record(stream)
        e2e_cubes[0].copy_(host_cube, non_blocking=True)
    l1 = torch.cuda.Event(enable_timing=True)
    l1.record(stream)
    l1.synchronize()
    link_gbs = host_cube.numel() * 4 * 5 / (l0.elapsed_time(l1) / 1e3) / 1e9
    n_e2e = max(F, args.steps)
    done = [None] * F
    replicas.barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(n_e2e):
        j = i % F
        if done[j] is not None:
            done[j].synchronize()  # context j's last frame is out: its host labels are read
        with torch.cuda.stream(streams[j]):
            dcube, mj = e2e_cubes[j], e2e_models[j]
            dcube.copy_(host_cube, non_blocking=True)
            for d, h in zip((mj.w, mj.b, mj.platt_a, mj.platt_b), host_model):
                d.copy_(h, non_blocking=True)
            hsc.hsc_classify(ctxs[j], dcube, mj, f.K, f.window_rows, f.lam, labels=outs[j][3])
            host_labs[j].copy_(outs[j][3], non_blocking=True)
            done[j] = torch.cuda.Event()
            done[j].record(streams[j])
    for s in streams:
        s.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = replicas.whole_job_rate(N * n_e2e, world,
                                        replicas.max_over_ranks([e2e_s], world, dev)[0])
    ctx.sync()

    # ---- batched uneven frames vs the plain per-frame path (same GPU)
    batch = None
    if not args.no_batch:
        batch = run_batch(hsc, ctx, stream, dev, args)
    serving = None
    if not args.no_serving and world == 1:
        serving = run_serving(hsc, ctx, stream, dev, args)
    mixed = None
    if not args.no_mixed and world == 1:
        mixed = run_mixed(hsc, ctx, stream, dev, args)

    # ---- roofline of the dominant stage
    peaks, peak_src = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 / FP64 multiply-add issue rates of this GPU, measured here (T lane-ops/s)
    fp32_rate = hsc.hsc_measure_fma_rate(dev.index) / 1e12
    fp64_rate = hsc.hsc_measure_fma_rate(dev.index, fp64=True) / 1e12
    work = stage_work(f, knn_evals_per_launch, refine_iters)
    stages = {}
    for name, ms in stage_ms.items():
        if stage_kernels[name] == 0:  # the min-max normalisation runs inside the pruned KNN
            continue
        launches = max(1, args.steps)
        avg_ms = ms / launches
        bound, units = work[name]
        entry = {"ms_per_launch": avg_ms, "share": ms / max(1e-12, sum(stage_ms.values())),
                 "kernels_per_launch": stage_kernels[name] / launches, "bound": bound}
        if bound == "hbm":
            ach = units / (avg_ms / 1e3) / 1e9
            entry.update(achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                         frac=ach / peaks["hbm_gbs"], algorithmic=units)
        elif bound in ("alu", "alu_sm"):
            sms = sm_count if bound == "alu" else 1
            peak = fp32_rate * sms / sm_count
            ach = units / (avg_ms / 1e3) / 1e12
            entry.update(achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                         algorithmic=units, bound="alu")
            if bound == "alu_sm":
                entry["note"] = "one CTA: peak of the one SM it runs on (FP32 lane-ops)"
        stages[name] = entry
    # the dominant kernel: the stage with the largest time per launch
    dom = max(stages, key=lambda s: stages[s]["ms_per_launch"])
    d = stages[dom]
    one_sm = d.get("note") is not None
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"],
                "peak": d["peak"], "unit": d["unit"], "frac": d["frac"],
                "traffic": traffic_from_profiles(dom),
                "peak_source": ("FP32 FFMA issue rate measured in this run (hsc_measure_fma_rate)%s"
                                % (", per SM" if one_sm else "")
                                if d["bound"] == "alu" else "hbm_gbs, %s" % peak_src),
                "work_per_launch": d["algorithmic"]}
    if one_sm:
        roofline["note"] = d["note"]

    fp32_peak = fp32_rate
    full_ops = 4.0 * knn_pairs(H, W, f.window_rows)
    full_ach = full_ops / (full_ms_launch / 1e3) / 1e12
    knn_full = {"search": "full window (the paper's procedure: every window candidate)",
                "bound": "alu", "ms_per_launch": full_ms_launch, "achieved": full_ach,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": full_ach / fp32_peak,
                "work_per_launch": full_ops,
                "traffic": traffic_from_profiles("knn"),
                "note": "same neighbour sets as the pruned walk used in the step"}
    knn_heap = {"search": "heap selection (the paper's partial heapsort: every window candidate "
                          "keyed, the K smallest kept in a max-heap)", "ms_per_launch": heap_ms_launch,
                "note": "same neighbour sets as the other searches; an A/B point, not the step"}
    pruned_ms = stages["knn"]["ms_per_launch"]
    knn_pruned = {"search": "pruned walk (exact)", "candidates_per_launch": knn_evals_per_launch,
                  "window_pairs_per_launch": knn_pairs(H, W, f.window_rows),
                  "ms_per_launch": pruned_ms,
                  "frac_on_evaluated_pairs": stages["knn"].get("frac"),
                  # the full window's work (4 FP32 ops per window pair) over the pruned
                  # walk's time, against the FP32 pipe: the same neighbour sets in less
                  # time than the full scan could take at the pipe's peak when above 1
                  "window_equivalent_frac": full_ops / (pruned_ms / 1e3) / 1e12 / fp32_peak}

    def pct(v):
        v = sorted(v)
        return {"p50": v[len(v) // 2], "p99": v[min(len(v) - 1, int(0.99 * len(v)))]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(f, {"frames_per_step_per_gpu": 1,
                                          "frames_in_flight": F}),
            "latency_ms": pct(per_step),
            "one_in_flight": {"value": value1, "unit": UNIT,
                              "ms_per_step": elapsed1_max / args.steps,
                              "latency_ms": pct(per_step1),
                              "note": "the same steps on one context, one frame at a time"},
            "roofline": roofline,
            "stages": stages,
            "knn_full_window": knn_full,
            "knn_pruned": knn_pruned,
            "knn_heap": knn_heap,
            "batch": batch,
            "serving": serving,
            "mixed_precision": mixed,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": n_e2e,
                    "h2d_link_gbs": link_gbs,
                    "link_bound": world * link_gbs * 1e9 / h2d * N,
                    "frac_of_link_bound": e2e_value / (world * link_gbs * 1e9 / h2d * N),
                    "note": "each frame's cube crosses the host link once (pinned host -> device); "
                            "h2d_link_gbs is that copy alone, timed in this run (rank 0), and "
                            "link_bound the pixels/s it allows on every rank's own link"},
            "gpu_launches": int(sum(stage_kernels.values())),
            "autotune": tune,
            "fp_peaks": {"fp32_lane_ops_per_s": fp32_rate * 1e12, "fp64_lane_ops_per_s": fp64_rate * 1e12,
                         "fp32_nominal": fp32_pipe_peak_tops(sm_count, peaks.get("sm_max_mhz", 2070.0)) * 1e12,
                         "how": "hsc_measure_fma_rate: 8 independent FFMA / DFMA chains per thread, "
                                "1024 threads per SM, CUDA events"},
            "jacobi": {"fp32_sweeps": sweeps, "refine_iters": refine_iters,
                       "sweep_cycles": sweep_cyc, "refine_cycles": refine_cyc},
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = np.linspace(0, H - 1, 16).astype(int)
        t_frame, desc, state = oracle_sample(f, rows)
        t_par, cores, desc_par = oracle_parallel(f, state)
        line["cpu_baseline"] = {"value": N / t_par, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": desc_par,
                                "single_core": {"value": N / t_frame, "unit": UNIT, "cores": 1,
                                                "sample": desc}}
    if replicas.reports(rank):
        print(json.dumps(line), flush=True)
    for c in ctxs[1:]:
        c.close()
    ctx.close()
    replicas.finalize(world)


def run_mixed(hsc, ctx, stream, dev, args, reps=5):
    """The 1024 x 1024 x 256-band frame (two wide Gaussians per class
    spectrum, sigma 0.01; 1 GiB float32): the covariance on the tensor cores
    as FP16 hi/lo parts with FP32 accumulation, the eigenvector refined in
    double-float, the rest FP32. hsc_classify one frame at a time on one
    context (the cube is 8x L2), with per-stage device times and the HBM
    fraction of the two passes over the cube."""
    import torch
    f = synth.make_config(4)
    B, H, W = f.cube.shape
    N = H * W
    k = f.model.n_classes
    cube = torch.as_tensor(f.cube, device=dev)
    model = hsc.Model.from_host(f.model, device=dev)
    lab = torch.empty((H, W), dtype=torch.int32, device=dev)
    ctx.reserve(B, H, W, k)

    def one():
        hsc.hsc_classify(ctx, cube, model, f.K, f.window_rows, f.lam, labels=lab)

    for _ in range(3):
        one()
    ctx.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for i in range(reps):
        one()
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    ctx.sync()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(reps))
    ms = ev[0].elapsed_time(ev[reps]) / reps
    ctx.profile(True)
    ctx.profile_read()
    for _ in range(reps):
        one()
    ctx.sync()
    st_ms, _, _ = ctx.profile_read()
    ctx.profile(False)
    stages = {n: round(v / reps, 4) for n, v in st_ms.items() if v > 0}
    peaks, _ = load_peaks()
    cube_bytes = 4.0 * B * N

    def hbm_frac(stage, nbytes):
        t = stages.get(stage)
        return None if not t else nbytes / (t / 1e3) / 1e9 / peaks["hbm_gbs"]

    del cube
    torch.cuda.empty_cache()
    return {"workload": "mixed-precision frame 1024x1024x256 float32 (1 GiB), 4 classes, K=40, "
                        "14-row window, lambda=1: FP16 hi/lo tensor-core covariance with FP32 "
                        "accumulation, double-float eigen-refinement, FP32 SVM and KNN",
            "value": N / (ms / 1e3), "unit": UNIT, "ms_per_frame": ms,
            "p50_ms": per[len(per) // 2], "p99_ms": per[-1], "frames": reps,
            "stages_ms": stages,
            "hbm_frac": {"moments": hbm_frac("moments", cube_bytes),
                         "project_svm": hbm_frac("project_svm",
                                                 cube_bytes + 4.0 * N + 4.0 * k * N)},
            "errors": "per-stage errors against the FP64 oracle: tests/test_gpu_mixed.py"}


def run_batch(hsc, ctx, stream, dev, args, n_frames=256, reps=10):
    """256 square snapshot frames (sides 40-64 px, 125 bands, shared model,
    K=16, 7-row window): one hsc_classify_batch call (CUDA-graph replay) per
    step against hsc_classify called frame by frame on the same GPU."""
    import torch
    frames = synth.make_batch(n_frames)
    f0 = frames[0]
    k = f0.model.n_classes
    model = hsc.Model.from_host(f0.model, device=dev)
    cubes = [torch.as_tensor(f.cube, device=dev) for f in frames]
    labs = [torch.empty(f.cube.shape[1:], dtype=torch.int32, device=dev) for f in frames]
    px = sum(f.cube.shape[1] * f.cube.shape[2] for f in frames)

    def batched():
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam,
                               flags=hsc.HSC_BATCH_GRAPH, labels=labs)

    def pooled():
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam,
                               flags=hsc.HSC_BATCH_GRAPH | hsc.HSC_BATCH_POOL, labels=labs)

    def per_frame():
        for c, l in zip(cubes, labs):
            hsc.hsc_classify(ctx, c, model, f0.K, f0.window_rows, f0.lam, labels=l)

    def timed(fn, n):
        for _ in range(3):
            fn()
        ctx.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        ev[0].record(stream)
        for i in range(n):
            fn()
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        ctx.sync()
        per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(n))
        return ev[0].elapsed_time(ev[n]) / n, per

    b_ms, b_per = timed(batched, reps)
    o_ms, _ = timed(pooled, 3)
    p_ms, p_per = timed(per_frame, 3)
    # per-stage device time of the stage-major form (calls without a graph)
    ctx.profile(True)
    ctx.profile_read()
    for _ in range(3):
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam, labels=labs)
    ctx.sync()
    st_ms, st_k, _ = ctx.profile_read()
    ctx.profile(False)
    stages = {n: round(ms / 3, 4) for n, ms in st_ms.items() if ms > 0}
    return {"workload": "%d square snapshot frames, sides 40-64 px, 125 bands float32, "
                        "4 classes (shared model), K=16, 7-row window, lambda=1" % n_frames,
            "pixels_per_batch": px,
            "batched": {"value": px / (b_ms / 1e3), "unit": UNIT, "ms_per_batch": b_ms,
                        "p50_ms": b_per[len(b_per) // 2], "p99_ms": b_per[-1],
                        "api": "hsc_classify_batch, stage-major (one launch per stage over "
                               "every frame), CUDA-graph replay",
                        "stages_ms": stages},
            "stream_pool": {"value": px / (o_ms / 1e3), "unit": UNIT, "ms_per_batch": o_ms,
                            "api": "hsc_classify_batch with HSC_BATCH_POOL (frames on 64 "
                                   "streams), CUDA-graph replay"},
            "plain_per_frame": {"value": px / (p_ms / 1e3), "unit": UNIT, "ms_per_batch": p_ms,
                                "api": "hsc_classify once per frame, one stream"},
            "speedup": p_ms / b_ms}


def run_serving(hsc, ctx, stream, dev, args, rates=(200.0, 400.0, 800.0, 1600.0),
                n_req=400, max_inflight=16):
    """Serving stream: Poisson arrivals of 70% snapshot cubes (40-64 px square,
    125 bands) and 30% pushbroom cubes (384-640 x 320-512 px, 128 bands), each
    with its own SVM model and K in {16, 40}; host cube in, host labels out.
    The native server (continuous batching under an HBM budget) against the
    plain per-frame path (copy in, hsc_classify, copy out, wait; one request
    at a time) on the same arrivals; 'saturation' submits all at time 0."""
    import queue
    import threading

    import torch
    n_snap, n_push = 24, 6
    pool = synth.make_serving_pool(n_snap, n_push)
    cubes = [torch.from_numpy(f.cube).pin_memory() for f in pool]
    models = [hsc.Model.from_host(f.model, device=dev) for f in pool]
    dcubes = [torch.empty(f.cube.shape, dtype=torch.float32, device=dev) for f in pool]
    dlabs = [torch.empty(f.cube.shape[1:], dtype=torch.int32, device=dev) for f in pool]
    outs = {i: [torch.empty(pool[i].cube.shape[1:], dtype=torch.int32).pin_memory()
                for _ in range(4)] for i in range(len(pool))}
    px_of = [f.cube.shape[1] * f.cube.shape[2] for f in pool]

    def server_run(srv, t_arr, idx):
        q = queue.Queue()
        t0 = time.perf_counter()

        def feeder():
            for j in range(len(idx)):
                dt = t_arr[j] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                i = int(idx[j])
                f = pool[i]
                ts = time.perf_counter() - t0
                q.put((j, ts, srv.submit(cubes[i], models[i], f.K, f.window_rows, f.lam,
                                         outs[i][j % 4])))

        th = threading.Thread(target=feeder)
        th.start()
        lat, done = [], []
        for _ in range(len(idx)):
            j, ts, t = q.get()
            ms = srv.wait(t)
            # latency from the arrival time (the feeder can only be late)
            lat.append(ms + 1e3 * (ts - t_arr[j]))
            done.append(ts + ms / 1e3)
        th.join()
        return lat, max(done)

    def per_frame_run(t_arr, idx):
        lat, t0 = [], time.perf_counter()
        for j in range(len(idx)):
            now = time.perf_counter() - t0
            if t_arr[j] > now:
                time.sleep(t_arr[j] - now)
            i = int(idx[j])
            f = pool[i]
            dcubes[i].copy_(cubes[i], non_blocking=True)
            hsc.hsc_classify(ctx, dcubes[i], models[i], f.K, f.window_rows, f.lam,
                             labels=dlabs[i])
            outs[i][j % 4].copy_(dlabs[i], non_blocking=True)
            stream.synchronize()
            lat.append(1e3 * (time.perf_counter() - t0 - t_arr[j]))
        ctx.sync()
        return lat, time.perf_counter() - t0

    def summary(lat, span, idx):
        lat = sorted(lat)
        px = sum(px_of[int(i)] for i in idx)
        return {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1,
                                                               int(0.99 * len(lat)))],
                "max_ms": lat[-1], "value": px / span, "unit": UNIT, "requests": len(lat)}

    # warm-up: every pool frame once through both paths
    warm_t, warm_i = np.zeros(len(pool)), np.arange(len(pool))
    srv = hsc.Server(dev.index or 0, max_inflight=max_inflight)
    server_run(srv, warm_t, warm_i)
    per_frame_run(warm_t, warm_i)
    rows = []
    for r in list(rates) + [None]:
        t_arr, idx = synth.serving_arrivals(n_req, r or 1.0, n_snap, n_push)
        if r is None:
            t_arr = np.zeros(n_req)
        lat_s, span_s = server_run(srv, t_arr, idx)
        lat_p, span_p = per_frame_run(t_arr, idx)
        rows.append({"offered_hz": r if r else "saturation",
                     "server": summary(lat_s, span_s, idx),
                     "plain_per_frame": summary(lat_p, span_p, idx)})
    st = srv.stats()
    srv.close()
    return {"workload": "Poisson arrivals, 70%% snapshot cubes (40-64 px square, 125 bands) / "
                        "30%% pushbroom cubes (384-640 x 320-512 px, 128 bands), float32, "
                        "4 classes, own model per request, K in {16, 40}; %d requests per rate; "
                        "host cube in, host labels out" % n_req,
            "server": "hsc_server (max_inflight %d, HBM budget 80%% of free memory)"
                      % max_inflight,
            "plain_per_frame": "H2D copy + hsc_classify + D2H copy + wait, one request at a time",
            "rates": rows, "server_peak_inflight": st["peak_inflight"],
            "server_peak_bytes": st["peak_bytes"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the 1024x1024x256 mixed-precision frame")
    ap.add_argument("--frames-in-flight", type=int, default=8,
                    help="contexts (streams) the steps rotate over; 1 = one frame at a time")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    f = synth.make_config(CFG)
    if args.impl == "reference":
        run_reference(args, f)
    else:
        run_ours(args, f)


if __name__ == "__main__":
    main()
