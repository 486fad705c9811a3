#!/usr/bin/env python3
"""Throughput of the spatial-spectral classification hot path on GB300.

One step = one hsc_classify call (PCA one-band, SVM probabilities, KNN
filter, labels) on a 1024 x 1024 x 256-band float32 frame (1 GiB; class
spectra of two wide Gaussians, sigma 0.01), K = 40, 14-row window,
lambda = 1, with the library's defaults: the covariance on the tensor cores
(FP16 hi/lo parts, FP32 accumulation), the exact pruned KNN search. The
steps are a stream of frames: step i runs on context i % F
(--frames-in-flight F, default 8; each context has its own CUDA stream,
scratch and outputs), so while one frame's eigensolver occupies one SM (or,
for 129-256 bands, its first sweep a cluster of 16) the other frames'
GPU-wide stages run beside it. "value" is pixels/s over the K
steps, "latency_ms" the per-frame latency in that stream, "one_in_flight"
the same steps on one context, and "plain_fp32" the plain per-frame FP32
path on the same GPU: the covariance on the FP32 pipe (HSC_COV_FP32_PIPE),
one frame at a time. The same measurements on the 416 x 512 x 128
neurosurgery-scale frame are under "neuro"; the batched and served forms
under "batch" and "serving". Prints one JSON line.

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

HEADLINE_CFG = 4
NEURO_CFG = 2
METRIC = "KNN-filtered pixels/s (whole classification path) on 1 GB300"
UNIT = "pixels/s"
L2_BYTES = 129e6


def workload_name(f):
    B, H, W = f.cube.shape
    kind = {256: "mixed-precision-scale frame", 128: "neurosurgery-scale frame"}.get(B, "frame")
    return ("%s %dx%dx%d float32, %d classes, K=%d, %d-row window, lambda=%g"
            % (kind, H, W, B, f.model.n_classes, f.K, f.window_rows, f.lam))


def n_rotating(f):
    """Distinct device copies of the cube the steps rotate over, so that
    together they exceed L2 (one copy when a single cube already does)."""
    return max(1, min(4, int(np.ceil(1.5 * L2_BYTES / f.cube.nbytes))))


def workload_config(f, extra=None):
    B, H, W = f.cube.shape
    nr = n_rotating(f)
    cfg = {"workload": workload_name(f),
           "H": H, "W": W, "B": B, "classes": f.model.n_classes, "K": f.K,
           "window_rows": f.window_rows, "lambda": f.lam,
           "l2": "%d rotating cube cop%s of %.0f MB (%.0f MB > 129 MB L2)" % (
               nr, "y" if nr == 1 else "ies", f.cube.nbytes / 1e6, nr * f.cube.nbytes / 1e6),
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


def stage_work(f, knn_pairs_per_launch=None):
    """Algorithmic work per launch of each stage and the roofline that bounds
    it: HBM bytes for the two passes over the cube and the normalisation,
    FP32-pipe lane-ops for the KNN (4 per (pixel, candidate) pair it
    evaluates: the whole window for the full scan, the measured count for the
    pruned walk), and no roofline for the one-CTA eigensolver (a latency,
    reported in microseconds). The covariance also carries its tensor work
    (2 B^2 flops per pixel)."""
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
        "jacobi": ("latency", None),
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
    from ncu_summary import source_sha
    return source_sha(stage)


def traffic_from_profiles(stage, workload):
    """DRAM bytes per launch of a stage from the committed ncu summary, if it
    was taken on this frame shape (workload: HxWxB) and on the current source
    of that stage."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(stage)
    for ln in open(path):
        parts = ln.split()
        if (len(parts) >= 4 and parts[0] == stage and parts[1] == sha
                and parts[3] == workload):
            return float(parts[2])
    return None


# ----------------------------------------------------------------- oracle --
def oracle_state(f):
    """Frame-wide inputs of the oracle's per-pixel stages and the time of its
    per-frame eigensolver. The band means and covariance (their timing comes
    from the row samples) use the oracle's C means and, above a million
    pixels, the same definition contracted by a library matmul per pixel
    chunk; the Jacobi is the oracle's own and is timed whole; the projection
    and probabilities are the oracle's, the latter computed in row blocks on
    all host cores."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    B, H, W = f.cube.shape
    mu = oracle.band_means(f.cube)
    C = (oracle.covariance_matmul(f.cube, mu) if H * W >= (1 << 20)
         else oracle.covariance(f.cube, mu))
    t0 = time.perf_counter()
    ev, V, _, st = oracle.jacobi(C)
    t_jac = time.perf_counter() - t0
    v1 = V[:, int(np.argmax(ev))]
    v1 = v1 if v1[int(np.argmax(np.abs(v1)))] > 0 else -v1
    _, I_norm = oracle.project(f.cube, mu, v1)
    blocks = [(r, min(H, r + 32)) for r in range(0, H, 32)]

    def probs(rr):
        return oracle.svm_probs(np.ascontiguousarray(f.cube[:, rr[0]:rr[1], :]), f.model)[0]

    with ThreadPoolExecutor(max_workers=host_cores()) as ex:
        P = np.concatenate(list(ex.map(probs, blocks)), axis=1)
    return {"mu": mu, "v1": v1, "t_jacobi": t_jac,
            "I32": I_norm.reshape(H, W).astype(np.float32), "P32": P.astype(np.float32)}


def oracle_rows_single(f, state, rows):
    """The oracle's per-pixel stages on a row sample, one core; seconds per
    frame (scaled by H / rows, plus the per-frame Jacobi) and a description."""
    import oracle
    B, H, W = f.cube.shape
    sub = np.ascontiguousarray(f.cube[:, rows, :])
    t0 = time.perf_counter()
    mu_s = oracle.band_means(sub)
    oracle.covariance(sub, mu_s)
    oracle.project(sub, state["mu"], state["v1"])
    oracle.svm_probs(sub, f.model)
    for r in rows:
        oracle.knn(state["I32"], state["P32"], f.K, f.window_rows, f.lam, r * W, (r + 1) * W)
    t = time.perf_counter() - t0
    scale = H / float(len(rows))
    desc = ("oracle (single-threaded C, FP64) on %d of %d rows: band means + covariance, "
            "projection, SVM + coupling and KNN timed on the rows and scaled by %.1f; "
            "full-frame Jacobi timed whole (%.2f s)" % (len(rows), H, scale, state["t_jacobi"]))
    return t * scale + state["t_jacobi"], desc


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


def oracle_parallel(f, state, rows_per_core=2, rounds=2, warmup=1):
    """The oracle as it stands, on every host core at once: one spawned
    process per core, each running the per-pixel stages (band means +
    covariance, projection, SVM + coupling, KNN) on its own rows of the
    frame. Each round is one such sample; its pixels are charged the
    per-frame Jacobi pro rata. Returns (pixels/s, cores, per-round walls in
    seconds including the Jacobi share, sample pixels per round, description)."""
    import multiprocessing as mp
    B, H, W = f.cube.shape
    N = H * W
    cores = host_cores()
    init = {"mu": state["mu"], "v1": state["v1"], "model": f.model, "I32": state["I32"],
            "P32": state["P32"], "K": f.K, "R": f.window_rows, "lam": f.lam, "W": W}
    rng = np.random.default_rng(1)
    sample_px = cores * rows_per_core * W
    jac_share = state["t_jacobi"] * sample_px / float(N)
    walls = []
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(init,)) as pool:
        for rnd in range(warmup + rounds):  # the first rounds warm the workers up
            blocks = []
            for c in range(cores):
                rows = np.sort(rng.choice(H, rows_per_core, replace=False))
                blocks.append((np.ascontiguousarray(f.cube[:, rows, :]), rows))
            t0 = time.perf_counter()
            pool.map(_oracle_rows, blocks, chunksize=1)
            if rnd >= warmup:
                walls.append(time.perf_counter() - t0 + jac_share)
    rate = sample_px / float(np.median(walls))
    desc = ("oracle (C, FP64) as it stands on %d host cores at once: %d spawned processes, each "
            "running band means + covariance, projection, SVM + coupling and KNN on %d random rows "
            "of the frame per round (%d pixels per round), each round charged the per-frame "
            "Jacobi pro rata (%.2f s per frame, timed whole on one core); median of %d rounds"
            % (cores, cores, rows_per_core, sample_px, state["t_jacobi"], len(walls)))
    return rate, cores, walls, sample_px, desc


def run_reference(args, f):
    """The oracle arm: the FP64 oracle as it stands on every host core, on the
    same workload; each step is one round of the row sample (one spawned
    process per core on its own rows), so the steps' time is what they ran."""
    from paper_2404_10631_gb300 import replicas
    _, rank, _ = replicas.env_ranks()
    if not replicas.reports(rank):  # under torchrun rank 0 alone times the oracle
        return
    state = oracle_state(f)  # frame-wide inputs (untimed but for the Jacobi)
    rate, cores, walls, sample_px, desc = oracle_parallel(
        f, state, rows_per_core=1, rounds=max(1, args.steps), warmup=max(1, min(args.warmup, 3)))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(walls)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(f, {"pixels_per_step": sample_px}),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours --
def pct(v):
    v = sorted(v)
    return {"p50": v[len(v) // 2], "p99": v[min(len(v) - 1, int(0.99 * len(v)))]}


def frame_stream(hsc, f, dev, args, world, F, fp32_rate, fp32_peak_note, with_e2e=True,
                 clocks=None):
    """Everything timed on one single-frame workload; returns a dict.

    value        K steps with F frames in flight (F contexts), cubes resident
    one_in_flight, plain_fp32
                 the same steps one frame at a time; plain_fp32 with the
                 covariance on the FP32 pipe (the plain per-frame FP32 path)
    coupling_f64 one frame at a time with the coupling solved in FP64
    stages       per-stage device time (CUDA events around each stage launch)
                 and its roofline fraction
    knn_*        the full-window scan and the heap selection on the same maps
    e2e          the steps through the public API with the cube copied from
                 pinned host memory and the labels read back every step"""
    import torch

    from paper_2404_10631_gb300 import replicas
    B, H, W = f.cube.shape
    N = H * W
    k = f.model.n_classes
    nr = n_rotating(f)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = hsc.Context(dev.index or 0, stream=stream)
    ctx.reserve(B, H, W, k)
    cubes = [torch.as_tensor(f.cube, device=dev)]
    cubes += [cubes[0].clone() for _ in range(nr - 1)]
    model = hsc.Model.from_host(f.model, device=dev)
    # launch shapes for this frame shape, picked by the library's autotuner
    t0 = time.perf_counter()
    tune_cfg = ctx.autotune(cubes[0], model, f.K, f.window_rows, f.lam)
    tune = {"config": tune_cfg, "seconds": time.perf_counter() - t0,
            "how": "hsc_autotune on the first cube: Gram TMA staging depth {3, 4} (B <= 128), "
                   "projection/SVM {1, 4} pixels per thread x {2, 4, 8, 16} CTAs per SM, pruned "
                   "KNN walk {32 px x 8, 32 x 6, 32 x 12, 64 x 8, and 32 x 8 and 64 x 8 with "
                   "the window tile staged by TMA} (pixels per CTA x undecided keys per lane), "
                   "median of 3 runs each; results do not depend on them"}
    streams = [stream] + [torch.cuda.Stream(dev) for _ in range(F - 1)]
    ctxs = [ctx] + [hsc.Context(dev.index or 0, stream=s) for s in streams[1:]]
    for c in ctxs[1:]:
        c.reserve(B, H, W, k)
        c.set_tuning(B, H, W, k, (tune_cfg["gram_stages"], tune_cfg["svm_px"],
                                  tune_cfg["svm_blocks_per_sm"],
                                  tune_cfg["knn_variant"]))  # the same launch shapes
    outs = [(torch.empty((H, W), dtype=torch.float32, device=dev),
             torch.empty((k, H, W), dtype=torch.float32, device=dev),
             torch.empty((k, H, W), dtype=torch.float32, device=dev),
             torch.empty((H, W), dtype=torch.int32, device=dev)) for _ in range(F)]
    I, P, O, lab = outs[0]

    def step(i, nf=F, flags=0):
        j = i % nf
        Ij, Pj, Oj, labj = outs[j]
        hsc.hsc_classify(ctxs[j], cubes[i % nr], model, f.K, f.window_rows, f.lam, flags=flags,
                         labels=labj, out_probs=Oj, one_band=Ij, probs=Pj)

    tstream = torch.cuda.Stream(dev)  # brackets the timed region across the F streams

    def timed(nf, flags=0, clk=None):
        """K steps with nf frames in flight: (elapsed ms, per-frame latencies, clocks)."""
        for i in range(args.warmup):
            step(i, nf, flags)
        for c in ctxs[:nf]:
            c.sync()
        replicas.barrier(world)
        torch.cuda.synchronize(dev)
        if clk:
            clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e0.record(tstream)
        for s in streams[:nf]:
            s.wait_event(e0)
        for i in range(args.steps):
            st[i].record(streams[i % nf])
            step(i, nf, flags)
            en[i].record(streams[i % nf])
        for s in streams[:nf]:
            ev_s = torch.cuda.Event()
            ev_s.record(s)
            tstream.wait_event(ev_s)
        e1.record(tstream)
        torch.cuda.synchronize(dev)
        replicas.barrier(world)
        for c in ctxs[:nf]:
            c.sync()  # raises on a device-side error of the timed steps
        return (e0.elapsed_time(e1), [st[i].elapsed_time(en[i]) for i in range(args.steps)],
                clk.stop() if clk else None)

    # ---- device-resident timed regions: F frames in flight, one at a time,
    # the plain FP32 path one at a time
    elapsed, per_step, clk = timed(F, 0, clocks)
    elapsed1, per_step1, _ = timed(1) if F > 1 else (elapsed, per_step, None)
    elapsed_p, per_step_p, _ = timed(1, hsc.HSC_COV_FP32_PIPE)
    sweeps, refine_iters, sweep_cyc, refine_cyc = ctx.pca_diagnostics(cycles=True)

    def profiled(flags=0):
        """Per-stage device ms per launch over the steps, one frame at a time
        on the first context, CUDA events around each stage launch."""
        ctx.profile(True)
        ctx.profile_read()
        for i in range(args.steps):
            step(i, 1, flags)
        ctx.sync()
        ms, kern, _ = ctx.profile_read()
        ctx.profile(False)
        return {n: v / args.steps for n, v in ms.items()}, kern

    ctx.knn_diagnostics()  # reset the pruned walk's counters
    stage_ms, stage_kernels = profiled()
    knn_evals, knn_redo = ctx.knn_diagnostics()  # the profiled steps
    knn_evals_per_launch = knn_evals / float(args.steps)
    plain_ms, _ = profiled(hsc.HSC_COV_FP32_PIPE)
    f64_ms, _ = profiled(hsc.HSC_SVM_COUPLE_F64)

    # ---- the paper's full-window KNN on the same maps (timed on its own),
    # and its heap selection as an A/B point
    ctx.profile(True)
    ctx.profile_read()
    n_full = min(args.steps, 16)
    for i in range(n_full):
        hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, f.lam, out_probs=O, labels=lab,
                           search=hsc.HSC_KNN_SEARCH_FULL)
    full_ms, _, _ = ctx.profile_read()
    n_heap = min(args.steps, 2)
    for i in range(n_heap):
        hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, f.lam, out_probs=O, labels=lab,
                           search=hsc.HSC_KNN_SEARCH_HEAP)
    heap_ms, _, _ = ctx.profile_read()
    ctx.profile(False)
    ctx.sync()
    full_ms_launch = full_ms["knn"] / n_full
    heap_ms_launch = heap_ms["knn"] / n_heap
    # ---- the pruned walk's variants (the autotuner's candidates; 4 and 5
    # stage the window tile with one TMA box instead of 16-byte asynchronous
    # copies): the KNN stage of the profiled steps per variant, then the tuned
    # variant again
    walk_ms = {}
    for v in range(6):
        ctx.set_tuning(B, H, W, k, (tune_cfg["gram_stages"], tune_cfg["svm_px"],
                                    tune_cfg["svm_blocks_per_sm"], v))
        v_ms, _ = profiled()
        walk_ms[v] = v_ms["knn"]
    ctx.set_tuning(B, H, W, k, (tune_cfg["gram_stages"], tune_cfg["svm_px"],
                                tune_cfg["svm_blocks_per_sm"], tune_cfg["knn_variant"]))
    knn_walks = {"ms_per_launch": {("%d: %s" % (v, name)): round(walk_ms[v], 5)
                                   for v, name in enumerate(("32 px x 8 keys", "32 x 6", "32 x 12",
                                                             "64 x 8", "32 x 8, TMA tile",
                                                             "64 x 8, TMA tile"))},
                 "tuned": tune_cfg["knn_variant"],
                 "note": "the KNN stage (pruned walk + redo pass) of the profiled steps per walk "
                         "variant; the outputs are the same bit for bit"}
    e_max, e1_max, ep_max = replicas.max_over_ranks([elapsed, elapsed1, elapsed_p], world, dev)
    value = replicas.whole_job_rate(N * args.steps, world, e_max / 1e3)
    value1 = replicas.whole_job_rate(N * args.steps, world, e1_max / 1e3)
    value_p = replicas.whole_job_rate(N * args.steps, world, ep_max / 1e3)

    # ---- per-stage rooflines (SURVEY-style bounds: HBM for the passes over
    # the cube, FP32 pipe for the KNN, latency for the one-CTA eigensolver)
    peaks, peak_src = load_peaks()
    work = stage_work(f, knn_evals_per_launch)
    wname = "%dx%dx%d" % (H, W, B)  # the shape tag of the committed traffic lines
    stages = {}
    for name, ms in stage_ms.items():
        if stage_kernels[name] == 0:
            continue
        bound, units = work[name]
        entry = {"ms_per_launch": ms, "share": ms / max(1e-12, sum(stage_ms.values())),
                 "kernels_per_launch": stage_kernels[name] / float(args.steps), "bound": bound}
        if bound == "hbm":
            ach = units / (ms / 1e3) / 1e9
            entry.update(achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                         frac=ach / peaks["hbm_gbs"], algorithmic=units,
                         traffic=traffic_from_profiles(name, wname))
        elif bound == "alu":
            ach = units / (ms / 1e3) / 1e12
            entry.update(achieved=ach, peak=fp32_rate, unit="TFLOP/s", frac=ach / fp32_rate,
                         algorithmic=units, traffic=traffic_from_profiles(name, wname),
                         note="4 FP32-pipe ops per (pixel, candidate) pair the pruned walk "
                              "evaluated; peak: " + fp32_peak_note)
        else:
            entry["us_per_launch"] = 1e3 * ms
            entry["note"] = ("a latency, no roofline: one CTA per frame up to 128 bands; for "
                             "129-256 bands the first sweep on a 16-CTA cluster, then one CTA; "
                             "with frames in flight the other frames' GPU-wide stages run "
                             "beside it")
        if name == "moments":
            flops = 2.0 * B * B * N
            entry["tensor"] = {"algorithmic_flops": flops,
                               "achieved_tflops": flops / (ms / 1e3) / 1e12,
                               "frac_of_bf16_burst": flops / (ms / 1e3) / 1e12 / peaks["bf16_tflops"],
                               "note": "the Gram's 2 B^2 flops per pixel (the hi/lo split issues "
                                       "three MMAs per product)"}
        stages[name] = entry
    # the roofline object: the dominant stage among those with a roofline
    # (the eigensolver holds one SM and overlaps other frames' stages)
    dom = max((n for n in stages if stages[n]["bound"] in ("hbm", "alu")),
              key=lambda n: stages[n]["ms_per_launch"])
    d = stages[dom]
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"],
                "peak": d["peak"], "unit": d["unit"], "frac": d["frac"],
                "traffic": d.get("traffic"),
                "peak_source": ("FP32 FFMA issue rate measured in this run (hsc_measure_fma_rate)"
                                if d["bound"] == "alu" else
                                "hbm_gbs (burst copy) of MEASURED_PEAKS.json, %s" % peak_src),
                "work_per_launch": d["algorithmic"],
                "ms_per_launch": d["ms_per_launch"],
                "rule": "the stage with the largest device time among those with a roofline "
                        "(moments, projection + SVM, normalisation: HBM; KNN: FP32 pipe); the "
                        "eigensolver is a latency, reported in stages.jacobi"}
    full_ops = 4.0 * knn_pairs(H, W, f.window_rows)
    full_ach = full_ops / (full_ms_launch / 1e3) / 1e12
    knn_full = {"search": "full window (the paper's procedure: every window candidate)",
                "bound": "alu", "ms_per_launch": full_ms_launch, "achieved": full_ach,
                "peak": fp32_rate, "unit": "TFLOP/s", "frac": full_ach / fp32_rate,
                "work_per_launch": full_ops,
                "traffic": traffic_from_profiles("knn_full", wname),
                "note": "same neighbour sets as the pruned walk used in the step"}
    knn_heap = {"search": "heap selection (the paper's partial heapsort: every window candidate "
                          "keyed, the K smallest kept in a max-heap)",
                "ms_per_launch": heap_ms_launch,
                "note": "same neighbour sets as the other searches; an A/B point, not the step"}
    pruned_ms = stages["knn"]["ms_per_launch"]
    knn_pruned = {"search": "pruned walk (exact)", "candidates_per_launch": knn_evals_per_launch,
                  "window_pairs_per_launch": knn_pairs(H, W, f.window_rows),
                  "redo_pixels_per_launch": knn_redo / float(args.steps),
                  "ms_per_launch": pruned_ms,
                  "frac_on_evaluated_pairs": stages["knn"].get("frac"),
                  # the full window's work (4 FP32 ops per window pair) over the pruned
                  # walk's time, against the FP32 pipe: the same neighbour sets in less
                  # time than the full scan could take at the pipe's peak when above 1
                  "window_equivalent_frac": full_ops / (pruned_ms / 1e3) / 1e12 / fp32_rate}

    out = {"workload": workload_name(f), "config": workload_config(f, {"frames_in_flight": F}),
           "value": value, "unit": UNIT, "ms_per_step": e_max / args.steps,
           "latency_ms": pct(per_step),
           "one_in_flight": {"value": value1, "unit": UNIT, "ms_per_step": e1_max / args.steps,
                             "latency_ms": pct(per_step1),
                             "note": "the same steps on one context, one frame at a time"},
           "plain_fp32": {"value": value_p, "unit": UNIT, "ms_per_step": ep_max / args.steps,
                          "latency_ms": pct(per_step_p),
                          "stages_ms": {n: v for n, v in plain_ms.items() if v > 0},
                          "note": "the plain per-frame FP32 path: covariance Gram on the FP32 "
                                  "pipe (HSC_COV_FP32_PIPE), FP32 SVM and KNN, one frame at a "
                                  "time on one context",
                          "speedup_in_flight": value / value_p,
                          "speedup_one_in_flight": value1 / value_p,
                          "p99_ratio_in_flight": pct(per_step)["p99"] / pct(per_step_p)["p99"]},
           "coupling_f64": {"project_svm_ms": f64_ms.get("project_svm"),
                            "project_svm_ms_fp32": stage_ms.get("project_svm"),
                            "frame_ms": sum(f64_ms.values()),
                            "note": "HSC_SVM_COUPLE_F64: the per-pixel coupling solve in FP64, "
                                    "one frame at a time (stage device times)"},
           "roofline": roofline, "stages": stages,
           "knn_full_window": knn_full, "knn_pruned": knn_pruned, "knn_heap": knn_heap,
           "knn_walk_variants": knn_walks,
           "gpu_launches": int(round(sum(stage_kernels.values()))),
           "autotune": tune,
           "jacobi": {"fp32_sweeps": sweeps, "refine_iters": refine_iters,
                      "sweep_cycles": sweep_cyc, "refine_cycles": refine_cyc},
           "clocks": clk}

    if with_e2e:
        # ---- end to end through the public API with host buffers
        host_cube = torch.empty((B, H, W), dtype=torch.float32).pin_memory()
        host_cube.copy_(torch.from_numpy(f.cube))
        host_labs = [torch.empty((H, W), dtype=torch.int32).pin_memory() for _ in range(F)]
        host_model = [torch.from_numpy(a).pin_memory() for a in
                      (f.model.w, f.model.b, f.model.platt_a, f.model.platt_b)]
        # per context: its device cube and its own model copy (the copies of one
        # step and the kernels of another never share a buffer)
        e2e_models = [hsc.Model.from_host(f.model, device=dev) for _ in range(F)]
        e2e_cubes = [cubes[j] if j < nr else torch.empty((B, H, W), dtype=torch.float32,
                                                           device=dev) for j in range(F)]
        h2d = host_cube.numel() * 4 + sum(a.numel() * 4 for a in host_model)
        d2h = host_labs[0].numel() * 4
        # the host link's own rate for this copy (pinned cube -> device, CUDA
        # events), the ceiling of the end-to-end number
        for r in range(6):
            if r == 2:
                l0 = torch.cuda.Event(enable_timing=True)
                l0.record(stream)
            e2e_cubes[0].copy_(host_cube, non_blocking=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l1.record(stream)
        l1.synchronize()
        link_gbs = host_cube.numel() * 4 * 4 / (l0.elapsed_time(l1) / 1e3) / 1e9
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
                for d_, h in zip((mj.w, mj.b, mj.platt_a, mj.platt_b), host_model):
                    d_.copy_(h, non_blocking=True)
                hsc.hsc_classify(ctxs[j], dcube, mj, f.K, f.window_rows, f.lam,
                                 labels=outs[j][3])
                host_labs[j].copy_(outs[j][3], non_blocking=True)
                done[j] = torch.cuda.Event()
                done[j].record(streams[j])
        for s_ in streams:
            s_.synchronize()
        e2e_s = time.perf_counter() - t0
        for c in ctxs:
            c.sync()
        e2e_value = replicas.whole_job_rate(N * n_e2e, world,
                                            replicas.max_over_ranks([e2e_s], world, dev)[0])
        bound = world * link_gbs * 1e9 / h2d * N
        out["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "steps": n_e2e, "h2d_link_gbs": link_gbs,
                      "link_bound": bound, "frac_of_link_bound": e2e_value / bound,
                      "note": "each frame's cube crosses the host link once (pinned host -> "
                              "device); h2d_link_gbs is that copy alone, timed in this run, and "
                              "link_bound the pixels/s it allows on every rank's own link"}
        del host_cube, e2e_cubes
    for c in ctxs[1:]:
        c.close()
    ctx.close()
    del cubes, outs
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    return out


def run_ours(args, f):
    import torch

    import paper_2404_10631_gb300 as hsc
    from paper_2404_10631_gb300 import build as hbuild
    from paper_2404_10631_gb300 import replicas

    world, rank, local = replicas.env_ranks()
    torch.cuda.set_device(local)
    replicas.init(world, local, "nccl")
    if rank == 0:
        hbuild.build()
    replicas.barrier(world)
    dev = torch.device("cuda", local)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, peak_src = load_peaks()
    # FP32 / FP64 multiply-add issue rates of this GPU, measured here (T lane-ops/s)
    fp32_rate = hsc.hsc_measure_fma_rate(dev.index) / 1e12
    fp64_rate = hsc.hsc_measure_fma_rate(dev.index, fp64=True) / 1e12
    note = "FP32 FFMA issue rate measured in this run (hsc_measure_fma_rate)"
    F = max(1, args.frames_in_flight)

    head = frame_stream(hsc, f, dev, args, world, F, fp32_rate, note, clocks=ClockSampler(local))
    neuro = None
    if not args.no_neuro:
        fn = synth.make_config(NEURO_CFG)
        neuro = frame_stream(hsc, fn, dev, args, world, F, fp32_rate, note)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = hsc.Context(local, stream=stream)
    batch = None
    if not args.no_batch:
        batch = run_batch(hsc, ctx, stream, dev, args)
    serving = None
    if not args.no_serving and world == 1:
        serving = run_serving(hsc, ctx, stream, dev, args)
    ctx.close()

    B, H, W = f.cube.shape
    N = H * W
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(f, {"frames_per_step_per_gpu": 1, "frames_in_flight": F,
                                          "precision": "cube float32; covariance Gram FP16 hi/lo "
                                                       "on tensor cores, FP32 accumulation; "
                                                       "eigenpair refined to an FP64-level "
                                                       "residual; SVM, coupling and KNN FP32"}),
            "latency_ms": head["latency_ms"],
            "one_in_flight": head["one_in_flight"],
            "plain_fp32": head["plain_fp32"],
            "coupling_f64": head["coupling_f64"],
            "roofline": head["roofline"],
            "stages": head["stages"],
            "knn_full_window": head["knn_full_window"],
            "knn_pruned": head["knn_pruned"],
            "knn_heap": head["knn_heap"],
            "knn_walk_variants": head["knn_walk_variants"],
            "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"],
            "autotune": head["autotune"],
            "jacobi": head["jacobi"],
            "neuro": neuro,
            "batch": batch,
            "serving": serving,
            "fp_peaks": {"fp32_lane_ops_per_s": fp32_rate * 1e12,
                         "fp64_lane_ops_per_s": fp64_rate * 1e12,
                         "fp32_nominal": fp32_pipe_peak_tops(sm_count,
                                                             peaks.get("sm_max_mhz", 2070.0)) * 1e12,
                         "how": "hsc_measure_fma_rate: 8 independent FFMA / DFMA chains per "
                                "thread, 1024 threads per SM, CUDA events"},
            "clocks": head["clocks"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        state = oracle_state(f)
        rows = np.linspace(0, H - 1, 4).astype(int)
        t_frame, desc = oracle_rows_single(f, state, rows)
        rate, cores, walls, sample_px, desc_par = oracle_parallel(f, state)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": desc_par,
                                "single_core": {"value": N / t_frame, "unit": UNIT, "cores": 1,
                                                "sample": desc}}
    if replicas.reports(rank):
        print(json.dumps(line), flush=True)
    replicas.finalize(world)


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

    def fused():
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam,
                               flags=hsc.HSC_BATCH_GRAPH | hsc.HSC_BATCH_FUSED, labels=labs)

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
    s_ms, s_per = timed(fused, reps)
    o_ms, _ = timed(pooled, 3)
    p_ms, p_per = timed(per_frame, 3)
    # per-stage device time of the stage-major form (calls without a graph)
    def stage_ms(flags):
        ctx.profile(True)
        ctx.profile_read()
        for _ in range(3):
            hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam, flags=flags,
                                   labels=labs)
        ctx.sync()
        st_ms, _, _ = ctx.profile_read()
        ctx.profile(False)
        return {n: round(ms / 3, 4) for n, ms in st_ms.items() if ms > 0}

    stages = stage_ms(0)
    stages_fused = stage_ms(hsc.HSC_BATCH_FUSED)
    return {"workload": "%d square snapshot frames, sides 40-64 px, 125 bands float32, "
                        "4 classes (shared model), K=16, 7-row window, lambda=1" % n_frames,
            "pixels_per_batch": px,
            "batched": {"value": px / (b_ms / 1e3), "unit": UNIT, "ms_per_batch": b_ms,
                        "p50_ms": b_per[len(b_per) // 2], "p99_ms": b_per[-1],
                        "api": "hsc_classify_batch, stage-major (one launch per stage over "
                               "every frame), CUDA-graph replay",
                        "stages_ms": stages},
            "fused": {"value": px / (s_ms / 1e3), "unit": UNIT, "ms_per_batch": s_ms,
                      "p50_ms": s_per[len(s_per) // 2], "p99_ms": s_per[-1],
                      "api": "the same with the projection/SVM, normalisation and KNN of each "
                             "frame group in one persistent kernel (HSC_BATCH_FUSED; booked to "
                             "the knn stage), CUDA-graph replay",
                      "stages_ms": stages_fused},
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
    ap.add_argument("--no-neuro", action="store_true",
                    help="skip the 416x512x128 neurosurgery-scale frame")
    ap.add_argument("--frames-in-flight", type=int, default=8,
                    help="contexts (streams) the steps rotate over; 1 = one frame at a time")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    f = synth.make_config(HEADLINE_CFG)
    if args.impl == "reference":
        run_reference(args, f)
    else:
        run_ours(args, f)


if __name__ == "__main__":
    main()
