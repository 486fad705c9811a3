"""Repeat one entry point on a synthetic workload, for profilers (ncu).

    python profile_case.py --op classify --reps 2

--op: classify | covariance | pca | svm | knn | batch. The first call is a
warm-up; an ncu capture of the second launch of a kernel uses ``-s 1 -c 1``.
--op batch: hsc_classify_batch over the 256 uneven snapshot frames (125
bands, sides 40-64 px, shared model, K = 16, 7-row window), stage-major
(15 launches per call: the pilots, the Gram items and the reductions, then
for each of the two frame groups the eigensolver's two launches and the
projection/SVM, normalisation, KNN walk and redo pass), --reps calls after the
same number of warm-up calls.
"""

from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="classify",
                    choices=("classify", "covariance", "pca", "svm", "knn", "batch"))
    ap.add_argument("--config", type=int, default=2, help="synthetic workload (1 tiny, 2 neuro)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--shape", default=None,
                    help="B,H,W: a frame of the 1024x1024x256 workload's generator (two wide "
                         "Gaussians per class spectrum, sigma 0.01) at this size instead of "
                         "--config")
    ap.add_argument("--search", default="auto", choices=("auto", "full", "pruned", "heap"),
                    help="KNN search of --op knn")
    ap.add_argument("--knn-variant", type=int, default=None,
                    help="pruned walk variant of --op classify (hsc_set_tuning; 4 and 5 stage "
                         "the window tile by TMA); default: the untuned one")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch

    import paper_2404_10631_gb300 as hsc
    import synth
    from paper_2404_10631_gb300 import build

    build.build()
    if a.op == "batch":
        frames = synth.make_batch(256)
        f0 = frames[0]
        ctx = hsc.Context(0)
        model = hsc.Model.from_host(f0.model)
        cubes = [torch.as_tensor(fr.cube, device="cuda") for fr in frames]
        labs = [torch.empty(fr.cube.shape[1:], dtype=torch.int32, device="cuda") for fr in frames]
        for _ in range(2 * a.reps):
            hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam, labels=labs)
        ctx.sync()
        print("ok batch: %d frames, %d calls" % (len(frames), 2 * a.reps))
        return
    if a.shape:
        B, H, W = (int(v) for v in a.shape.split(","))
        f = synth.make_frame(synth.SEEDS[4], H, W, B, sigma=0.01, n_seeds=32, n_gauss=2,
                             wide=True, K=40, window_rows=14, lam=1.0)
    else:
        f = synth.make_config(a.config)
    ctx = hsc.Context(0)
    cube = torch.as_tensor(f.cube, device="cuda")
    model = hsc.Model.from_host(f.model)
    if a.knn_variant is not None:
        B, H, W = f.cube.shape
        ctx.set_tuning(B, H, W, f.model.n_classes, (0, 0, 0, a.knn_variant))
    I = hsc.hsc_pca_one_band(ctx, cube)
    P = hsc.hsc_svm_probs(ctx, cube, model)
    for _ in range(a.reps):
        if a.op == "classify":
            hsc.hsc_classify(ctx, cube, model, f.K, f.window_rows, f.lam)
        elif a.op == "covariance":
            hsc.hsc_pca_covariance(ctx, cube)
        elif a.op == "pca":
            hsc.hsc_pca_one_band(ctx, cube, one_band=I)
        elif a.op == "svm":
            hsc.hsc_svm_probs(ctx, cube, model, probs=P)
        else:
            search = {"auto": hsc.HSC_KNN_SEARCH_AUTO, "full": hsc.HSC_KNN_SEARCH_FULL,
                      "pruned": hsc.HSC_KNN_SEARCH_PRUNED, "heap": hsc.HSC_KNN_SEARCH_HEAP}[a.search]
            hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, f.lam, search=search)
    ctx.sync()
    print("ok", a.op, "jacobi sweeps, refine iters, sweep cycles, refine cycles:",
          ctx.pca_diagnostics(cycles=True))


if __name__ == "__main__":
    main()
