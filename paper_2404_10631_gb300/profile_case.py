"""Repeat one entry point on a synthetic workload, for profilers (ncu).

    python -m paper_2404_10631_gb300.profile_case --op classify --reps 2

--op: classify | covariance | pca | svm | knn. The first call is a warm-up; an
ncu capture of the second launch of a kernel uses ``-s 1 -c 1``.
"""

from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="classify",
                    choices=("classify", "covariance", "pca", "svm", "knn"))
    ap.add_argument("--config", type=int, default=2, help="synthetic workload (1 tiny, 2 neuro)")
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_2404_10631_gb300 as hsc
    import synth
    from paper_2404_10631_gb300 import build

    build.build()
    f = synth.make_config(a.config)
    ctx = hsc.Context(0)
    cube = torch.as_tensor(f.cube, device="cuda")
    model = hsc.Model.from_host(f.model)
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
            hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, f.lam)
    ctx.sync()
    print("ok", a.op, "jacobi sweeps, refine iters, sweep cycles, refine cycles:",
          ctx.pca_diagnostics(cycles=True))


if __name__ == "__main__":
    main()
