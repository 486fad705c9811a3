"""Frames in flight: several contexts, each with its own stream, classify
different frames at the same time (the throughput form bench.py times);
every frame's outputs equal what one context gives for it alone, bit for
bit: the contexts share no scratch and no kernel reads another's buffers."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_frames_in_flight_equal_one_at_a_time(hsc, ctx):
    import torch
    frames = [synth.make_config(2)] + [synth.make_frame(600 + i, 96 + 8 * i, 128 - 4 * i, 128,
                                                        sigma=0.02, K=40, window_rows=14)
                                       for i in range(5)]
    k = 4
    F = 4
    streams = [torch.cuda.Stream() for _ in range(F)]
    ctxs = [hsc.Context(0, stream=s) for s in streams]
    try:
        cubes = [torch.as_tensor(f.cube, device="cuda") for f in frames]
        models = [hsc.Model.from_host(f.model) for f in frames]

        def outputs(f):
            H, W = f.cube.shape[1:]
            return (torch.empty((H, W), dtype=torch.int32, device="cuda"),
                    torch.empty((k, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
                    torch.empty((k, H, W), device="cuda"))

        ref = []
        for f, c, m in zip(frames, cubes, models):  # one at a time on one context
            lab, O, I, P = outputs(f)
            hsc.hsc_classify(ctx, c, m, f.K, f.window_rows, f.lam, labels=lab, out_probs=O,
                             one_band=I, probs=P)
            ctx.sync()
            ref.append((lab, O, I, P))
        for rep in range(2):
            got = []
            for i, (f, c, m) in enumerate(zip(frames, cubes, models)):  # all in flight
                lab, O, I, P = outputs(f)
                hsc.hsc_classify(ctxs[i % F], c, m, f.K, f.window_rows, f.lam, labels=lab,
                                 out_probs=O, one_band=I, probs=P)
                got.append((lab, O, I, P))
            for c in ctxs:
                c.sync()
            for g, r in zip(got, ref):
                for x, y in zip(g, r):
                    np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    finally:
        for c in ctxs:
            c.close()
