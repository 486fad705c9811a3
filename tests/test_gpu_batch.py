"""hsc_classify_batch: every frame's outputs are bit-identical to what
hsc_classify gives for that frame alone (uneven snapshot frames, shared
model), in the stage-major form (its projection/SVM, normalisation and KNN
as three launches, or fused in one persistent kernel) and the stream-pool form,
with and without CUDA-graph replay; long work items (two accumulator segments), pixel counts
that are not a multiple of 4, a cube that is not 16-byte aligned and an
out-of-range pixel (the FP32 recompute) included."""

import numpy as np
import pytest

import synth
from parity import e2e_check

pytestmark = pytest.mark.gpu


def frames_to_device(frames):
    import torch
    return [torch.as_tensor(f.cube, device="cuda") for f in frames]


def outputs(frames, k):
    import torch
    labs = [torch.full(f.cube.shape[1:], -1, dtype=torch.int32, device="cuda") for f in frames]
    O = [torch.full((k,) + f.cube.shape[1:], -1.0, device="cuda") for f in frames]
    I = [torch.full(f.cube.shape[1:], -1.0, device="cuda") for f in frames]
    P = [torch.full((k,) + f.cube.shape[1:], -1.0, device="cuda") for f in frames]
    return labs, O, I, P


def alone(hsc, ctx, f, cube, model):
    import torch
    k = f.model.n_classes
    lab = torch.empty(f.cube.shape[1:], dtype=torch.int32, device="cuda")
    O = torch.empty((k,) + f.cube.shape[1:], device="cuda")
    I = torch.empty(f.cube.shape[1:], device="cuda")
    P = torch.empty((k,) + f.cube.shape[1:], device="cuda")
    hsc.hsc_classify(ctx, cube, model, f.K, f.window_rows, f.lam, labels=lab, out_probs=O,
                     one_band=I, probs=P)
    ctx.sync()  # the context's stream does not order with torch's
    return lab, O, I, P


def assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("pool", [False, True])
def test_batch_equals_frames_alone(hsc, ctx, graph, pool):
    frames = synth.make_batch(12)
    # two frames whose pixel count is not a multiple of 4 (scalar loads,
    # FP32-pipe covariance)
    frames += [synth.make_frame(77, 41, 43, 125, sigma=0.03, K=16, window_rows=7,
                                spectra=frames[0].spectra),
               synth.make_frame(78, 9, 61, 125, sigma=0.03, K=16, window_rows=7,
                                spectra=frames[0].spectra)]
    f0 = frames[0]
    model = hsc.Model.from_host(f0.model)
    cubes = frames_to_device(frames)
    labs, O, I, P = outputs(frames, 4)
    flags = (hsc.HSC_BATCH_GRAPH if graph else 0) | (hsc.HSC_BATCH_POOL if pool else 0)
    for rep in range(2):  # the second call replays the graph
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam, flags=flags,
                               labels=labs, out_probs=O, one_bands=I, probs=P)
        ctx.sync()
        for i, f in enumerate(frames):
            assert_same((labs[i], O[i], I[i], P[i]), alone(hsc, ctx, f, cubes[i], model))
        ctx.sync()


def test_graph_replay_sees_new_data(hsc, ctx):
    import torch
    frames = synth.make_batch(6)
    f0 = frames[0]
    model = hsc.Model.from_host(f0.model)
    cubes = frames_to_device(frames)
    labs, O, I, P = outputs(frames, 4)
    args = dict(labels=labs, out_probs=O, one_bands=I, probs=P, flags=hsc.HSC_BATCH_GRAPH)
    hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam, **args)
    ctx.sync()
    # new contents in the same buffers: the replayed graph must read them
    other = synth.make_batch(6, seed=4242)
    for c, f2 in zip(cubes, other):
        if tuple(c.shape) == f2.cube.shape:
            c.copy_(torch.as_tensor(f2.cube, device="cuda"))
        else:
            c.copy_(torch.flip(c, dims=[1]))
    torch.cuda.synchronize()  # the edits are done before the library reads the cubes
    hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam, **args)
    ctx.sync()
    for i, f in enumerate(frames):
        assert_same((labs[i], O[i], I[i], P[i]), alone(hsc, ctx, f, cubes[i], model))


def test_more_frames_than_streams(hsc, ctx):
    frames = synth.make_batch(70)
    f0 = frames[0]
    model = hsc.Model.from_host(f0.model)
    cubes = frames_to_device(frames)
    labs = hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam)
    ctx.sync()
    for i in (0, 1, 63, 64, 65, 69):
        ref = alone(hsc, ctx, frames[i], cubes[i], model)[0]
        np.testing.assert_array_equal(labs[i].cpu().numpy(), ref.cpu().numpy())
    # labels follow the synthetic regions
    acc = np.mean([(l.cpu().numpy() == f.truth).mean() for l, f in zip(labs, frames)])
    assert acc > 0.95


def test_batch_rejects_bad_frame(hsc, ctx):
    import torch
    frames = synth.make_batch(3)
    f0 = frames[0]
    model = hsc.Model.from_host(f0.model)
    cubes = frames_to_device(frames)
    cubes[1] = cubes[1][:100].contiguous()  # band count differs
    with pytest.raises(ValueError):
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam)


def _alone_vs_batch(hsc, ctx, frames, cubes, flags=0, batch_flags=0):
    import torch
    f0 = frames[0]
    k = f0.model.n_classes
    model = hsc.Model.from_host(f0.model)
    labs, O, I, P = outputs(frames, k)
    hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam,
                           flags=flags | batch_flags, labels=labs, out_probs=O, one_bands=I,
                           probs=P)
    ctx.sync()
    for i, f in enumerate(frames):
        lab = torch.empty(f.cube.shape[1:], dtype=torch.int32, device="cuda")
        Oa = torch.empty((k,) + f.cube.shape[1:], device="cuda")
        Ia = torch.empty(f.cube.shape[1:], device="cuda")
        Pa = torch.empty((k,) + f.cube.shape[1:], device="cuda")
        hsc.hsc_classify(ctx, cubes[i], model, f.K, f.window_rows, f.lam, flags=flags,
                         labels=lab, out_probs=Oa, one_band=Ia, probs=Pa)
        ctx.sync()
        assert_same((labs[i], O[i], I[i], P[i]), (lab, Oa, Ia, Pa))


def test_staged_batch_long_items_and_alignment(hsc, ctx):
    """A 768 x 1024 frame (81 chunks per Gram item: two accumulator segments;
    alone it takes the tensor-map kernel), a 331 x 257 frame (odd pixel
    count: 4-byte copies, and alone the work-item kernel), a cube 4 bytes off
    16-byte alignment, and small frames, 32 bands, in one stage-major batch."""
    import torch
    B = 32
    big = synth.make_frame(501, 768, 1024, B, sigma=0.03, K=16, window_rows=7)
    sp = big.spectra
    frames = [big,
              synth.make_frame(502, 331, 257, B, sigma=0.03, K=16, window_rows=7, spectra=sp),
              synth.make_frame(503, 48, 64, B, sigma=0.03, K=16, window_rows=7, spectra=sp),
              synth.make_frame(504, 40, 40, B, sigma=0.03, K=16, window_rows=7, spectra=sp),
              synth.make_frame(505, 9, 61, B, sigma=0.03, K=16, window_rows=7, spectra=sp)]
    cubes = frames_to_device(frames)
    # frame 3 from a buffer one float past a 16-byte boundary
    n3 = frames[3].cube.size
    buf = torch.empty(n3 + 1, device="cuda")
    buf[1:].copy_(torch.as_tensor(frames[3].cube.ravel(), device="cuda"))
    cubes[3] = buf[1:].view(frames[3].cube.shape)
    torch.cuda.synchronize()
    assert cubes[3].data_ptr() % 16 != 0
    _alone_vs_batch(hsc, ctx, frames, cubes)


def test_staged_batch_out_of_range_pixel(hsc, ctx):
    """One pixel of one frame far outside FP16's range after scaling: its
    Gram item is recomputed on the FP32 pipe in the batch as it is alone."""
    frames = synth.make_batch(4, seed=777)
    # 128 x 128: the pilot samples runs of 256 pixels starting at r (N - 256) / 15,
    # so pixel 700 is outside it
    frames.insert(2, synth.make_frame(779, 128, 128, 125, sigma=0.03, K=16, window_rows=7,
                                      spectra=frames[0].spectra))
    cubes = frames_to_device(frames)
    cubes[2][5].view(-1)[700] += 5e3
    import torch
    torch.cuda.synchronize()  # the outlier is in place before the library reads the cube
    _alone_vs_batch(hsc, ctx, frames, cubes)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("flags", ["raw", "f64"])
def test_staged_batch_flags(hsc, ctx, flags, fused):
    """HSC_CLASSIFY_RAW_I and HSC_SVM_COUPLE_F64 in the stage-major batch,
    with the projection/SVM, normalisation and KNN as three launches and
    fused in one persistent kernel (HSC_BATCH_FUSED)."""
    frames = synth.make_batch(6, seed=778)
    fl = hsc.HSC_CLASSIFY_RAW_I if flags == "raw" else hsc.HSC_SVM_COUPLE_F64
    _alone_vs_batch(hsc, ctx, frames, frames_to_device(frames), flags=fl,
                    batch_flags=hsc.HSC_BATCH_FUSED if fused else 0)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("graph", [False, True])
def test_staged_batch_more_frames_than_sms(hsc, ctx, graph, fused):
    """More frames than SMs: the first wave's frames and the rest run their
    eigensolver-to-KNN chains on two streams (the second on a high-priority
    one), each group's projection/SVM, normalisation and KNN as three
    launches or (fused) in one persistent kernel with its own work counters;
    every frame still equals its single-frame call."""
    import torch
    frames = synth.make_batch(170, seed=780)
    assert len(frames) > torch.cuda.get_device_properties(0).multi_processor_count
    cubes = frames_to_device(frames)
    bflags = (hsc.HSC_BATCH_GRAPH if graph else 0) | (hsc.HSC_BATCH_FUSED if fused else 0)
    _alone_vs_batch(hsc, ctx, frames, cubes, batch_flags=bflags)
    if graph:  # the replay (the work counters start from zero again)
        _alone_vs_batch(hsc, ctx, frames, cubes, batch_flags=bflags)


def test_staged_graph_replay_with_frames_permuted(hsc, ctx):
    """More frames than SMs, graph mode, then the same frames in another
    order: the frame counts, work-item counts and window rows match, but the
    split between the two frame groups (first wave of eigensolvers, the rest
    on the high-priority stream) moves. The replay must not reuse the old
    split; every frame must still equal its single-frame call."""
    import torch
    frames = synth.make_batch(170, seed=781)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert len(frames) > sm
    cubes = frames_to_device(frames)
    _alone_vs_batch(hsc, ctx, frames, cubes, batch_flags=hsc.HSC_BATCH_GRAPH)
    perm = np.random.default_rng(5).permutation(len(frames))
    # the first wave now holds other frames (another pixel split)
    assert sum(frames[i].cube[0].size for i in perm[:sm]) != \
        sum(f.cube[0].size for f in frames[:sm])
    _alone_vs_batch(hsc, ctx, [frames[i] for i in perm], [cubes[i] for i in perm],
                    batch_flags=hsc.HSC_BATCH_GRAPH)


def test_batch_frames_against_oracle(hsc, ctx):
    """The 256 uneven snapshot frames (40-64 px square, 125 bands, K = 16,
    7-row window) through one stage-major call with graph capture; a sample
    of frames from both eigensolver waves checked against the FP64 oracle at
    every pixel (the near-tie rule of the end-to-end checks)."""
    import torch
    frames = synth.make_batch(256)
    f0 = frames[0]
    k = f0.model.n_classes
    model = hsc.Model.from_host(f0.model)
    cubes = frames_to_device(frames)
    labs, O, I, P = outputs(frames, k)
    for rep in range(2):  # capture, then replay
        hsc.hsc_classify_batch(ctx, cubes, model, f0.K, f0.window_rows, f0.lam,
                               flags=hsc.HSC_BATCH_GRAPH, labels=labs, out_probs=O, one_bands=I,
                               probs=P)
        ctx.sync()
    n_all = agree_all = ties_all = 0
    for i in (0, 1, 37, 100, 151, 152, 153, 200, 254, 255):
        f = frames[i]
        N = f.cube.shape[1] * f.cube.shape[2]
        n, agree, ties = e2e_check(f, labs[i].cpu().numpy(), O[i].cpu().numpy(),
                                   I[i].cpu().numpy(), P[i].cpu().numpy(), [(0, N)])
        assert agree >= n - ties
        n_all += n
        agree_all += agree
        ties_all += ties
    print("\nbatch frames vs oracle: %d pixels, %d labels agree, %d near-ties"
          % (n_all, agree_all, ties_all))
    assert agree_all >= 0.995 * n_all
