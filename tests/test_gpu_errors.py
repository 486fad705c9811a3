"""Argument validation (synchronous, before any launch) and device-side
status reporting; the context stays usable after every error."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def frame_tensors(hsc):
    import torch
    f = synth.make_config(1)
    return f, torch.as_tensor(f.cube, device="cuda"), hsc.Model.from_host(f.model)


def test_invalid_knn_arguments(hsc, ctx):
    f, c, m = frame_tensors(hsc)
    for K, R, lam in [(0, 5, 1.0), (8, 0, 1.0), (8, 5, -1.0), (8, 5, float("nan")),
                      (97, 5, 1.0)]:
        with pytest.raises(hsc.HscError) as e:
            hsc.hsc_classify(ctx, c, m, K, R, lam)
        assert e.value.status in (hsc.HSC_ERR_INVALID_ARG, hsc.HSC_ERR_UNSUPPORTED)
    # K above the smallest window: R = 1 -> 32 candidates per pixel
    with pytest.raises(hsc.HscError) as e:
        hsc.hsc_classify(ctx, c, m, 33, 1, 1.0)
    assert e.value.status == hsc.HSC_ERR_INVALID_ARG
    hsc.hsc_classify(ctx, c, m, 32, 1, 1.0)
    ctx.sync()


def test_model_band_mismatch(hsc, ctx):
    import torch
    f, c, m = frame_tensors(hsc)
    with pytest.raises(hsc.HscError) as e:
        hsc.hsc_svm_probs(ctx, c[:8].contiguous(), m)
    assert e.value.status == hsc.HSC_ERR_INVALID_ARG


def test_nan_in_cube_is_reported(hsc, ctx):
    import torch
    f, c, m = frame_tensors(hsc)
    bad = c.clone()
    bad[3, 5, 7] = float("nan")
    hsc.hsc_classify(ctx, bad, m, 8, 5, 1.0)
    with pytest.raises(hsc.HscError) as e:
        ctx.sync()
    assert e.value.status == hsc.HSC_ERR_NONFINITE
    hsc.hsc_classify(ctx, c, m, 8, 5, 1.0)  # the context is still usable
    ctx.sync()


def test_scratch_cap_gives_oom(hsc):
    import torch
    f, c, m = frame_tensors(hsc)
    small = hsc.Context(0, scratch_cap_bytes=4096)
    with pytest.raises(hsc.HscError) as e:
        hsc.hsc_classify(small, c, m, 8, 5, 1.0)
    assert e.value.status == hsc.HSC_ERR_OOM
    small.close()


def test_reserve_then_classify_keeps_scratch(hsc):
    import torch
    f, c, m = frame_tensors(hsc)
    cx = hsc.Context(0)
    cx.reserve(16, 32, 32, 4)
    before = cx.scratch_bytes
    hsc.hsc_classify(cx, c, m, 8, 5, 1.0)
    cx.sync()
    assert cx.scratch_bytes == before > 0
    cx.close()


def test_torch_stream(hsc):
    import torch
    f, c, m = frame_tensors(hsc)
    s = torch.cuda.Stream()
    cx = hsc.Context(0, stream=s)
    with torch.cuda.stream(s):
        lab = hsc.hsc_classify(cx, c, m, 8, 5, 1.0)
    cx.sync()
    cx.set_stream(None)
    lab2 = hsc.hsc_classify(cx, c, m, 8, 5, 1.0)
    cx.sync()
    np.testing.assert_array_equal(lab.cpu().numpy(), lab2.cpu().numpy())
    cx.close()
