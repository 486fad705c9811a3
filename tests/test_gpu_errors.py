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
    torch.cuda.synchronize()
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


@pytest.mark.parametrize("shape", [(16, 32, 32), (128, 96, 128), (200, 40, 48)])
def test_gram_wait_timeout_is_reported(hsc, shape):
    """The device-side timeout path: the tensor-core Gram told to issue no
    loads gives up its first bounded wait (no copy or MMA in flight), flags
    the status and frees its tensor memory; hsc_sync returns HSC_ERR_TIMEOUT
    and the same context then classifies the frame as a fresh one does."""
    import torch
    B, H, W = shape
    f = synth.make_frame(B + H, H, W, B, sigma=0.02, K=8, window_rows=5)
    c = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    fresh = hsc.Context(0)
    ref = hsc.hsc_classify(fresh, c, m, 8, 5, 1.0)
    fresh.sync()
    cx = hsc.Context(0)
    cx.test_stall_next_gram()
    hsc.hsc_classify(cx, c, m, 8, 5, 1.0)
    with pytest.raises(hsc.HscError) as e:
        cx.sync()
    assert e.value.status == hsc.HSC_ERR_TIMEOUT
    lab = hsc.hsc_classify(cx, c, m, 8, 5, 1.0)  # the knob applied to one call only
    cx.sync()
    np.testing.assert_array_equal(lab.cpu().numpy(), ref.cpu().numpy())
    # the covariance entry point takes the same path
    cx.test_stall_next_gram()
    hsc.hsc_pca_covariance(cx, c)
    with pytest.raises(hsc.HscError) as e:
        cx.sync()
    assert e.value.status == hsc.HSC_ERR_TIMEOUT
    mu, C = hsc.hsc_pca_covariance(cx, c)
    mu2, C2 = hsc.hsc_pca_covariance(fresh, c)
    cx.sync()
    fresh.sync()
    np.testing.assert_array_equal(C.cpu().numpy(), C2.cpu().numpy())
    cx.close()
    fresh.close()


def test_fused_batch_wait_timeout_is_reported(hsc):
    """The fused batch kernel's bounded wait (HSC_BATCH_FUSED): with the first
    frame's projection/SVM item count raised by one in the uploaded table, that
    frame is never complete, so its KNN row segments give up their waits after
    the bound and flag the status; hsc_sync returns HSC_ERR_TIMEOUT and the
    same context's next fused batch equals the frames classified alone."""
    import torch
    frames = synth.make_batch(4, seed=790)
    f0 = frames[0]
    model = hsc.Model.from_host(f0.model)
    cubes = [torch.as_tensor(f.cube, device="cuda") for f in frames]
    labs = [torch.full(f.cube.shape[1:], -1, dtype=torch.int32, device="cuda") for f in frames]
    cx = hsc.Context(0)
    cx.test_stall_next_batch_wait()
    hsc.hsc_classify_batch(cx, cubes, model, f0.K, f0.window_rows, f0.lam,
                           flags=hsc.HSC_BATCH_FUSED, labels=labs)
    with pytest.raises(hsc.HscError) as e:
        cx.sync()
    assert e.value.status == hsc.HSC_ERR_TIMEOUT
    hsc.hsc_classify_batch(cx, cubes, model, f0.K, f0.window_rows, f0.lam,
                           flags=hsc.HSC_BATCH_FUSED, labels=labs)
    cx.sync()
    for f, c, lab in zip(frames, cubes, labs):
        ref = hsc.hsc_classify(cx, c, model, f.K, f.window_rows, f.lam)
        cx.sync()
        np.testing.assert_array_equal(lab.cpu().numpy(), ref.cpu().numpy())
    cx.close()
