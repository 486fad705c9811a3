"""hsc_autotune / hsc_set_tuning: the tuned launch parameters (Gram staging
depth, projection/SVM pixels per thread and CTAs per SM, the pruned KNN
walk's pixels per CTA and undecided-key buffer) change speed only: every
candidate gives outputs identical bit for bit to the defaults."""

import itertools

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def classify(hsc, ctx, f, cube, m):
    import torch
    B, H, W = f.cube.shape
    k = f.model.n_classes
    I = torch.empty((H, W), device="cuda")
    P = torch.empty((k, H, W), device="cuda")
    O = torch.empty((k, H, W), device="cuda")
    lab = hsc.hsc_classify(ctx, cube, m, f.K, f.window_rows, f.lam, out_probs=O, one_band=I,
                           probs=P)
    ctx.sync()
    return [t.cpu().numpy() for t in (lab, O, I, P)]


@pytest.mark.parametrize("shape", [(128, 64, 96), (125, 37, 41)])
def test_every_candidate_gives_identical_outputs(hsc, ctx, shape):
    import torch
    B, H, W = shape
    f = synth.make_frame(B + H, H, W, B, sigma=0.02)
    cube = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    k = f.model.n_classes
    ctx.set_tuning(B, H, W, k, None)
    ref = classify(hsc, ctx, f, cube, m)
    for stg, px, bps, kv in itertools.product((3, 4), (1, 4), (2, 16), (0, 1, 2, 3, 4, 5)):
        ctx.set_tuning(B, H, W, k, (stg, px, bps, kv))
        out = classify(hsc, ctx, f, cube, m)
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b)
    ctx.set_tuning(B, H, W, k, None)


def test_autotune_picks_a_candidate_and_keeps_results(hsc, ctx):
    import torch
    f = synth.make_config(2)
    cube = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    B, H, W = f.cube.shape
    ctx.set_tuning(B, H, W, f.model.n_classes, None)
    ref = classify(hsc, ctx, f, cube, m)
    cfg = ctx.autotune(cube, m, f.K, f.window_rows, f.lam)
    assert cfg["gram_stages"] in (3, 4)
    assert cfg["svm_px"] in (1, 4) and cfg["svm_blocks_per_sm"] in (2, 4, 8, 16)
    assert cfg["knn_variant"] in (0, 1, 2, 3, 4, 5)
    out = classify(hsc, ctx, f, cube, m)
    for a, b in zip(ref, out):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(hsc.HscError):
        ctx.set_tuning(B, H, W, f.model.n_classes, (5, 1, 2))
    with pytest.raises(hsc.HscError):
        ctx.set_tuning(B, H, W, f.model.n_classes, (3, 1, 2, 6))
    ctx.set_tuning(B, H, W, f.model.n_classes, None)


@pytest.mark.parametrize("lam", [1.0, 0.5])
def test_walk_variants_and_searches_give_identical_outputs(hsc, ctx, lam):
    """Every walk variant, every search, with and without neighbour-index
    output: the same O and labels bit for bit on the 416 x 512 maps (the
    pixels the redo pass completes differ between them; the canonical
    summation order makes that invisible)."""
    import torch
    f = synth.make_config(2)
    B, H, W = f.cube.shape
    k = f.model.n_classes
    cube = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    I = torch.empty((H, W), device="cuda")
    P = torch.empty((k, H, W), device="cuda")
    ref_lab, ref_O = None, None
    for kv in range(6):  # 4 and 5: the window tile staged by TMA
        ctx.set_tuning(B, H, W, k, (0, 0, 0, kv))
        O = torch.empty((k, H, W), device="cuda")
        lab = hsc.hsc_classify(ctx, cube, m, f.K, f.window_rows, lam, out_probs=O, one_band=I,
                               probs=P)
        ctx.sync()
        if ref_lab is None:
            ref_lab, ref_O = lab.cpu().numpy(), O.cpu().numpy()
        else:
            np.testing.assert_array_equal(lab.cpu().numpy(), ref_lab)
            np.testing.assert_array_equal(O.cpu().numpy(), ref_O)
    ctx.set_tuning(B, H, W, k, None)
    for search in (hsc.HSC_KNN_SEARCH_FULL, hsc.HSC_KNN_SEARCH_PRUNED, hsc.HSC_KNN_SEARCH_HEAP):
        for with_nbr in (False, True):
            O = torch.empty((k, H, W), device="cuda")
            nbr = torch.empty((H, W, f.K), dtype=torch.int32, device="cuda") if with_nbr else None
            lab = hsc.hsc_knn_filter(ctx, I, P, f.K, f.window_rows, lam, out_probs=O,
                                     nbr_idx=nbr, search=search)
            ctx.sync()
            np.testing.assert_array_equal(lab.cpu().numpy(), ref_lab)
            np.testing.assert_array_equal(O.cpu().numpy(), ref_O)
