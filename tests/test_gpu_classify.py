"""End-to-end classification (Fig. 2) on the GPU through hsc_classify against
the FP64 oracle run on the same cube."""

import numpy as np
import pytest

import oracle
import synth
from parity import e2e_check, sample_rows

pytestmark = pytest.mark.gpu


def gpu_classify(hsc, ctx, f, flags=0):
    import torch
    B, H, W = f.cube.shape
    k = f.model.n_classes
    c = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    I = torch.empty((H, W), dtype=torch.float32, device="cuda")
    P = torch.empty((k, H, W), dtype=torch.float32, device="cuda")
    O = torch.empty((k, H, W), dtype=torch.float32, device="cuda")
    lab = hsc.hsc_classify(ctx, c, m, f.K, f.window_rows, f.lam, flags=flags, out_probs=O,
                           one_band=I, probs=P)
    ctx.sync()
    return lab.cpu().numpy(), O.cpu().numpy(), I.cpu().numpy(), P.cpu().numpy()


def test_tiny_frame_all_pixels(hsc, ctx):
    f = synth.make_config(1)
    lab, O, I, P = gpu_classify(hsc, ctx, f)
    n, agree, ties = e2e_check(f, lab, O, I, P, [(0, 32 * 32)])
    assert agree >= n - ties


def test_neuro_frame_sampled_rows(hsc, ctx):
    f = synth.make_config(2)
    lab, O, I, P = gpu_classify(hsc, ctx, f)
    H, W = lab.shape
    n, agree, ties = e2e_check(f, lab, O, I, P, sample_rows(H, W, [0, 3, 100, 207, 330, 415]))
    assert agree >= 0.999 * n
    # the filter smooths the SVM map: labels follow the synthetic regions
    assert (lab == f.truth).mean() > 0.99


def test_classify_matches_stagewise_calls(hsc, ctx):
    """hsc_classify equals hsc_pca_one_band + hsc_svm_probs + hsc_knn_filter."""
    import torch
    f = synth.make_config(1)
    lab, O, I, P = gpu_classify(hsc, ctx, f)
    c = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    I2 = hsc.hsc_pca_one_band(ctx, c)
    P2 = hsc.hsc_svm_probs(ctx, c, m)
    O2 = torch.empty_like(P2)
    lab2 = hsc.hsc_knn_filter(ctx, I2, P2, f.K, f.window_rows, f.lam, out_probs=O2)
    ctx.sync()
    np.testing.assert_array_equal(I2.cpu().numpy(), I)
    np.testing.assert_array_equal(P2.cpu().numpy(), P)
    np.testing.assert_array_equal(O2.cpu().numpy(), O)
    np.testing.assert_array_equal(lab2.cpu().numpy(), lab)


def test_classify_without_optional_outputs(hsc, ctx):
    import torch
    f = synth.make_config(1)
    lab_ref, _, _, _ = gpu_classify(hsc, ctx, f)
    c = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    lab = hsc.hsc_classify(ctx, c, m, f.K, f.window_rows, f.lam)
    ctx.sync()
    np.testing.assert_array_equal(lab.cpu().numpy(), lab_ref)


def test_classify_on_raw_one_band(hsc, ctx):
    """Method variant HSC_CLASSIFY_RAW_I: the KNN runs on the raw projection I
    (no min-max). one_band is that I; labels and O equal the oracle's chain
    on its own raw projection and probabilities outside near-ties (the GPU's
    I differs by dI, which moves a distance by at most 4 dI (range + dI)),
    and equal, bit for bit, hsc_knn_filter on the GPU's own maps."""
    import torch
    f = synth.make_config(1)
    lab, O, I, P = gpu_classify(hsc, ctx, f, flags=hsc.HSC_CLASSIFY_RAW_I)
    ref = oracle.pca_one_band(f.cube)
    Pref = oracle.svm_probs(f.cube, f.model)[0]
    I_raw = ref["I_raw"]
    dI = float(np.abs(I - I_raw).max())
    assert dI < 2e-5 * max(1.0, np.abs(I_raw).max())
    assert np.abs(P - Pref).max() < 1e-4
    k = f.model.n_classes
    out = oracle.knn(I_raw.astype(np.float32), Pref.astype(np.float32), f.K, f.window_rows,
                     f.lam, 0, I.size)
    rng_I = float(I_raw.max() - I_raw.min())
    tie = (out["dK1"] - out["dK"]) < np.maximum(1e-6 * out["dK1"], 8 * dI * (rng_I + dI))
    clear = ~tie & (out["gapO"] > 2e-4)
    np.testing.assert_array_equal(lab.reshape(-1)[clear], out["labels"][clear])
    assert np.abs(O.reshape(k, -1)[:, ~tie] - out["O"][:, ~tie]).max(initial=0.0) < 1e-4
    assert tie.mean() < 0.5
    # the same KNN call on the GPU's own maps gives the same outputs
    O2 = torch.empty((k,) + I.shape, device="cuda")
    lab2 = hsc.hsc_knn_filter(ctx, torch.as_tensor(I, device="cuda"),
                              torch.as_tensor(P, device="cuda"), f.K, f.window_rows, f.lam,
                              out_probs=O2)
    ctx.sync()
    np.testing.assert_array_equal(lab2.cpu().numpy(), lab)
    np.testing.assert_array_equal(O2.cpu().numpy(), O)
    # and it differs from the normalised form (the map's scale enters Eq. 1)
    lab_n, _, I_n, _ = gpu_classify(hsc, ctx, f)
    assert not np.allclose(I, I_n)


def test_bip_cube_equals_band_sequential(hsc, ctx):
    """Method variant HSC_CUBE_BIP: the same frame stored pixel-interleaved
    (H x W x B) gives results identical, bit for bit, to the band-sequential
    call (the cube is transposed on the device, then the same kernels run);
    the PCA entry point likewise. Ragged sizes (not multiples of the 32 x 32
    transpose tile)."""
    import torch
    f = synth.make_frame(11, 45, 37, 70, sigma=0.02)
    B, H, W = f.cube.shape
    k = f.model.n_classes
    m = hsc.Model.from_host(f.model)
    bsq = torch.as_tensor(f.cube, device="cuda")
    bip = torch.as_tensor(np.ascontiguousarray(np.transpose(f.cube, (1, 2, 0))), device="cuda")
    outs = []
    for cube, flags in ((bsq, 0), (bip, hsc.HSC_CUBE_BIP)):
        I = torch.empty((H, W), device="cuda")
        O = torch.empty((k, H, W), device="cuda")
        lab = hsc.hsc_classify(ctx, cube, m, f.K, f.window_rows, f.lam, flags=flags, out_probs=O,
                               one_band=I)
        I2 = hsc.hsc_pca_one_band(ctx, cube, flags=hsc.HSC_PCA_MINMAX | flags)
        ctx.sync()
        outs.append([t.cpu().numpy() for t in (lab, O, I, I2)])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
