"""End-to-end classification (Fig. 2) on the GPU through hsc_classify against
the FP64 oracle run on the same cube."""

import numpy as np
import pytest

import oracle
import synth
from parity import sample_rows

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


def e2e_check(f, lab, O, I, P, ranges):
    """The oracle's FP64 path from the cube; the GPU's one-band image differs
    by dI, which moves each distance by at most 4 dI (|I_p - I_q| <= 1), so a
    pixel is a near-tie when d_K+1 - d_K < max(1e-6 d_K+1, 8 dI)."""
    ref = oracle.pca_one_band(f.cube)
    Pref, _, _ = oracle.svm_probs(f.cube, f.model)
    dI = float(np.abs(I - ref["I_norm"]).max())
    assert dI < 2e-5
    assert np.abs(P - Pref).max() < 1e-4
    I32 = ref["I_norm"].astype(np.float32)
    P32 = Pref.astype(np.float32)
    H, W = I.shape
    n = agree = ties = 0
    for p0, p1 in ranges:
        out = oracle.knn(I32, P32, f.K, f.window_rows, f.lam, p0, p1)
        gap = out["dK1"] - out["dK"]
        tie = gap < np.maximum(1e-6 * out["dK1"], 8 * dI)
        labg = lab.reshape(-1)[p0:p1]
        Og = O.reshape(O.shape[0], -1)[:, p0:p1]
        clear = ~tie & (out["gapO"] > 2e-4)
        np.testing.assert_array_equal(labg[clear], out["labels"][clear])
        assert np.abs(Og[:, ~tie] - out["O"][:, ~tie]).max(initial=0.0) < 1e-4
        n += p1 - p0
        ties += int(tie.sum())
        agree += int((labg == out["labels"]).sum())
    return n, agree, ties


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
    (no min-max). one_band is that I, and labels and O equal the oracle's KNN
    on the same map (selection on the float terms of Eq. 1, as the kernels)."""
    f = synth.make_config(1)
    lab, O, I, P = gpu_classify(hsc, ctx, f, flags=hsc.HSC_CLASSIFY_RAW_I)
    ref = oracle.pca_one_band(f.cube)
    assert np.abs(I - ref["I_raw"]).max() < 2e-5 * max(1.0, np.abs(ref["I_raw"]).max())
    k = f.model.n_classes
    out = oracle.knn(I, P, f.K, f.window_rows, f.lam, 0, I.size, float_keys=True)
    clear = out["gapO"] > 2e-5
    np.testing.assert_array_equal(lab.reshape(-1)[clear], out["labels"][clear])
    assert np.abs(O.reshape(k, -1) - out["O"]).max() < 1e-5
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
