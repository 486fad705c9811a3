"""The 1024 x 1024 x 256 frame (class spectra of two wide Gaussians, sigma
0.01): covariance on the tensor cores (FP16 hi/lo parts, FP32 accumulation in
TMEM, two launches of 128-band halves), the eigenpair refined in double-float,
projection, SVM and KNN in FP32. Each stage's error against the FP64 oracle is
measured, printed (pytest -s) and bounded by the same bars as the FP32 path."""

import numpy as np
import pytest

import oracle
import synth
from parity import check_knn_outputs, knn_ranges

pytestmark = pytest.mark.gpu

ROWS = (0, 511, 512, 1023)  # sampled rows: both edges and the middle


@pytest.fixture(scope="module")
def mixed():
    """The frame and its FP64 oracle PCA: means, covariance (library matmul
    per pixel chunk, same definition as the C two-pass form), Jacobi, the
    signed leading eigenvector and the normalised projection."""
    f = synth.make_config(4)
    B, H, W = f.cube.shape
    mu = oracle.band_means(f.cube)
    C = oracle.covariance_matmul(f.cube, mu)
    ev, V, _, st = oracle.jacobi(C)
    assert st == 0
    v1 = V[:, int(np.argmax(ev))]
    v1 = v1 if v1[int(np.argmax(np.abs(v1)))] > 0 else -v1
    _, I_ref = oracle.project(f.cube, mu, v1)
    return f, mu, C, v1, I_ref.reshape(H, W)


def test_mixed_precision_frame_errors(hsc, ctx, mixed):
    import torch
    f, mu, C, v1, I_ref = mixed
    B, H, W = f.cube.shape
    k = f.model.n_classes
    cube = torch.as_tensor(f.cube, device="cuda")
    model = hsc.Model.from_host(f.model)
    lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
    O = torch.empty((k, H, W), device="cuda")
    I = torch.empty((H, W), device="cuda")
    P = torch.empty((k, H, W), device="cuda")
    hsc.hsc_classify(ctx, cube, model, f.K, f.window_rows, f.lam, labels=lab, out_probs=O,
                     one_band=I, probs=P)
    mu_g, C_g = hsc.hsc_pca_covariance(ctx, cube)
    v_g = torch.zeros(B, dtype=torch.float64, device="cuda")
    hsc.hsc_pca_one_band(ctx, cube, eigvec=v_g)
    ctx.sync()
    lab, O, I, P = (t.cpu().numpy() for t in (lab, O, I, P))
    mu_g, C_g, v_g = mu_g.cpu().numpy(), C_g.cpu().numpy(), v_g.cpu().numpy()

    err = {}
    err["C_rel"] = float(np.abs(C_g - C).max() / np.abs(C).max())
    err["mu"] = float(np.abs(mu_g - mu).max())
    cos = abs(float(v_g @ v1))
    err["v1_angle"] = float(np.sqrt(max(0.0, 1.0 - cos * cos)))
    err["I"] = float(np.abs(I - I_ref).max())

    # SVM and KNN on the sampled rows (and the window rows they read)
    need = sorted({i for r in ROWS for i in range(max(0, r - 7), min(H, r + 7))})
    sub = np.ascontiguousarray(f.cube[:, need, :])
    P_sub = oracle.svm_probs(sub, f.model)[0]
    P_ref = np.zeros((k, H, W))
    P_ref[:, need, :] = P_sub
    err["P"] = float(np.abs(P[:, need, :] - P_sub).max())

    # end to end against the FP64 chain (maps rounded to float32 as stored);
    # the GPU's one-band image differs by dI, which moves each distance by at
    # most 4 dI, so a pixel is a near-tie when d_K+1 - d_K < max(1e-6 d_K+1, 8 dI)
    I32r, P32r = I_ref.astype(np.float32), P_ref.astype(np.float32)
    o_chain, lab_bad, lab_agree, ties, npx = 0.0, 0, 0, 0, 0
    for r in ROWS:
        chain = knn_ranges(I32r, P32r, f.K, f.window_rows, f.lam, [(r * W, (r + 1) * W)])
        tie = (chain["dK1"] - chain["dK"]) < np.maximum(1e-6 * chain["dK1"], 8 * err["I"])
        o_chain = max(o_chain, float(np.abs(O[:, r, ~tie] - chain["O"][:, ~tie]).max(initial=0.0)))
        clear = ~tie & (chain["gapO"] > 2e-4)
        lab_bad += int((lab[r][clear] != chain["labels"][clear]).sum())
        lab_agree += int((lab[r] == chain["labels"]).sum())
        ties += int(tie.sum())
        npx += W
    err["O_end_to_end"] = o_chain
    err["labels_end_to_end_mismatch_outside_ties"] = lab_bad
    err["labels_end_to_end_agreement"] = lab_agree / npx
    err["near_ties"] = ties
    print("\nmixed-precision frame 1024x1024x256 errors vs the FP64 oracle:", err)

    assert err["C_rel"] < 1e-5
    assert err["mu"] < 1e-6
    assert err["v1_angle"] < 1e-5
    assert err["I"] < 2e-5
    assert err["P"] < 1e-4
    assert err["O_end_to_end"] < 1e-4
    assert err["labels_end_to_end_mismatch_outside_ties"] == 0
    assert err["labels_end_to_end_agreement"] > 0.999


def test_fast_path_mixed_frame_rows(hsc, ctx, mixed):
    """The classifier's KNN call (no neighbour-index output) on the oracle's
    normalised one-band image of the 1024 x 1024 frame, K = 40, 14-row
    window, with probability maps independent of the image (O then
    fingerprints each pixel's selected set): 64 rows in four blocks (both
    edges and two inside) against the oracle, every pixel; the pruned walk
    must have finished nearly all pixels itself."""
    import torch
    f, _, _, _, I_ref = mixed
    H, W = I_ref.shape
    I32 = np.ascontiguousarray(I_ref, dtype=np.float32)
    rng = np.random.default_rng(4096)
    P = rng.random((4, H, W))
    P = (P / P.sum(axis=0)).astype(np.float32)
    It = torch.as_tensor(I32, device="cuda")
    Pt = torch.as_tensor(P, device="cuda")
    O = torch.full((4, H, W), -1.0, device="cuda")
    ctx.knn_diagnostics()
    lab = hsc.hsc_knn_filter(ctx, It, Pt, f.K, f.window_rows, f.lam, out_probs=O)
    ctx.sync()
    _, redo = ctx.knn_diagnostics()
    rows = [r for r0 in (0, 300, 700, 1008) for r in range(r0, r0 + 16)]
    ranges = [(r * W, (r + 1) * W) for r in rows]
    st = check_knn_outputs(I32, P, f.K, f.window_rows, f.lam, O.cpu().numpy(),
                           lab.cpu().numpy(), pixels=ranges)
    print("\n1024x1024 map, 64 rows: O max error %.2e; FP64 rule decided %d of %d pixels; "
          "%d of %d pixels handed to the redo pass"
          % (st["o_max_err"], st["fp64_checked"], st["pixels"], redo, H * W))
    assert st["pixels"] == 64 * W
    assert redo <= 0.05 * H * W
