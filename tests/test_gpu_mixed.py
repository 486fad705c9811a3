"""The 1024 x 1024 x 256 frame (class spectra of two wide Gaussians, sigma
0.01): covariance on the tensor cores (FP16 hi/lo parts, FP32 accumulation in
TMEM, two launches of 128-band halves), the eigenpair refined in double-float,
projection, SVM and KNN in FP32. Each stage's error against the FP64 oracle is
measured, printed (pytest -s) and bounded by the same bars as the FP32 path."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROWS = (0, 511, 512, 1023)  # sampled rows: both edges and the middle


def test_mixed_precision_frame_errors(hsc, ctx):
    import torch
    f = synth.make_config(4)
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

    # FP64 oracle: steps (i)-(iv)
    mu = oracle.band_means(f.cube)
    C = oracle.covariance_matmul(f.cube, mu)
    ev, V, _, st = oracle.jacobi(C)
    assert st == 0
    v1 = V[:, int(np.argmax(ev))]
    v1 = v1 if v1[int(np.argmax(np.abs(v1)))] > 0 else -v1
    _, I_ref = oracle.project(f.cube, mu, v1)
    I_ref = I_ref.reshape(H, W)

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

    o_own, o_chain, lab_own_bad, lab_chain_bad, npx = 0.0, 0.0, 0, 0, 0
    for r in ROWS:
        p0, p1 = r * W, (r + 1) * W
        # selection on the GPU's own maps, in the kernel's precision (r15)
        own = oracle.knn(I, P, f.K, f.window_rows, f.lam, p0=p0, p1=p1, float_keys=True)
        o_own = max(o_own, float(np.abs(O[:, r, :] - own["O"]).max()))
        clear = own["gapO"] > 2e-5
        lab_own_bad += int((lab[r][clear] != own["labels"][clear]).sum())
        # end to end against the FP64 chain (maps rounded to float32 as stored)
        chain = oracle.knn(I_ref.astype(np.float32), P_ref.astype(np.float32), f.K,
                           f.window_rows, f.lam, p0=p0, p1=p1)
        o_chain = max(o_chain, float(np.abs(O[:, r, :] - chain["O"]).max()))
        lab_chain_bad += int((lab[r] != chain["labels"]).sum())
        npx += W
    err["O_own_maps"] = o_own
    err["O_end_to_end"] = o_chain
    err["labels_own_maps_mismatch"] = lab_own_bad
    err["labels_end_to_end_agreement"] = 1.0 - lab_chain_bad / npx
    print("\nmixed-precision frame 1024x1024x256 errors vs the FP64 oracle:", err)

    assert err["C_rel"] < 1e-5
    assert err["mu"] < 1e-6
    assert err["v1_angle"] < 1e-5
    assert err["I"] < 2e-5
    assert err["P"] < 1e-4
    assert err["O_own_maps"] < 1e-5
    assert err["labels_own_maps_mismatch"] == 0
    assert err["labels_end_to_end_agreement"] > 0.999
