"""hsc_pca_project: projections on several principal components (Section
III.A.2 d with more than one component) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def oracle_pcs(cube, n):
    """The n leading eigenvectors of the oracle's Jacobi (decreasing
    eigenvalue), each signed by the rule (largest |component| positive,
    smaller band on a tie), and the projections."""
    mu = oracle.band_means(cube)
    C = oracle.covariance(cube, mu)
    ev, V, _, st = oracle.jacobi(C)
    assert st == 0
    order = np.argsort(-ev, kind="stable")[:n]
    vecs, projs = [], []
    for j in order:
        v = V[:, j]
        a = np.abs(v)
        i = int(np.flatnonzero(a == a.max())[0])
        v = v if v[i] > 0 else -v
        vecs.append(v)
        projs.append(oracle.project(cube, mu, v)[0].reshape(cube.shape[1:]))
    return ev[order], np.array(vecs), np.array(projs), C


@pytest.mark.parametrize("cfg,n", [(1, 3), (2, 3), ("snap", 3)])
def test_multi_pc_against_oracle(hsc, ctx, cfg, n):
    """Against the GPU's own FP64 covariance: each (v_j, lambda_j) is an
    eigenpair to the residual bound of the one-band PCA, with lambda_j its
    j-th largest eigenvalue. Against the oracle: the same vectors (sign rule
    included) within ||dC|| / gap (the GPU's covariance differs by ~1e-6 of
    |C|), and out_j the projection of the cube on v_j."""
    import torch
    f = synth.make_batch(1)[0] if cfg == "snap" else synth.make_config(cfg)
    B, H, W = f.cube.shape
    cube = torch.as_tensor(f.cube, device="cuda")
    vec = torch.empty((n, B), dtype=torch.float64, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    out = hsc.hsc_pca_project(ctx, cube, n, eigvecs=vec, eigvals=lam)
    _, Cg = hsc.hsc_pca_covariance(ctx, cube)
    ctx.sync()
    out, vec, lam, Cg = out.cpu().numpy(), vec.cpu().numpy(), lam.cpu().numpy(), Cg.cpu().numpy()
    evg = np.sort(np.linalg.eigvalsh(Cg))[::-1]
    ev, V, proj, C = oracle_pcs(f.cube, n)
    mu = oracle.band_means(f.cube)
    xnorm = float(np.sqrt(((f.cube.reshape(B, -1) - mu[:, None]) ** 2).sum(axis=0)).max())
    cn = max(abs(evg[0]), np.abs(np.diag(Cg)).max())
    for j in range(n):
        r = Cg @ vec[j] - lam[j] * vec[j]
        assert np.linalg.norm(r) <= 2e-13 * cn, (j, np.linalg.norm(r) / cn)
        assert abs(lam[j] - evg[j]) <= 1e-12 * cn, j
        assert abs(np.linalg.norm(vec[j]) - 1.0) < 1e-14
        gap = min(abs(ev[j] - ev[j - 1]) if j else np.inf, abs(ev[j] - evg[j + 1]))
        cos = float(vec[j] @ V[j])
        assert cos > 0, j  # the same sign rule
        ang = np.sqrt(max(0.0, 1 - cos * cos))
        assert ang < 2e-6 * cn / gap, (j, gap / cn)
        # the oracle's own projection on its own vector: apart by at most the
        # angle times the largest centred pixel norm, plus FP32 rounding
        pj = proj[j]  # raw I
        tol = 2e-5 * max(1.0, np.abs(pj).max()) + 2 * max(ang, 1e-12) * xnorm
        assert np.abs(out[j] - pj).max() < tol, j


def test_first_component_is_the_one_band_projection(hsc, ctx):
    import torch
    f = synth.make_config(2)
    cube = torch.as_tensor(f.cube, device="cuda")
    out = hsc.hsc_pca_project(ctx, cube, 3)
    I = hsc.hsc_pca_one_band(ctx, cube, flags=0)  # raw projection
    one = hsc.hsc_pca_project(ctx, cube, 1)
    ctx.sync()
    np.testing.assert_array_equal(out[0].cpu().numpy(), I.cpu().numpy())
    np.testing.assert_array_equal(one[0].cpu().numpy(), I.cpu().numpy())


def test_multi_pc_rejects_bad_counts(hsc, ctx):
    import torch
    f = synth.make_config(1)
    cube = torch.as_tensor(f.cube, device="cuda")
    for n in (0, hsc.HSC_MAX_PC + 1):
        with pytest.raises(hsc.HscError):
            hsc.hsc_pca_project(ctx, cube, n, out=torch.empty((1, 32, 32), device="cuda"))


def test_component_inside_the_noise_cluster_reports_not_converged(hsc, ctx):
    """The 416 x 512 x 128 frame has three components above a flat noise floor
    (lambda_4 .. lambda_16 equal to ~1e-7 of lambda_1): a fourth is not defined
    to the residual bound. The call reports HSC_ERR_NOT_CONVERGED, its first
    three components are still the converged ones and every output is finite."""
    import torch
    f = synth.make_config(2)
    B, H, W = f.cube.shape
    cube = torch.as_tensor(f.cube, device="cuda")
    vec = torch.empty((4, B), dtype=torch.float64, device="cuda")
    out = hsc.hsc_pca_project(ctx, cube, 4, eigvecs=vec)
    with pytest.raises(hsc.HscError) as e:
        ctx.sync()
    assert e.value.status == hsc.HSC_ERR_NOT_CONVERGED
    assert np.isfinite(out.cpu().numpy()).all() and np.isfinite(vec.cpu().numpy()).all()
    vec3 = torch.empty((3, B), dtype=torch.float64, device="cuda")
    hsc.hsc_pca_project(ctx, cube, 3, eigvecs=vec3)
    ctx.sync()
    np.testing.assert_array_equal(vec.cpu().numpy()[:3], vec3.cpu().numpy())
