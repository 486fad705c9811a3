"""PCA steps (i)-(ii) on the GPU (tensor-core and FP32-pipe Gram) against the
FP64 oracle, element by element."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# FP32 accumulation of 1024-2048 pixels per partial (relative ~2e-6; frames
# are cut into partials of at least 1024 pixels, at most one per SM pair),
# FP16 hi/lo split of the shifted pixels (~2^-22 per product): 1e-5 of max|C|.
C_TOL = 1e-5
MU_TOL = 1e-6


def check(hsc, ctx, cube, flags):
    import torch
    c = torch.as_tensor(np.ascontiguousarray(cube), device="cuda")
    mu, C = hsc.hsc_pca_covariance(ctx, c, flags=flags)
    ctx.sync()
    mu_ref = oracle.band_means(cube)
    C_ref = oracle.covariance(cube, mu_ref)
    np.testing.assert_allclose(mu.cpu().numpy(), mu_ref, atol=MU_TOL)
    scale = np.abs(C_ref).max()
    err = np.abs(C.cpu().numpy() - C_ref).max() / scale
    assert err < C_TOL, err
    np.testing.assert_array_equal(C.cpu().numpy(), C.cpu().numpy().T)
    return err


@pytest.mark.parametrize("flags", [0, 4])
@pytest.mark.parametrize("shape", [(16, 32, 32), (128, 416, 512), (125, 50, 52), (100, 33, 36),
                                   (37, 9, 13), (128, 7, 9), (1, 12, 12), (200, 20, 20),
                                   (256, 48, 64), (129, 40, 40), (250, 64, 100)])
def test_covariance_against_oracle(hsc, ctx, flags, shape):
    B, H, W = shape
    if shape == (128, 416, 512):
        cube = synth.make_config(2).cube
    else:
        cube = synth.make_frame(B * 7 + H, H, W, B, sigma=0.03).cube
    check(hsc, ctx, cube, flags)


def test_covariance_exact_rank_one(hsc, ctx):
    """Dyadic rank-one cube: C = var(a) u u^T in exact arithmetic; the GPU's
    one-pass FP32 accumulation stays within C_TOL of it."""
    rng = np.random.default_rng(4)
    B, H, W = 96, 40, 44
    u = rng.integers(-4, 5, size=B).astype(np.float64)
    m = rng.integers(8, 24, size=B) / 32.0
    a = rng.integers(-8, 9, size=H * W) / 64.0
    cube = (m[:, None] + u[:, None] * a[None, :]).reshape(B, H, W).astype(np.float32)
    import torch
    mu, C = hsc.hsc_pca_covariance(ctx, torch.as_tensor(cube, device="cuda"))
    ctx.sync()
    ref = np.var(a) * np.outer(u, u)
    assert np.abs(C.cpu().numpy() - ref).max() < C_TOL * np.abs(ref).max()
