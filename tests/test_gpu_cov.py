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


def test_covariance_raw_counts(hsc, ctx):
    """A cube in raw sensor counts (offset 1000, a band gain in [0.5, 2], values
    up to ~20000): shifted deviations reach ~10^4, beyond FP16 once scaled by a
    fixed factor; the per-band power-of-two scale of the tensor-core path keeps
    the FP16 parts in range."""
    B, H, W = 128, 96, 128
    f = synth.make_frame(31, H, W, B, sigma=0.03).cube.astype(np.float64)
    gain = np.random.default_rng(5).uniform(0.5, 2.0, size=B)[:, None, None]
    cube = (1000.0 + 20000.0 * gain * f).astype(np.float32)
    check(hsc, ctx, cube, 0)


@pytest.mark.parametrize("B,ob", [(64, 5), (200, 5), (200, 170)])
def test_covariance_outlier_outside_pilot_sample(hsc, ctx, B, ob):
    """One pixel ~10^4 times further from its band's mean than any other, at a
    position the pilot sample skips (its runs start at r(N - 256)/15): its
    scaled value leaves FP16's range, so that CTA recomputes its partial on the
    FP32 pipe (B = 200: the one-read 129-256-band kernel, the outlier in either
    half of the bands). Both the outlier band's row and the rest of C match
    the oracle, each against its own scale."""
    import torch
    H, W = 128, 128
    cube = synth.make_frame(77, H, W, B, sigma=0.03).cube.copy()
    p = 700
    cube[ob].flat[p] += np.float32(5e3)
    c = torch.as_tensor(cube, device="cuda")
    mu, C = hsc.hsc_pca_covariance(ctx, c)
    ctx.sync()
    C = C.cpu().numpy()
    mu_ref = oracle.band_means(cube)
    C_ref = oracle.covariance(cube, mu_ref)
    np.testing.assert_allclose(mu.cpu().numpy(), mu_ref, atol=MU_TOL, rtol=1e-7)
    rest = np.ones(B, bool)
    rest[ob] = False
    sub, sub_ref = C[np.ix_(rest, rest)], C_ref[np.ix_(rest, rest)]
    assert np.abs(sub - sub_ref).max() < C_TOL * np.abs(sub_ref).max()
    row, row_ref = C[ob], C_ref[ob]
    assert np.abs(row - row_ref).max() < C_TOL * np.abs(row_ref).max()
