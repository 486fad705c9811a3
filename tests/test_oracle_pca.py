"""Pins of the oracle's one-band PCA (Section II.C.2 steps (i)-(iv)) against
closed forms, invariants, a hand-worked example and a library eigensolver."""

import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_two_band_hand_example():
    g = json.load(open(os.path.join(GOLDEN, "pca_2band.json")))
    cube = np.asarray(g["cube"], dtype=np.float32)
    out = oracle.pca_one_band(cube)
    np.testing.assert_allclose(out["mu"], g["mu"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(out["C"], g["C"], rtol=0, atol=1e-15)
    assert out["lambda1"] == pytest.approx(g["lambda1"], abs=1e-14)
    assert sorted(out["evals"])[0] == pytest.approx(g["lambda2"], abs=1e-14)
    np.testing.assert_allclose(out["v1"], g["v1"], atol=1e-14)
    np.testing.assert_allclose(out["I_raw"], g["I_raw"], atol=1e-14)
    np.testing.assert_allclose(out["I_norm"], g["I_norm"], atol=1e-14)


def test_band_means_exact_on_integers():
    rng = np.random.default_rng(1)
    cube = rng.integers(0, 100, size=(5, 7, 9)).astype(np.float32)
    mu = oracle.band_means(cube)
    exact = cube.reshape(5, -1).astype(np.int64).sum(axis=1) / 63.0
    np.testing.assert_array_equal(mu, exact)


def _rank_one_cube(B, H, W, seed):
    """x_p = m + a_p u, all values exactly representable in float32, so the
    covariance is exactly var(a) u u^T (a rank-one closed form)."""
    rng = np.random.default_rng(seed)
    u = rng.integers(-4, 5, size=B).astype(np.float64)
    u[np.argmax(np.abs(u))] = 7.0  # unique largest component
    m = rng.integers(8, 24, size=B) / 32.0
    a = rng.integers(-8, 9, size=H * W) / 64.0
    cube = (m[:, None] + u[:, None] * a[None, :]).reshape(B, H, W).astype(np.float32)
    assert np.array_equal(cube.astype(np.float64).reshape(B, -1), m[:, None] + u[:, None] * a[None, :])
    return cube, u, a


@pytest.mark.parametrize("B,H,W", [(3, 4, 5), (16, 8, 8), (40, 6, 11)])
def test_rank_one_closed_form(B, H, W):
    cube, u, a = _rank_one_cube(B, H, W, seed=B)
    out = oracle.pca_one_band(cube)
    v = u / np.linalg.norm(u)  # largest component (7) is positive
    np.testing.assert_allclose(out["v1"], v, atol=1e-12)
    assert out["lambda1"] == pytest.approx(np.var(a) * (u @ u), rel=1e-12)
    # I = a_p * ||u|| - mean, then min-max
    I = (a - a.mean()) * np.linalg.norm(u)
    np.testing.assert_allclose(out["I_raw"].ravel(), I, atol=1e-12)
    In = (I - I.min()) / (I.max() - I.min())
    np.testing.assert_allclose(out["I_norm"].ravel(), In, atol=1e-12)


def test_diagonal_covariance_picks_largest_band():
    """Bands built from distinct zero-mean Walsh rows are uncorrelated, so C is
    diagonal and v1 is the unit vector of the band with the largest variance."""
    n = 64
    Hm = np.array([[1.0]])
    while Hm.shape[0] < n:
        Hm = np.block([[Hm, Hm], [Hm, -Hm]])
    B = 6
    scales = np.array([0.5, 1.0, 0.25, 2.0, 0.75, 1.5])
    cube = (Hm[1:B + 1] * scales[:, None] + 0.5).reshape(B, 8, 8).astype(np.float32)
    out = oracle.pca_one_band(cube)
    np.testing.assert_allclose(out["C"], np.diag(scales ** 2), atol=1e-15)
    e = np.zeros(B)
    e[3] = 1.0
    np.testing.assert_allclose(out["v1"], e, atol=1e-15)
    assert out["lambda1"] == pytest.approx(4.0, abs=1e-15)


def test_flat_cube_gives_zero_one_band():
    cube = np.full((4, 3, 5), 0.25, dtype=np.float32)
    out = oracle.pca_one_band(cube)
    assert np.all(out["I_norm"] == 0.0)


def test_jacobi_against_eigh_and_invariants():
    rng = np.random.default_rng(7)
    for B in (2, 5, 17, 48):
        X = rng.standard_normal((B, 3 * B))
        C = X @ X.T / (3 * B)
        ev, V, nrot, st = oracle.jacobi(C)
        assert st == oracle.OK and nrot > 0
        w, U = np.linalg.eigh(C)
        np.testing.assert_allclose(np.sort(ev), w, rtol=0, atol=1e-12 * w.max())
        np.testing.assert_allclose(V.T @ V, np.eye(B), atol=1e-13)
        D = V.T @ C @ V
        off = D - np.diag(np.diag(D))
        assert np.abs(off).max() <= 1e-12 * np.linalg.norm(C)
        assert np.trace(C) == pytest.approx(ev.sum(), rel=1e-13)
        lead = np.argmax(ev)
        assert abs(abs(V[:, lead] @ U[:, -1]) - 1.0) < 1e-12


def test_jacobi_two_by_two_closed_form():
    a, b, c = 3.0, 1.25, -0.5
    ev, V, nrot, st = oracle.jacobi(np.array([[a, b], [b, c]]))
    m, r = (a + c) / 2, np.hypot((a - c) / 2, b)
    np.testing.assert_allclose(np.sort(ev), [m - r, m + r], atol=1e-14)
    assert nrot == 1  # one rotation zeroes the only off-diagonal pair


def test_jacobi_reports_non_convergence():
    C = np.array([[2.0, 1.0, 0.5], [1.0, 3.0, 0.25], [0.5, 0.25, 1.0]])
    ev, V, nrot, st = oracle.jacobi(C, max_rot=1)
    assert st == oracle.NOT_CONVERGED and nrot == 1


def test_rank_one_plus_noise_davis_kahan():
    """sin(angle(v1, u)) <= ||E||_2 / (s - 2||E||_2) for C = s u u^T + E (Davis-Kahan)."""
    rng = np.random.default_rng(3)
    B, H, W = 24, 30, 30
    u = rng.standard_normal(B)
    u /= np.linalg.norm(u)
    a = rng.standard_normal(H * W)
    noise = 0.05 * rng.standard_normal((B, H * W))
    X = 0.3 + 0.1 * u[:, None] * a[None, :] + noise
    cube = X.reshape(B, H, W).astype(np.float32)
    out = oracle.pca_one_band(cube)
    Xc = cube.reshape(B, -1).astype(np.float64)
    Xc = Xc - Xc.mean(axis=1, keepdims=True)
    S = 0.01 * np.var(a) * np.outer(u, u)
    E = Xc @ Xc.T / (H * W) - S
    e2 = np.linalg.norm(E, 2)
    gap = 0.01 * np.var(a) - 2 * e2
    assert gap > 0
    sin = np.sqrt(max(0.0, 1 - (out["v1"] @ u) ** 2))
    assert sin <= e2 / gap + 1e-12


def test_projection_matches_dot_and_sign_rule():
    rng = np.random.default_rng(11)
    cube = rng.random((9, 7, 6)).astype(np.float32)
    out = oracle.pca_one_band(cube)
    X = cube.reshape(9, -1).astype(np.float64)
    I = out["v1"] @ (X - out["mu"][:, None])
    np.testing.assert_allclose(out["I_raw"].ravel(), I, atol=1e-13)
    big = np.argmax(np.abs(out["v1"]))
    assert out["v1"][big] > 0
    # the normalised image does not depend on the eigenvector's sign
    In = (-I - (-I).min()) / ((-I).max() - (-I).min())
    np.testing.assert_allclose(1.0 - out["I_norm"].ravel(), In, atol=1e-13)


def test_covariance_matmul_equals_two_pass_and_closed_form():
    """The chunked-matmul covariance is the same definition as the C two-pass
    one: equal on random cubes (uneven chunks), and exact on a dyadic rank-one
    cube (C = var(a) u u^T)."""
    rng = np.random.default_rng(11)
    cube = rng.random((23, 17, 19)).astype(np.float32)
    mu = oracle.band_means(cube)
    C2 = oracle.covariance(cube, mu)
    Cm = oracle.covariance_matmul(cube, mu, chunk=37)
    assert np.abs(Cm - C2).max() <= 1e-13 * np.abs(C2).max()
    B, H, W = 12, 16, 16
    u = rng.integers(-4, 5, size=B).astype(np.float64)
    m = rng.integers(8, 24, size=B) / 32.0
    a = rng.integers(-8, 9, size=H * W) / 64.0
    cube = (m[:, None] + u[:, None] * a[None, :]).reshape(B, H, W).astype(np.float32)
    Cm = oracle.covariance_matmul(cube, oracle.band_means(cube), chunk=100)
    np.testing.assert_allclose(Cm, np.var(a) * np.outer(u, u), rtol=0, atol=1e-15)
