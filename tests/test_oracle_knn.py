"""Pins of the oracle's KNN filter (Section II.C.3, Eq. 1 and Eq. 2, row window
of Section III.A.3): hand-worked examples, special cases with closed forms,
symmetries, and an independent NumPy brute force on tiny images."""

import json
import os

import numpy as np
import pytest

import oracle
from numpy_ref import knn_bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name", ["knn_line5.json", "knn_window_ties.json"])
def test_golden_hand_examples(name):
    g = json.load(open(os.path.join(GOLDEN, name)))
    I = np.asarray(g["I"], dtype=np.float32)
    P = np.asarray(g["P"], dtype=np.float32)
    out = oracle.knn(I, P, g["K"], g["R"], g["lambda"], want_nbr=True)
    K = g["K"]
    np.testing.assert_array_equal(out["nbr"][:, :K], g["nbr"])
    np.testing.assert_allclose(out["O"].reshape(P.shape), g["O"], atol=1e-7)
    np.testing.assert_array_equal(out["labels"].reshape(I.shape), g["labels"])
    if "dK" in g:
        np.testing.assert_array_equal(out["dK"], g["dK"])
        np.testing.assert_array_equal(out["dK1"], g["dK1"])


def _rand(H, W, k, seed):
    rng = np.random.default_rng(seed)
    I = rng.random((H, W)).astype(np.float32)
    P = rng.random((k, H, W))
    P = (P / P.sum(axis=0)).astype(np.float32)
    return I, P


def test_k1_window1_returns_own_probabilities():
    I, P = _rand(9, 13, 4, 1)
    out = oracle.knn(I, P, K=1, R=1, lam=1.0)
    np.testing.assert_array_equal(out["O"].reshape(P.shape), P.astype(np.float64))
    np.testing.assert_array_equal(out["labels"].reshape(I.shape), np.argmax(P, axis=0))


def test_lambda0_constant_image_takes_smallest_indices():
    H, W, R, K = 7, 5, 3, 6
    I = np.full((H, W), 0.5, dtype=np.float32)
    _, P = _rand(H, W, 3, 2)
    out = oracle.knn(I, P, K, R, 0.0, want_nbr=True)
    for p in range(H * W):
        r = p // W
        lo = max(0, r - R // 2)
        np.testing.assert_array_equal(out["nbr"][p, :K], lo * W + np.arange(K))


def test_constant_probabilities_pass_through():
    I, _ = _rand(8, 8, 3, 3)
    P = np.tile(np.array([0.2, 0.5, 0.3], dtype=np.float32)[:, None, None], (1, 8, 8))
    out = oracle.knn(I, P, K=5, R=3, lam=1.0)
    np.testing.assert_allclose(out["O"].reshape(P.shape), P, atol=1e-15)


def test_rows_of_O_sum_to_one():
    I, P = _rand(10, 12, 5, 4)
    out = oracle.knn(I, P, K=7, R=4, lam=1.0)
    np.testing.assert_allclose(out["O"].sum(axis=0), 1.0, atol=1e-6)


def test_whole_window_is_a_box_filter():
    """H <= ceil(R/2): every pixel's window is the whole image, so K = H*W
    averages all of P."""
    H, W = 3, 7
    I, P = _rand(H, W, 4, 5)
    out = oracle.knn(I, P, K=H * W, R=6, lam=1.0)
    mean = P.astype(np.float64).reshape(4, -1).mean(axis=1)
    np.testing.assert_allclose(out["O"], np.repeat(mean[:, None], H * W, axis=1), atol=1e-15)


@pytest.mark.parametrize("H,W,K,R,lam", [(16, 16, 8, 5, 1.0), (12, 9, 3, 14, 1.0),
                                          (10, 10, 20, 4, 0.3), (7, 11, 1, 1, 2.0),
                                          (9, 8, 5, 3, 0.0)])
def test_bruteforce_numpy_agrees(H, W, K, R, lam):
    I, P = _rand(H, W, 4, H * W + K)
    out = oracle.knn(I, P, K, R, lam, want_nbr=True)
    O, lab, nbr = knn_bruteforce(I, P, K, R, lam)
    np.testing.assert_array_equal(out["nbr"][:, :K], nbr)
    np.testing.assert_allclose(out["O"].reshape(O.shape), O, atol=1e-15)
    np.testing.assert_array_equal(out["labels"].reshape(lab.shape), lab)


def test_reflection_of_image_is_invisible():
    """I -> 1 - I keeps every |I_p - I_q| (exact on a dyadic grid)."""
    rng = np.random.default_rng(6)
    I = (rng.integers(0, 1024, size=(12, 10)) / 1024.0).astype(np.float32)
    _, P = _rand(12, 10, 3, 7)
    a = oracle.knn(I, P, 6, 5, 1.0, want_nbr=True)
    b = oracle.knn((1.0 - I).astype(np.float32), P, 6, 5, 1.0, want_nbr=True)
    np.testing.assert_array_equal(a["nbr"], b["nbr"])
    np.testing.assert_array_equal(a["O"], b["O"])


def test_column_mirror_mirrors_the_result():
    """Reversing the columns reverses the output when no distances tie (pins
    the (c - j) column term and the column indexing)."""
    I, P = _rand(9, 14, 3, 8)
    a = oracle.knn(I, P, 7, 5, 1.0)
    b = oracle.knn(np.ascontiguousarray(I[:, ::-1]), np.ascontiguousarray(P[:, :, ::-1]), 7, 5, 1.0)
    np.testing.assert_allclose(a["O"].reshape(3, 9, 14)[:, :, ::-1], b["O"].reshape(3, 9, 14),
                               atol=1e-15)


def test_distance_bookkeeping():
    I, P = _rand(11, 9, 2, 9)
    K, R = 4, 5
    out = oracle.knn(I, P, K, R, 1.0, want_nbr=True)
    I64 = I.astype(np.float64)
    W = 9
    for p in range(0, 99, 7):
        r, c = divmod(p, W)
        q = out["nbr"][p]
        d = (I64[r, c] - I64.ravel()[q]) ** 2 + (r - q // W) ** 2 + (c - q % W) ** 2
        assert np.all(np.diff(d) >= 0)
        assert out["dK"][p] == d[K - 1] and out["dK1"][p] == d[K]


def test_rejects_k_above_candidates():
    I, P = _rand(4, 3, 2, 10)
    assert oracle.knn_min_candidates(4, 3, 4) == 6  # rows r..r+1 at the top
    with pytest.raises(oracle.OracleError):
        oracle.knn(I, P, 7, 4, 1.0)
    oracle.knn(I, P, 6, 4, 1.0)


def test_float_keys_equal_fp64_on_exact_inputs():
    """Dyadic grey levels and lambda = 1: every float term is exact, so the
    float-key selection is the FP64 selection, ties included."""
    rng = np.random.default_rng(12)
    I = (rng.integers(0, 64, size=(14, 23)) / 64.0).astype(np.float32)
    _, P = _rand(14, 23, 3, 13)
    a = oracle.knn(I, P, 11, 6, 1.0, want_nbr=True)
    b = oracle.knn(I, P, 11, 6, 1.0, want_nbr=True, float_keys=True)
    np.testing.assert_array_equal(a["nbr"], b["nbr"])
    np.testing.assert_array_equal(a["O"], b["O"])


@pytest.mark.parametrize("lam", [1.0, 0.3, 1.7])
def test_float_keys_against_numpy_float32(lam):
    from numpy_ref import knn_float_keys_bruteforce
    I, P = _rand(11, 17, 3, 14)
    out = oracle.knn(I, P, 9, 5, lam, want_nbr=True, float_keys=True)
    np.testing.assert_array_equal(out["nbr"][:, :9], knn_float_keys_bruteforce(I, P, 9, 5, lam))


def test_float_keys_differ_from_fp64_only_inside_rounding():
    """The float terms carry at most 3 ulp (e) and 2 ulp (s) of error, so
    the two selections can only disagree where the FP64 K-th and (K+1)-th
    distances are that close."""
    I, P = _rand(20, 60, 3, 15)
    I = (I * np.float32(1e-2)).astype(np.float32)  # small contrasts: many close keys
    K, R, lam = 12, 7, 0.7
    a = oracle.knn(I, P, K, R, lam, want_nbr=True)
    b = oracle.knn(I, P, K, R, lam, want_nbr=True, float_keys=True)
    u = 2.0 ** -24
    diff = np.any(np.sort(a["nbr"][:, :K], 1) != np.sort(b["nbr"][:, :K], 1), axis=1)
    bound = 2 * (3 * u * 1e-4 + 2 * u * lam * lam * 2 * (3 ** 2 + 59 ** 2))
    assert np.all((a["dK1"] - a["dK"])[diff] <= bound)
