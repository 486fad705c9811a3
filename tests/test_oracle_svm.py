"""Pins of the oracle's SVM stage (Section II.C.1): decision values, Platt
probabilities and the pairwise coupling of the paper's reference [30]."""

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from numpy_ref import couple_numpy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _model(k, w, b, a=-5.0, bp=0.0):
    M = k * (k - 1) // 2
    return synth.SvmModel(n_classes=k, w=np.asarray(w, dtype=np.float32).reshape(M, -1),
                          b=np.asarray(b, dtype=np.float32),
                          platt_a=np.full(M, a, dtype=np.float32),
                          platt_b=np.full(M, bp, dtype=np.float32))


def test_golden_k3_consistent_probabilities():
    g = json.load(open(os.path.join(GOLDEN, "svm_k3_consistent.json")))
    cube = np.asarray(g["x"], dtype=np.float32).reshape(g["B"], 1, 1)
    m = synth.SvmModel(n_classes=g["k"], w=np.asarray(g["w"], dtype=np.float32),
                       b=np.asarray(g["b"], dtype=np.float32),
                       platt_a=np.asarray(g["platt_a"], dtype=np.float32),
                       platt_b=np.asarray(g["platt_b"], dtype=np.float32))
    P, lab, _ = oracle.svm_probs(cube, m)
    np.testing.assert_allclose(P[:, 0, 0], g["p"], atol=g["tol"])
    assert lab[0, 0] == g["label"]


def test_decision_values_match_dot():
    f = synth.make_config(1)
    P, lab, dec = oracle.svm_probs(f.cube, f.model, want_dec=True)
    X = f.cube.reshape(f.cube.shape[0], -1).astype(np.float64)
    ref = f.model.w.astype(np.float64) @ X + f.model.b.astype(np.float64)[:, None]
    np.testing.assert_allclose(dec.reshape(ref.shape), ref, rtol=0, atol=1e-12)


def test_zero_decision_gives_uniform():
    for k in (2, 3, 4, 7):
        M = k * (k - 1) // 2
        cube = np.random.default_rng(k).random((5, 3, 4)).astype(np.float32)
        P, lab, _ = oracle.svm_probs(cube, _model(k, np.zeros((M, 5)), np.zeros(M)))
        np.testing.assert_allclose(P, 1.0 / k, atol=1e-15)
        # the label is the first maximum of the returned probabilities
        np.testing.assert_array_equal(lab, np.argmax(P, axis=0))
        if k == 2:  # exact tie (0.5, 0.5): the smaller class wins
            assert np.all(P[0] == P[1]) and np.all(lab == 0)


def test_two_classes_is_the_binary_probability():
    """k = 2: the coupling returns (r_01, 1 - r_01) exactly."""
    f01 = math.log(3.0) / 5.0  # r = 1/(1+exp(-5 f)) = 0.75
    cube = np.ones((1, 1, 1), dtype=np.float32)
    P, lab, _ = oracle.svm_probs(cube, _model(2, [[0.0]], [f01]))
    r = 1.0 / (1.0 + math.exp(-5.0 * float(np.float32(f01))))
    np.testing.assert_allclose(P[:, 0, 0], [r, 1 - r], atol=1e-15)
    assert P[0, 0, 0] == pytest.approx(0.75, abs=1e-7)


def test_consistent_pairwise_recovers_p_star():
    rng = np.random.default_rng(5)
    for k in (3, 4, 6, 9):
        p = rng.random(k) + 0.05
        p /= p.sum()
        r = p[:, None] / (p[:, None] + p[None, :])
        np.testing.assert_allclose(oracle.couple(r), p, atol=1e-14)


def test_coupling_is_the_constrained_minimiser():
    """KKT: Q p is a multiple of e, sum p = 1, p >= 0, and any feasible move
    raises the objective; also agrees with an independent dense solve."""
    rng = np.random.default_rng(9)
    for k in (2, 3, 4, 5, 8):
        r = rng.uniform(1e-3, 1 - 1e-3, size=(k, k))
        r = np.triu(r, 1)
        r = r + (1 - r.T) * np.tril(np.ones((k, k)), -1)
        np.fill_diagonal(r, 0.0)
        p = oracle.couple(r)
        ref, Q = couple_numpy(r)
        np.testing.assert_allclose(p, ref, atol=1e-13)
        assert p.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.all(p >= 0)
        g = Q @ p
        np.testing.assert_allclose(g, g.mean(), atol=1e-13)

        def obj(x):
            return sum((r[j, i] * x[i] - r[i, j] * x[j]) ** 2
                       for i in range(k) for j in range(k) if i != j)
        for _ in range(5):
            d = rng.standard_normal(k)
            d -= d.mean()
            assert obj(p + 1e-3 * d) > obj(p)


def test_platt_clip():
    """|f| huge: r is clipped to [1e-7, 1-1e-7], the edge of the open interval."""
    cube = np.ones((1, 1, 1), dtype=np.float32)
    P, lab, _ = oracle.svm_probs(cube, _model(2, [[0.0]], [100.0]))
    np.testing.assert_allclose(P[:, 0, 0], [1 - 1e-7, 1e-7], atol=1e-16)


def test_synthetic_frame_is_classified():
    f = synth.make_config(1)
    P, lab, _ = oracle.svm_probs(f.cube, f.model)
    np.testing.assert_allclose(P.sum(axis=0), 1.0, atol=1e-13)
    assert (lab == f.truth).mean() > 0.99
