"""Parity helpers: GPU results against the FP64 oracle with the tolerance
masks of the method.

KNN selection is index work decided by floating point, so the GPU and the
oracle take it in the same precision: the kernel forms the float terms of
Eq. 1 (as the paper's float KNN does) and compares their sums exactly; the
oracle's float-key mode does the same, and the neighbour sets must then be
identical at every pixel. The FP64 selection is checked with the task's
near-tie rule.
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def knn_ranges(I, P, K, R, lam, ranges, want_nbr=False, float_keys=False, chunk=2048):
    """oracle.knn over the pixel ranges, split into chunks run on all host
    cores (the oracle's C code runs outside the interpreter lock); the
    chunks' outputs are concatenated in range order."""
    I = np.ascontiguousarray(I, dtype=np.float32)
    P = np.ascontiguousarray(P, dtype=np.float32)
    parts = []
    for p0, p1 in ranges:
        parts += [(a, min(p1, a + chunk)) for a in range(p0, p1, chunk)]

    def one(pr):
        return oracle.knn(I, P, K, R, lam, pr[0], pr[1], want_nbr=want_nbr,
                          float_keys=float_keys)

    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        outs = list(ex.map(one, parts))
    res = {}
    for key in ("labels", "dK", "dK1", "gapO"):
        res[key] = np.concatenate([o[key] for o in outs])
    res["O"] = np.concatenate([o["O"] for o in outs], axis=1)
    res["nbr"] = np.concatenate([o["nbr"] for o in outs]) if want_nbr else None
    return res


def check_knn(I, P, K, R, lam, nbr_gpu, O_gpu, lab_gpu, pixels=None, o_tol=1e-5):
    """Compare GPU KNN outputs (full H x W arrays) with the oracle on
    ``pixels`` (contiguous ranges as (p0, p1) tuples; default: all).

    * neighbour sets: identical to the oracle's selection taken in the
      kernel's precision (float terms, exact comparison), at every pixel;
    * O: within o_tol of the FP64 mean over that set; labels equal where the
      top two O differ by more than 2 o_tol;
    * the task's rule against the FP64-distance selection: labels equal
      except where d_K+1 - d_K < 1e-6 d_K+1 (near-ties) or O nearly ties.
    Returns a dict of counts; raises AssertionError on a violation."""
    I = np.ascontiguousarray(I, dtype=np.float32)
    P = np.ascontiguousarray(P, dtype=np.float32)
    H, W = I.shape
    k = P.shape[0]
    N = H * W
    nbr_gpu = np.asarray(nbr_gpu).reshape(N, K)
    O_gpu = np.asarray(O_gpu).reshape(k, N)
    lab_gpu = np.asarray(lab_gpu).reshape(N)
    if pixels is None:
        pixels = [(0, N)]
    stats = dict(pixels=0, official_near_ties=0, fp64_set_differs=0)
    for p0, p1 in pixels:
        fk = knn_ranges(I, P, K, R, lam, [(p0, p1)], want_nbr=True, float_keys=True)
        d64 = knn_ranges(I, P, K, R, lam, [(p0, p1)], want_nbr=True)
        g = np.sort(nbr_gpu[p0:p1], axis=1)
        ref = np.sort(fk["nbr"][:, :K], axis=1)
        bad = np.nonzero(np.any(g != ref, axis=1))[0]
        assert bad.size == 0, "pixels %s: neighbour set differs from the oracle's" % (
            (bad[:10] + p0).tolist())
        np.testing.assert_allclose(O_gpu[:, p0:p1], fk["O"], atol=o_tol)
        clear = fk["gapO"] > 2 * o_tol
        np.testing.assert_array_equal(lab_gpu[p0:p1][clear], fk["labels"][clear])
        tie = (d64["dK1"] - d64["dK"]) < 1e-6 * d64["dK1"]
        ok = ~tie & (d64["gapO"] > 2 * o_tol)
        np.testing.assert_array_equal(lab_gpu[p0:p1][ok], d64["labels"][ok])
        stats["pixels"] += p1 - p0
        stats["official_near_ties"] += int(tie.sum())
        stats["fp64_set_differs"] += int(np.any(np.sort(d64["nbr"][:, :K], 1) != ref, axis=1).sum())
    return stats


def sample_rows(H, W, rows):
    """Pixel ranges covering whole rows (top, bottom and a few inside)."""
    return [(r * W, (r + 1) * W) for r in rows if 0 <= r < H]


def check_knn_outputs(I, P, K, R, lam, O_gpu, lab_gpu, pixels=None, o_tol=1e-5):
    """The KNN outputs of a call made without neighbour-index output (the
    path the classifier runs: the pruned walk finishes most pixels itself,
    summing probabilities as it decides them) against the oracle on
    ``pixels`` (ranges; default all):

    * O within o_tol of the FP64 mean over the oracle's selection taken in
      the kernel's precision (a different set moves O by the difference of
      two neighbours' probabilities over K);
    * labels equal to that selection's where its top two O differ by more
      than 2 o_tol;
    * labels equal to the FP64-distance selection's outside the task's
      near-ties (d_K+1 - d_K < 1e-6 d_K+1) and O near-ties.
    Returns counts, including ``fp64_checked``: the pixels the FP64 rule
    decided (the rest are its near-ties)."""
    I = np.ascontiguousarray(I, dtype=np.float32)
    P = np.ascontiguousarray(P, dtype=np.float32)
    H, W = I.shape
    k = P.shape[0]
    N = H * W
    O_gpu = np.asarray(O_gpu).reshape(k, N)
    lab_gpu = np.asarray(lab_gpu).reshape(N)
    if pixels is None:
        pixels = [(0, N)]
    idx = np.concatenate([np.arange(p0, p1) for p0, p1 in pixels])
    fk = knn_ranges(I, P, K, R, lam, pixels, float_keys=True)
    d64 = knn_ranges(I, P, K, R, lam, pixels)
    err = np.abs(O_gpu[:, idx] - fk["O"])
    worst = int(np.argmax(err.max(axis=0)))
    assert err.max() <= o_tol, "O differs by %g at pixel %d" % (err.max(), idx[worst])
    clear = fk["gapO"] > 2 * o_tol
    np.testing.assert_array_equal(lab_gpu[idx][clear], fk["labels"][clear])
    tie = (d64["dK1"] - d64["dK"]) < 1e-6 * d64["dK1"]
    ok = ~tie & (d64["gapO"] > 2 * o_tol)
    np.testing.assert_array_equal(lab_gpu[idx][ok], d64["labels"][ok])
    return dict(pixels=int(idx.size), official_near_ties=int(tie.sum()),
                fp64_checked=int(ok.sum()), o_max_err=float(err.max()))


def e2e_check(f, lab, O, I, P, ranges):
    """The oracle's FP64 path from the cube; the GPU's one-band image differs
    by dI, which moves each distance by at most 4 dI (|I_p - I_q| <= 1), so a
    pixel is a near-tie when d_K+1 - d_K < max(1e-6 d_K+1, 8 dI)."""
    ref = oracle.pca_one_band(f.cube)
    Pref, _, _ = oracle.svm_probs(f.cube, f.model)
    dI = float(np.abs(I - ref["I_norm"]).max())
    assert dI < 2e-5
    assert np.abs(P - Pref).max() < 1e-4
    return e2e_labels(f, lab, O, dI, ranges, ref=ref, Pref=Pref)


def e2e_labels(f, lab, O, dI, ranges, ref=None, Pref=None):
    """Labels and O of the whole path (computed from f.cube) against the
    oracle's FP64 chain on the pixel ranges, for outputs whose one-band image
    is within dI of the oracle's (the near-tie margin of e2e_check):
    labels equal where the selection is no near-tie and the top two O differ
    by more than 2e-4, O within 1e-4 outside near-ties. Returns (pixels,
    label agreements, near-ties)."""
    if ref is None:
        ref = oracle.pca_one_band(f.cube)
    if Pref is None:
        Pref = oracle.svm_probs(f.cube, f.model)[0]
    I32 = ref["I_norm"].astype(np.float32)
    P32 = Pref.astype(np.float32)
    n = agree = ties = 0
    for p0, p1 in ranges:
        out = knn_ranges(I32, P32, f.K, f.window_rows, f.lam, [(p0, p1)])
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
