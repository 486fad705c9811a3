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

import numpy as np

import oracle

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
        fk = oracle.knn(I, P, K, R, lam, p0, p1, want_nbr=True, float_keys=True)
        d64 = oracle.knn(I, P, K, R, lam, p0, p1, want_nbr=True)
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
