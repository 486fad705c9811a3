"""Independent NumPy restatements used to cross-check the C oracle on tiny
inputs (a second implementation of the same definitions: the pins catch a
mistake that only one of the two makes).
"""

import numpy as np


def window_rows(r: int, H: int, R: int):
    """Rows r - floor(R/2) .. r + ceil(R/2) - 1, truncated to the image."""
    lo = max(0, r - R // 2)
    hi = min(H - 1, r + (R + 1) // 2 - 1)
    return lo, hi


def knn_bruteforce(I, P, K, R, lam):
    """Eq. 1 / Eq. 2 via np.lexsort over every pixel's window candidates.

    Returns (O[k,H,W], labels[H,W], nbr[H*W, K]).
    """
    I = np.asarray(I, dtype=np.float32).astype(np.float64)
    P = np.asarray(P, dtype=np.float32).astype(np.float64)
    H, W = I.shape
    k = P.shape[0]
    O = np.zeros((k, H, W))
    nbr = np.zeros((H * W, K), dtype=np.int64)
    for r in range(H):
        lo, hi = window_rows(r, H, R)
        ii, jj = np.meshgrid(np.arange(lo, hi + 1), np.arange(W), indexing="ij")
        ii = ii.ravel()
        jj = jj.ravel()
        q = ii * W + jj
        for c in range(W):
            d = (I[r, c] - I[ii, jj]) ** 2 + lam * lam * ((r - ii) ** 2 + (c - jj) ** 2)
            order = np.lexsort((q, d))[:K]
            sel = q[order]
            nbr[r * W + c] = sel
            O[:, r, c] = P.reshape(k, -1)[:, sel].mean(axis=1)
    labels = np.argmax(O, axis=0)
    return O, labels, nbr


def couple_numpy(r):
    """Exact minimiser of the second coupling method via numpy.linalg.solve."""
    r = np.asarray(r, dtype=np.float64)
    k = r.shape[0]
    Q = np.zeros((k, k))
    for i in range(k):
        for j in range(k):
            if i != j:
                Q[i, i] += r[j, i] ** 2
                Q[i, j] = -r[j, i] * r[i, j]
    # optimality system of min p^T Q p s.t. sum p = 1 (Q is only PSD)
    M = np.zeros((k + 1, k + 1))
    M[:k, :k] = Q
    M[:k, k] = 1.0
    M[k, :k] = 1.0
    rhs = np.zeros(k + 1)
    rhs[k] = 1.0
    x = np.linalg.solve(M, rhs)
    return x[:k], Q


def knn_float_keys_bruteforce(I, P, K, R, lam):
    """Eq. 1 with float terms evaluated by numpy float32 arithmetic
    (round-to-nearest): dI = I_p - I_q, e = dI*dI, s = fl(lam^2)*(dr^2+dc^2),
    summed exactly with a float32 two-sum; candidates ordered by (hi, lo, q).
    Returns nbr[H*W, K]."""
    I = np.asarray(I, dtype=np.float32)
    H, W = I.shape
    f = np.float32
    lam32 = f(lam)
    l2 = f(lam32 * lam32)
    nbr = np.zeros((H * W, K), dtype=np.int64)
    for r in range(H):
        lo_r, hi_r = window_rows(r, H, R)
        ii, jj = np.meshgrid(np.arange(lo_r, hi_r + 1), np.arange(W), indexing="ij")
        ii = ii.ravel()
        jj = jj.ravel()
        q = ii * W + jj
        Iq = I[ii, jj]
        for c in range(W):
            dI = (I[r, c] - Iq).astype(np.float32)
            e = (dI * dI).astype(np.float32)
            s = (l2 * ((r - ii) ** 2 + (c - jj) ** 2).astype(np.float32)).astype(np.float32)
            h = (s + e).astype(np.float32)
            bb = (h - s).astype(np.float32)
            low = ((s - (h - bb)) + (e - bb)).astype(np.float32)
            order = np.lexsort((q, low, h))[:K]
            nbr[r * W + c] = q[order]
    return nbr
