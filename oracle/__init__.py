"""ctypes front end of the FP64 CPU oracle (``hsc_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA library never
imports, links or calls anything here.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, INVALID, NOT_CONVERGED = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc -O2 (no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int)
        i64p = ctypes.POINTER(ctypes.c_long)
        c_int, c_long, c_double = ctypes.c_int, ctypes.c_long, ctypes.c_double
        lib.oracle_band_means.argtypes = [f32p, c_int, c_long, f64p]
        lib.oracle_covariance.argtypes = [f32p, c_int, c_long, f64p, f64p]
        lib.oracle_jacobi.argtypes = [f64p, c_int, c_double, c_long, f64p, f64p, i64p]
        lib.oracle_pca_one_band.argtypes = [f32p, c_int, c_int, c_int, c_double,
                                            f64p, f64p, f64p, f64p, f64p, f64p,
                                            f64p, f64p, i64p]
        lib.oracle_project.argtypes = [f32p, c_int, c_long, f64p, f64p, f64p, f64p]
        lib.oracle_couple.argtypes = [f64p, c_int, f64p]
        lib.oracle_svm_probs.argtypes = [f32p, c_int, c_long, c_int, f32p, f32p,
                                         f32p, f32p, f64p, i32p, f64p]
        lib.oracle_knn_min_candidates.argtypes = [c_int, c_int, c_int]
        lib.oracle_knn_min_candidates.restype = c_long
        lib.oracle_knn.argtypes = [f32p, f32p, c_int, c_int, c_int, c_int, c_int,
                                   c_double, c_int, c_long, c_long, f64p, i32p, i32p,
                                   f64p, f64p, f64p]
        for name in ("oracle_band_means", "oracle_covariance", "oracle_jacobi",
                     "oracle_pca_one_band", "oracle_project", "oracle_couple", "oracle_svm_probs",
                     "oracle_knn"):
            getattr(lib, name).restype = c_int
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s returned status %d" % (what, status))
        self.status = status


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(st, what)


def band_means(cube: np.ndarray) -> np.ndarray:
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    B = cube.shape[0]
    N = cube.size // B
    mu = np.empty(B)
    _check(_load().oracle_band_means(_p(cube, ctypes.c_float), B, N, _p(mu, ctypes.c_double)),
           "oracle_band_means")
    return mu


def covariance(cube: np.ndarray, mu: np.ndarray) -> np.ndarray:
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    B = cube.shape[0]
    N = cube.size // B
    C = np.empty((B, B))
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    _check(_load().oracle_covariance(_p(cube, ctypes.c_float), B, N, _p(mu, ctypes.c_double),
                                     _p(C, ctypes.c_double)), "oracle_covariance")
    return C


def covariance_matmul(cube: np.ndarray, mu: np.ndarray, chunk: int = 65536) -> np.ndarray:
    """Step (ii) for large cubes: the same definition as covariance(),
    C = (1/N) sum_p (x_p - mu)(x_p - mu)^T in FP64, with each chunk of
    pixels contracted by a library matmul (the C loop takes minutes at
    1024 x 1024 x 256)."""
    cube = np.asarray(cube)
    B = cube.shape[0]
    X = cube.reshape(B, -1)
    N = X.shape[1]
    mu = np.asarray(mu, dtype=np.float64)
    C = np.zeros((B, B))
    for p0 in range(0, N, chunk):
        Y = X[:, p0:p0 + chunk].astype(np.float64) - mu[:, None]
        C += Y @ Y.T
    return C / N


def jacobi(C: np.ndarray, tol: float = 1e-13, max_rot: int = 0):
    """Classical Jacobi: returns (evals, V, n_rot, status)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    B = C.shape[0]
    ev = np.empty(B)
    V = np.empty((B, B))
    nrot = ctypes.c_long(0)
    st = _load().oracle_jacobi(_p(C, ctypes.c_double), B, tol, max_rot, _p(ev, ctypes.c_double),
                               _p(V, ctypes.c_double), ctypes.byref(nrot))
    return ev, V, int(nrot.value), st


def project(cube: np.ndarray, mu: np.ndarray, v1: np.ndarray):
    """Step (iv): (I_raw, I_norm) of the cube's pixels on v1."""
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    B = cube.shape[0]
    N = cube.size // B
    I = np.empty(N)
    In = np.empty(N)
    d = ctypes.c_double
    _check(_load().oracle_project(_p(cube, ctypes.c_float), B, N,
                                  _p(np.ascontiguousarray(mu, dtype=np.float64), d),
                                  _p(np.ascontiguousarray(v1, dtype=np.float64), d),
                                  _p(I, d), _p(In, d)), "oracle_project")
    return I, In


def pca_one_band(cube: np.ndarray, tol: float = 1e-13) -> Dict[str, np.ndarray]:
    """Steps (i)-(iv) of the PCA plus min-max normalisation, all FP64."""
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    B, H, W = cube.shape
    N = H * W
    out = dict(mu=np.empty(B), C=np.empty((B, B)), evals=np.empty(B), V=np.empty((B, B)),
               v1=np.empty(B), lambda1=np.empty(1), I_raw=np.empty(N), I_norm=np.empty(N))
    nrot = ctypes.c_long(0)
    d = ctypes.c_double
    st = _load().oracle_pca_one_band(
        _p(cube, ctypes.c_float), B, H, W, tol, _p(out["mu"], d), _p(out["C"], d),
        _p(out["evals"], d), _p(out["V"], d), _p(out["v1"], d), _p(out["lambda1"], d),
        _p(out["I_raw"], d), _p(out["I_norm"], d), ctypes.byref(nrot))
    _check(st, "oracle_pca_one_band")
    out["lambda1"] = float(out["lambda1"][0])
    out["n_rot"] = int(nrot.value)
    out["I_raw"] = out["I_raw"].reshape(H, W)
    out["I_norm"] = out["I_norm"].reshape(H, W)
    return out


def couple(r: np.ndarray) -> np.ndarray:
    """Wu-Lin-Weng second-method coupling of a k x k pairwise matrix."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    k = r.shape[0]
    p = np.empty(k)
    _check(_load().oracle_couple(_p(r, ctypes.c_double), k, _p(p, ctypes.c_double)),
           "oracle_couple")
    return p


def svm_probs(cube: np.ndarray, model, want_dec: bool = False):
    """Returns (P[k,H,W] f64, labels[H,W] i32, dec[M,H,W] or None)."""
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    B, H, W = cube.shape
    N = H * W
    k = model.n_classes
    M = k * (k - 1) // 2
    P = np.empty((k, N))
    lab = np.empty(N, dtype=np.int32)
    dec = np.empty((M, N)) if want_dec else None
    f = ctypes.c_float
    st = _load().oracle_svm_probs(
        _p(cube, f), B, N, k, _p(np.ascontiguousarray(model.w, dtype=np.float32), f),
        _p(np.ascontiguousarray(model.b, dtype=np.float32), f),
        _p(np.ascontiguousarray(model.platt_a, dtype=np.float32), f),
        _p(np.ascontiguousarray(model.platt_b, dtype=np.float32), f),
        _p(P, ctypes.c_double), _p(lab, ctypes.c_int), _p(dec, ctypes.c_double))
    _check(st, "oracle_svm_probs")
    return (P.reshape(k, H, W), lab.reshape(H, W),
            None if dec is None else dec.reshape(M, H, W))


def knn_min_candidates(H: int, W: int, R: int) -> int:
    return int(_load().oracle_knn_min_candidates(H, W, R))


def knn(I_norm: np.ndarray, P: np.ndarray, K: int, R: int, lam: float,
        p0: int = 0, p1: Optional[int] = None, want_nbr: bool = False,
        float_keys: bool = False):
    """KNN filter on pixels [p0, p1) of the float inputs (Eq. 1, Eq. 2).

    float_keys: take the selection on the float terms of Eq. 1 (fl(I_p-I_q)^2
    and fl(lambda^2)(dr^2+dc^2), each rounded to float, summed exactly)
    instead of on FP64 distances.

    Returns dict with O[k, n], labels[n], nbr[n, K+1] (if asked: the first
    K+1 candidates in (distance, index) order, -1 padded), dK, dK1, gapO.
    """
    I_norm = np.ascontiguousarray(I_norm, dtype=np.float32)
    P = np.ascontiguousarray(P, dtype=np.float32)
    H, W = I_norm.shape
    k = P.shape[0]
    if p1 is None:
        p1 = H * W
    n = p1 - p0
    O = np.empty((k, n))
    lab = np.empty(n, dtype=np.int32)
    nbr = np.empty((n, K + 1), dtype=np.int32) if want_nbr else None
    dK, dK1, gap = np.empty(n), np.empty(n), np.empty(n)
    d = ctypes.c_double
    st = _load().oracle_knn(_p(I_norm, ctypes.c_float), _p(P, ctypes.c_float), H, W, k, K, R,
                            float(lam), 1 if float_keys else 0, p0, p1, _p(O, d), _p(lab, ctypes.c_int),
                            _p(nbr, ctypes.c_int), _p(dK, d), _p(dK1, d), _p(gap, d))
    _check(st, "oracle_knn")
    return dict(O=O, labels=lab, nbr=nbr, dK=dK, dK1=dK1, gapO=gap)


def classify(cube: np.ndarray, model, K: int, R: int, lam: float):
    """Whole path in FP64: PCA one-band and SVM, then the KNN filter on the
    float32-rounded I_norm and P (the precision the maps are stored in)."""
    pca = pca_one_band(cube)
    P, svm_lab, _ = svm_probs(cube, model)
    I32 = pca["I_norm"].astype(np.float32)
    P32 = P.astype(np.float32)
    kn = knn(I32, P32, K, R, lam)
    H, W = I32.shape
    return dict(pca=pca, P=P, svm_labels=svm_lab, I32=I32, P32=P32, knn=kn,
                labels=kn["labels"].reshape(H, W), O=kn["O"].reshape(-1, H, W))
