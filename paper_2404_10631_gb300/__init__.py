"""Python binding of libhsc.so, the GB300 spatial-spectral HSI classifier.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels. PyTorch provides device memory and streams. The functions keep
the C names (``hsc_classify`` ...) and take CUDA tensors; ``Context`` owns an
``hsc_ctx``. Importing this package does not load the library; the first call
does, and it raises if ``libhsc.so`` has not been built (no CPU fallback).
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
# HSC_LIBRARY names another build to load (e.g. libhsc_checked.so, the build
# with index checks); by default the library built beside this file
LIB_PATH = os.environ.get("HSC_LIBRARY") or os.path.join(HERE, "libhsc.so")

HSC_OK = 0
HSC_ERR_INVALID_ARG = 1
HSC_ERR_OOM = 2
HSC_ERR_CUDA = 3
HSC_ERR_NOT_CONVERGED = 4
HSC_ERR_TIMEOUT = 5
HSC_ERR_UNSUPPORTED = 6
HSC_ERR_NONFINITE = 7

HSC_MAX_CLASSES = 8
HSC_MAX_K = 64
HSC_MAX_WINDOW_ROWS = 32
HSC_MAX_BANDS = 1024
HSC_MAX_PC = 8
HSC_PCA_MINMAX = 1
HSC_SVM_COUPLE_F64 = 2
HSC_CLASSIFY_RAW_I = 16
HSC_CUBE_BIP = 32
HSC_JACOBI_ONE_CTA = 128

EXPORTED = ("hsc_ctx_create", "hsc_ctx_destroy", "hsc_set_stream", "hsc_last_error",
            "hsc_status_string", "hsc_sync", "hsc_reserve", "hsc_scratch_bytes",
            "hsc_pca_one_band", "hsc_svm_probs", "hsc_knn_filter", "hsc_classify",
            "hsc_profile_enable", "hsc_profile_read", "hsc_pca_diagnostics", "hsc_measure_fma_rate",
            "hsc_autotune", "hsc_set_tuning", "hsc_pca_project",
            "hsc_pca_one_band_noalloc", "hsc_pca_covariance", "hsc_knn_diagnostics",
            "hsc_classify_batch", "hsc_server_create", "hsc_server_submit",
            "hsc_server_wait", "hsc_server_stats_get", "hsc_server_destroy",
            "hsc_test_stall_next_gram", "hsc_test_stall_next_batch_wait")
HSC_BATCH_GRAPH = 8
HSC_BATCH_POOL = 64
HSC_BATCH_FUSED = 256
HSC_COV_FP32_PIPE = 4
HSC_NOALLOC_MAX_BANDS = 128
STAGES = ("moments", "jacobi", "project_svm", "normalize", "knn")


class hsc_svm_model(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("n_bands", ctypes.c_int32),
                ("w", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("platt_a", ctypes.c_void_p), ("platt_b", ctypes.c_void_p)]


class hsc_knn_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("window_rows", ctypes.c_int32),
                ("lambda_", ctypes.c_float), ("search", ctypes.c_int32)]


HSC_KNN_SEARCH_AUTO = 0
HSC_KNN_SEARCH_FULL = 1
HSC_KNN_SEARCH_PRUNED = 2
HSC_KNN_SEARCH_HEAP = 3


class hsc_frame(ctypes.Structure):
    _fields_ = [("cube", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("labels", ctypes.c_void_p), ("out_probs", ctypes.c_void_p),
                ("one_band", ctypes.c_void_p), ("probs", ctypes.c_void_p)]


class hsc_request(ctypes.Structure):
    _fields_ = [("cube", ctypes.c_void_p), ("B", ctypes.c_int32), ("H", ctypes.c_int32),
                ("W", ctypes.c_int32), ("model", hsc_svm_model), ("params", hsc_knn_params),
                ("flags", ctypes.c_uint), ("labels", ctypes.c_void_p),
                ("out_probs", ctypes.c_void_p)]


class hsc_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("pixels", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("peak_inflight", ctypes.c_int32), ("peak_bytes", ctypes.c_size_t)]


class HscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_status_name(status), message))
        self.status = status


_lib = None


def _status_name(st: int) -> str:
    names = {0: "HSC_OK", 1: "HSC_ERR_INVALID_ARG", 2: "HSC_ERR_OOM", 3: "HSC_ERR_CUDA",
             4: "HSC_ERR_NOT_CONVERGED", 5: "HSC_ERR_TIMEOUT", 6: "HSC_ERR_UNSUPPORTED",
             7: "HSC_ERR_NONFINITE"}
    return names.get(st, "HSC_ERR_%d" % st)


def lib():
    """Load libhsc.so (raises when it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built (run paper_2404_10631_gb300.build.build())"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.hsc_ctx_create.argtypes = [i32, vp, sz, ctypes.POINTER(vp)]
        L.hsc_ctx_destroy.argtypes = [vp]
        L.hsc_ctx_destroy.restype = None
        L.hsc_set_stream.argtypes = [vp, vp]
        L.hsc_last_error.argtypes = [vp]
        L.hsc_last_error.restype = ctypes.c_char_p
        L.hsc_status_string.argtypes = [i32]
        L.hsc_status_string.restype = ctypes.c_char_p
        L.hsc_sync.argtypes = [vp]
        L.hsc_reserve.argtypes = [vp, i32, i32, i32, i32]
        L.hsc_scratch_bytes.argtypes = [vp]
        L.hsc_scratch_bytes.restype = sz
        L.hsc_pca_one_band.argtypes = [vp, vp, i32, i32, i32, ctypes.c_uint, vp, vp, vp]
        L.hsc_svm_probs.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(hsc_svm_model),
                                    ctypes.c_uint, vp, vp]
        L.hsc_knn_filter.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.POINTER(hsc_knn_params),
                                     vp, vp, vp]
        L.hsc_classify.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(hsc_svm_model),
                                   ctypes.POINTER(hsc_knn_params), ctypes.c_uint, vp, vp, vp, vp]
        L.hsc_classify_batch.argtypes = [vp, ctypes.POINTER(hsc_frame), i32, i32,
                                         ctypes.POINTER(hsc_svm_model),
                                         ctypes.POINTER(hsc_knn_params), ctypes.c_uint]
        L.hsc_server_create.argtypes = [i32, sz, i32, ctypes.POINTER(vp)]
        L.hsc_server_submit.argtypes = [vp, ctypes.POINTER(hsc_request),
                                        ctypes.POINTER(ctypes.c_uint64)]
        L.hsc_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
        L.hsc_server_stats_get.argtypes = [vp, ctypes.POINTER(hsc_server_stats)]
        L.hsc_server_destroy.argtypes = [vp]
        L.hsc_server_destroy.restype = None
        L.hsc_test_stall_next_gram.argtypes = [vp]
        L.hsc_test_stall_next_batch_wait.argtypes = [vp]
        L.hsc_knn_diagnostics.argtypes = [vp, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]
        L.hsc_pca_covariance.argtypes = [vp, vp, i32, i32, i32, ctypes.c_uint, vp, vp]
        L.hsc_pca_one_band_noalloc.argtypes = [vp, vp, i32, i32, i32, ctypes.c_uint, vp, vp, vp]
        L.hsc_profile_enable.argtypes = [vp, i32]
        L.hsc_measure_fma_rate.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double)]
        L.hsc_autotune.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(hsc_svm_model),
                                   ctypes.POINTER(hsc_knn_params), ctypes.POINTER(ctypes.c_int32)]
        L.hsc_set_tuning.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_int32)]
        L.hsc_pca_project.argtypes = [vp, vp, i32, i32, i32, i32, ctypes.c_uint, vp, vp, vp]
        L.hsc_pca_diagnostics.argtypes = [vp, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]
        L.hsc_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        for name in EXPORTED:
            fn = getattr(L, name)
            if name not in ("hsc_ctx_destroy", "hsc_last_error", "hsc_status_string",
                            "hsc_scratch_bytes"):
                fn.restype = ctypes.c_int
        _lib = L
    return _lib


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _stream_handle(stream) -> Optional[int]:
    """cudaStream_t of a torch stream (or raw handle). Handle 0 is the legacy
    default stream, which the C API must receive as cudaStreamLegacy because
    NULL there means "a stream owned by the context"."""
    if stream is None:
        return None
    h = int(getattr(stream, "cuda_stream", stream))
    return CUDA_STREAM_LEGACY if h == 0 else h


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class Model:
    """Device-resident OvO SVM model (float32 CUDA tensors)."""

    def __init__(self, n_classes: int, w, b, platt_a, platt_b):
        self.n_classes = int(n_classes)
        self.w, self.b, self.platt_a, self.platt_b = w, b, platt_a, platt_b
        self.n_bands = int(w.shape[1])

    @classmethod
    def from_host(cls, m, device="cuda"):
        import torch
        f = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        return cls(m.n_classes, f(m.w), f(m.b), f(m.platt_a), f(m.platt_b))

    def struct(self) -> hsc_svm_model:
        return hsc_svm_model(self.n_classes, self.n_bands, _ptr(self.w), _ptr(self.b),
                             _ptr(self.platt_a), _ptr(self.platt_b))


class Context:
    """An ``hsc_ctx`` on one device and stream (None = a stream it owns)."""

    def __init__(self, device: int = 0, stream=None, scratch_cap_bytes: int = 0):
        L = lib()
        h = ctypes.c_void_p()
        st = L.hsc_ctx_create(device, _stream_handle(stream), scratch_cap_bytes, ctypes.byref(h))
        if st != HSC_OK:
            raise HscError(st, "hsc_ctx_create(device=%d)" % device)
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().hsc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def check(self, st: int):
        if st != HSC_OK:
            raise HscError(st, lib().hsc_last_error(self.handle).decode())

    def set_stream(self, stream=None):
        self.check(lib().hsc_set_stream(self.handle, _stream_handle(stream)))

    def sync(self):
        self.check(lib().hsc_sync(self.handle))

    def reserve(self, B, H, W, n_classes):
        self.check(lib().hsc_reserve(self.handle, B, H, W, n_classes))

    def profile(self, enable: bool = True):
        """Bracket every stage launch with CUDA events on the context's stream."""
        self.check(lib().hsc_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self):
        """Wait for the stream; per-stage (ms, kernel launches) since the last read."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        kern = (ctypes.c_int64 * n)()
        dropped = ctypes.c_int64(0)
        self.check(lib().hsc_profile_read(self.handle, ms, kern, ctypes.byref(dropped)))
        return ({STAGES[i]: float(ms[i]) for i in range(n)},
                {STAGES[i]: int(kern[i]) for i in range(n)}, int(dropped.value))

    def pca_diagnostics(self, cycles: bool = False):
        """(FP32 Jacobi sweeps, FP64 refinement iterations) of the last PCA,
        plus (sweep cycles, refinement cycles) when ``cycles``."""
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        c, d = ctypes.c_int64(0), ctypes.c_int64(0)
        self.check(lib().hsc_pca_diagnostics(self.handle, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(c), ctypes.byref(d)))
        if cycles:
            return int(a.value), int(b.value), int(c.value), int(d.value)
        return int(a.value), int(b.value)

    def test_stall_next_gram(self):
        """Testing aid: the next tensor-core Gram of this context runs out its
        first bounded wait (see hsc_test_stall_next_gram)."""
        self.check(lib().hsc_test_stall_next_gram(self.handle))

    def test_stall_next_batch_wait(self):
        """Testing aid: the next fused stage-major batch of this context runs
        out its KNN segments' bounded waits on its first frame (see
        hsc_test_stall_next_batch_wait)."""
        self.check(lib().hsc_test_stall_next_batch_wait(self.handle))

    def knn_candidates_evaluated(self) -> int:
        """Candidates the pruned KNN search evaluated since the last call
        (resets the counters of knn_diagnostics too)."""
        return self.knn_diagnostics()[0]

    def knn_diagnostics(self):
        """(candidates evaluated, pixels handed to the redo pass) of the pruned
        KNN search since the last call; both counters are then reset."""
        v, r = ctypes.c_int64(0), ctypes.c_int64(0)
        self.check(lib().hsc_knn_diagnostics(self.handle, ctypes.byref(v), ctypes.byref(r)))
        return int(v.value), int(r.value)

    def autotune(self, cube, model, K=None, window_rows=None, lam=None,
                 search: int = HSC_KNN_SEARCH_AUTO) -> dict:
        """Times the launch-shape candidates on this cube (B x H x W) and keeps
        the fastest for frames of its shape; with K, window_rows and lam also
        the pruned KNN walk's variant. Returns the chosen parameters."""
        B, H, W = cube.shape
        cfg = (ctypes.c_int32 * 4)()
        ms = model.struct()
        prm = None
        if K is not None:
            prm = ctypes.byref(hsc_knn_params(K, window_rows, lam, search))
        self.check(lib().hsc_autotune(self.handle, _ptr(cube), B, H, W, ctypes.byref(ms), prm,
                                      cfg))
        return {"gram_stages": cfg[0], "svm_px": cfg[1], "svm_blocks_per_sm": cfg[2],
                "knn_variant": cfg[3]}

    def set_tuning(self, B, H, W, n_classes, config=None):
        """Sets (gram_stages, svm_px, svm_blocks_per_sm[, knn_variant]) for that
        frame shape, or clears the tuning (config None)."""
        if config is None:
            self.check(lib().hsc_set_tuning(self.handle, B, H, W, n_classes, None))
            return
        config = tuple(config) + (0,) * (4 - len(config))
        cfg = (ctypes.c_int32 * 4)(*config)
        self.check(lib().hsc_set_tuning(self.handle, B, H, W, n_classes, cfg))

    @property
    def scratch_bytes(self) -> int:
        return int(lib().hsc_scratch_bytes(self.handle))


def _bhw(cube, flags):
    """(B, H, W) of a band-sequential cube, or of a pixel-interleaved one."""
    if flags & HSC_CUBE_BIP:
        H, W, B = cube.shape
        return B, H, W
    return tuple(cube.shape)


def hsc_measure_fma_rate(device: int = 0, fp64: bool = False) -> float:
    """FP32 (or FP64) multiply-add lane-operations per second over all SMs."""
    r = ctypes.c_double(0.0)
    st = lib().hsc_measure_fma_rate(device, 1 if fp64 else 0, ctypes.byref(r))
    if st:
        raise HscError(st, "hsc_measure_fma_rate: " + _status_name(st))
    return r.value


def hsc_pca_one_band(ctx: Context, cube, flags: int = HSC_PCA_MINMAX, one_band=None,
                     eigvec=None, eigval=None):
    """Returns the H x W one-band image (allocated when not given). With
    HSC_CUBE_BIP the cube is H x W x B."""
    import torch
    B, H, W = _bhw(cube, flags)
    if one_band is None:
        one_band = torch.empty((H, W), dtype=torch.float32, device=cube.device)
    ctx.check(lib().hsc_pca_one_band(ctx.handle, _ptr(cube), B, H, W, flags, _ptr(one_band),
                                     _ptr(eigvec), _ptr(eigval)))
    return one_band


def hsc_pca_project(ctx: Context, cube, n_pc: int, flags: int = 0, out=None, eigvecs=None,
                    eigvals=None):
    """Projections on the n_pc leading principal components: n_pc x H x W
    (allocated when not given)."""
    import torch
    B, H, W = _bhw(cube, flags)
    if out is None:
        out = torch.empty((n_pc, H, W), dtype=torch.float32, device=cube.device)
    ctx.check(lib().hsc_pca_project(ctx.handle, _ptr(cube), B, H, W, n_pc, flags, _ptr(out),
                                    _ptr(eigvecs), _ptr(eigvals)))
    return out


def hsc_pca_covariance(ctx: Context, cube, flags: int = 0, mean=None, cov=None):
    """Band means (B, f64) and covariance (B x B, f64) of the cube."""
    import torch
    B, H, W = cube.shape
    if mean is None:
        mean = torch.empty(B, dtype=torch.float64, device=cube.device)
    if cov is None:
        cov = torch.empty((B, B), dtype=torch.float64, device=cube.device)
    ctx.check(lib().hsc_pca_covariance(ctx.handle, _ptr(cube), B, H, W, flags, _ptr(mean),
                                       _ptr(cov)))
    return mean, cov


def hsc_pca_one_band_noalloc(cube, flags: int = HSC_PCA_MINMAX, one_band=None, eigvec=None,
                             eigval=None, stream=None):
    """The allocation-free one-band PCA on ``stream`` (torch stream or handle;
    None = torch's current stream). All outputs must be passed in by callers
    that cannot allocate; those left as None are allocated here by torch for
    convenience. Raises HscError on a non-OK status."""
    import torch
    B, H, W = cube.shape
    if one_band is None:
        one_band = torch.empty((H, W), dtype=torch.float32, device=cube.device)
    if stream is None:
        stream = torch.cuda.current_stream(cube.device)
    st = lib().hsc_pca_one_band_noalloc(_stream_handle(stream), _ptr(cube), B, H, W, flags,
                                        _ptr(one_band), _ptr(eigvec), _ptr(eigval))
    if st != HSC_OK:
        raise HscError(st, "hsc_pca_one_band_noalloc")
    return one_band


def hsc_svm_probs(ctx: Context, cube, model: Model, flags: int = 0, probs=None,
                  svm_labels=None):
    import torch
    B, H, W = cube.shape
    if probs is None:
        probs = torch.empty((model.n_classes, H, W), dtype=torch.float32, device=cube.device)
    ms = model.struct()
    ctx.check(lib().hsc_svm_probs(ctx.handle, _ptr(cube), B, H, W, ctypes.byref(ms), flags,
                                  _ptr(probs), _ptr(svm_labels)))
    return probs


def hsc_knn_filter(ctx: Context, one_band, probs, K: int, window_rows: int, lam: float,
                   out_probs=None, labels=None, nbr_idx=None, search: int = HSC_KNN_SEARCH_AUTO):
    import torch
    k, H, W = probs.shape
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=probs.device)
    prm = hsc_knn_params(K, window_rows, lam, search)
    ctx.check(lib().hsc_knn_filter(ctx.handle, _ptr(one_band), _ptr(probs), k, H, W,
                                   ctypes.byref(prm), _ptr(out_probs), _ptr(labels),
                                   _ptr(nbr_idx)))
    return labels


def hsc_classify(ctx: Context, cube, model: Model, K: int, window_rows: int, lam: float,
                 flags: int = 0, labels=None, out_probs=None, one_band=None, probs=None,
                 search: int = HSC_KNN_SEARCH_AUTO):
    import torch
    B, H, W = _bhw(cube, flags)
    if labels is None:
        labels = torch.empty((H, W), dtype=torch.int32, device=cube.device)
    ms = model.struct()
    prm = hsc_knn_params(K, window_rows, lam, search)
    ctx.check(lib().hsc_classify(ctx.handle, _ptr(cube), B, H, W, ctypes.byref(ms),
                                 ctypes.byref(prm), flags, _ptr(labels), _ptr(out_probs),
                                 _ptr(one_band), _ptr(probs)))
    return labels


def hsc_classify_batch(ctx: Context, cubes, model: Model, K: int, window_rows: int, lam: float,
                       flags: int = 0, labels=None, out_probs=None, one_bands=None, probs=None,
                       search: int = HSC_KNN_SEARCH_AUTO):
    """Classify a list of B x H_i x W_i cubes in one call. Returns the list of
    label maps (allocated when not given); optional per-frame output lists."""
    import torch
    n = len(cubes)
    B = int(cubes[0].shape[0])
    if labels is None:
        labels = [torch.empty((c.shape[1], c.shape[2]), dtype=torch.int32, device=c.device)
                  for c in cubes]
    arr = (hsc_frame * n)()
    for i, c in enumerate(cubes):
        if int(c.shape[0]) != B:
            raise ValueError("all cubes need the same band count")
        arr[i] = hsc_frame(_ptr(c), int(c.shape[1]), int(c.shape[2]), _ptr(labels[i]),
                           _ptr(out_probs[i]) if out_probs else None,
                           _ptr(one_bands[i]) if one_bands else None,
                           _ptr(probs[i]) if probs else None)
    ms = model.struct()
    prm = hsc_knn_params(K, window_rows, lam, search)
    ctx.check(lib().hsc_classify_batch(ctx.handle, arr, n, B, ctypes.byref(ms),
                                       ctypes.byref(prm), flags))
    return labels


def _host_ptr(a, dtype_name: str) -> int:
    """Address of a C-contiguous host array (numpy or CPU torch tensor)."""
    if hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        if str(a.dtype) != "torch." + dtype_name:
            raise ValueError("expected %s" % dtype_name)
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"] or str(a.dtype) != dtype_name:
        raise ValueError("expected a C-contiguous %s array" % dtype_name)
    return a.ctypes.data


class Server:
    """An ``hsc_server``: requests with HOST cubes and HOST outputs, queued
    and admitted by a native dispatcher under an HBM budget (see
    hsc_server_create). ``submit`` returns a ticket, ``wait`` blocks on it."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_inflight: int = 8):
        h = ctypes.c_void_p()
        st = lib().hsc_server_create(device, hbm_budget_bytes, max_inflight, ctypes.byref(h))
        if st != HSC_OK:
            raise HscError(st, "hsc_server_create(device=%d)" % device)
        self.handle = h
        self._keep = {}  # ticket -> host buffers and model, alive until waited on

    def submit(self, cube, model: Model, K: int, window_rows: int, lam: float, labels,
               out_probs=None, flags: int = 0, search: int = HSC_KNN_SEARCH_AUTO) -> int:
        B, H, W = (int(x) for x in cube.shape)
        req = hsc_request(_host_ptr(cube, "float32"), B, H, W, model.struct(),
                          hsc_knn_params(K, window_rows, lam, search), flags,
                          _host_ptr(labels, "int32"),
                          _host_ptr(out_probs, "float32") if out_probs is not None else None)
        t = ctypes.c_uint64(0)
        st = lib().hsc_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if st != HSC_OK:
            raise HscError(st, "hsc_server_submit")
        self._keep[int(t.value)] = (cube, model, labels, out_probs)
        return int(t.value)

    def wait(self, ticket: int) -> float:
        """Blocks until the request is done; returns its latency in ms."""
        ms = ctypes.c_double(0.0)
        st = lib().hsc_server_wait(self.handle, ticket, ctypes.byref(ms))
        self._keep.pop(ticket, None)
        if st != HSC_OK:
            raise HscError(st, "request %d" % ticket)
        return float(ms.value)

    def stats(self) -> dict:
        s = hsc_server_stats()
        st = lib().hsc_server_stats_get(self.handle, ctypes.byref(s))
        if st != HSC_OK:
            raise HscError(st, "hsc_server_stats_get")
        return {name: getattr(s, name) for name, _ in hsc_server_stats._fields_}

    def close(self):
        if self.handle:
            lib().hsc_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
