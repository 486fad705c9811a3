"""Synthetic hyperspectral frames shaped like the paper's workloads.

The paper's brain and dermatology images (Section II.A, Table 1) are not
available, so seeded stand-ins with the same shapes are generated here:

* endmember spectra: each class spectrum is a sum of Gaussians over the band
  index plus a floor, rescaled to a maximum of 0.9 (smooth, highly correlated
  bands, as in a pre-processed reflectance cube);
* a label map: a Voronoi partition of random seed points, each region given a
  class (contiguous tissue regions, so the KNN filter has borders to work on);
* the cube: pixel = endmember[label] + i.i.d. Gaussian noise per band, clipped
  to [0, 1], stored float32 band-sequential (B x H x W), the "each row is a
  band" matrix of Section III.A.2;
* the SVM model: the training stage is out of scope, so the one-vs-one linear
  hyperplanes are placed between the class spectra: w_ij is the unit vector
  from mu_j to mu_i and the bias puts the plane at their midpoint. Platt
  parameters A = -5, B = 0. Pairs are in lexicographic order (0,1), (0,2), ...

Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class SvmModel:
    """One-vs-one linear SVM with Platt parameters, all float32.

    ``w`` is M x B row-major (M = k(k-1)/2), ``b``, ``platt_a`` and ``platt_b``
    have length M; row m belongs to pair ``ovo_pairs(k)[m]``.
    """

    n_classes: int
    w: np.ndarray
    b: np.ndarray
    platt_a: np.ndarray
    platt_b: np.ndarray

    @property
    def n_bands(self) -> int:
        return int(self.w.shape[1])


@dataclasses.dataclass
class Frame:
    """One synthetic frame: float32 cube (B, H, W), truth labels (H, W)."""

    cube: np.ndarray
    truth: np.ndarray
    spectra: np.ndarray  # k x B float64 class spectra
    model: Optional[SvmModel]  # None when two class spectra coincide (B = 1)
    K: int
    window_rows: int
    lam: float
    sigma: float
    seed: int

    @property
    def shape(self) -> Tuple[int, int, int]:
        B, H, W = self.cube.shape
        return B, H, W


def ovo_pairs(k: int) -> List[Tuple[int, int]]:
    """Lexicographic one-vs-one pair order (0,1), (0,2), ..., (k-2,k-1)."""
    return [(i, j) for i in range(k) for j in range(i + 1, k)]


def endmembers(rng: np.random.Generator, k: int, B: int, n_gauss: int = 3,
               wide: bool = False) -> np.ndarray:
    """k smooth spectra over B bands, each a sum of Gaussians, max 0.9."""
    b = np.arange(B, dtype=np.float64)
    out = np.empty((k, B), dtype=np.float64)
    for c in range(k):
        centres = rng.uniform(0.0, B - 1.0, size=n_gauss)
        if wide:
            widths = rng.uniform(B / 4.0, B / 2.0, size=n_gauss)
        else:
            widths = rng.uniform(B / 16.0, B / 4.0, size=n_gauss)
        amps = rng.uniform(0.3, 1.0, size=n_gauss)
        s = np.full(B, 0.05)
        for m, w, a in zip(centres, widths, amps):
            s += a * np.exp(-0.5 * ((b - m) / w) ** 2)
        out[c] = s * (0.9 / s.max())
    return out


def voronoi_labels(rng: np.random.Generator, H: int, W: int, k: int,
                   n_seeds: int, fractions: Optional[Sequence[float]] = None
                   ) -> np.ndarray:
    """Voronoi partition of ``n_seeds`` uniform points, one class per region.

    Without ``fractions``: seed s < k gets class s, the rest random classes.
    With ``fractions``: regions are visited by descending area and each goes
    to the class with the largest remaining pixel deficit against the target
    fractions. Distance ties go to the lower seed index.
    """
    sy = rng.uniform(0.0, H, size=n_seeds)
    sx = rng.uniform(0.0, W, size=n_seeds)
    region = np.empty((H, W), dtype=np.int32)
    xs = np.arange(W, dtype=np.float64) + 0.5
    for r0 in range(0, H, 64):
        r1 = min(H, r0 + 64)
        ys = np.arange(r0, r1, dtype=np.float64) + 0.5
        d2 = ((ys[None, :, None] - sy[:, None, None]) ** 2
              + (xs[None, None, :] - sx[:, None, None]) ** 2)
        region[r0:r1] = np.argmin(d2, axis=0)  # first minimum = lower seed
    if fractions is None:
        cls = np.empty(n_seeds, dtype=np.int32)
        cls[:min(k, n_seeds)] = np.arange(min(k, n_seeds))
        if n_seeds > k:
            cls[k:] = rng.integers(0, k, size=n_seeds - k)
    else:
        area = np.bincount(region.ravel(), minlength=n_seeds)
        target = np.asarray(fractions, dtype=np.float64) * H * W
        have = np.zeros(k)
        cls = np.zeros(n_seeds, dtype=np.int32)
        for s in np.argsort(-area, kind="stable"):
            c = int(np.argmax(target - have))
            cls[s] = c
            have[c] += area[s]
    return cls[region]


def svm_from_endmembers(spectra: np.ndarray, platt_a: float = -5.0,
                        platt_b: float = 0.0) -> SvmModel:
    """OvO hyperplanes between class spectra (stand-in for offline training)."""
    k, B = spectra.shape
    pairs = ovo_pairs(k)
    w = np.empty((len(pairs), B), dtype=np.float64)
    b = np.empty(len(pairs), dtype=np.float64)
    for m, (i, j) in enumerate(pairs):
        d = spectra[i] - spectra[j]
        nd = np.linalg.norm(d)
        if not nd > 0.0:
            raise ValueError("classes %d and %d have identical spectra: no separating "
                             "hyperplane" % (i, j))
        w[m] = d / nd
        b[m] = -w[m] @ (0.5 * (spectra[i] + spectra[j]))
    M = len(pairs)
    return SvmModel(
        n_classes=k,
        w=np.ascontiguousarray(w, dtype=np.float32),
        b=b.astype(np.float32),
        platt_a=np.full(M, platt_a, dtype=np.float32),
        platt_b=np.full(M, platt_b, dtype=np.float32),
    )


def make_frame(seed: int, H: int, W: int, B: int, k: int = 4,
               sigma: float = 0.02, n_seeds: Optional[int] = None,
               fractions: Optional[Sequence[float]] = (0.40, 0.25, 0.20, 0.15),
               n_gauss: int = 3, wide: bool = False, K: int = 40,
               window_rows: int = 14, lam: float = 1.0,
               spectra: Optional[np.ndarray] = None) -> Frame:
    """Generate one frame. ``spectra`` lets several frames share a model."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if spectra is None:
        spectra = endmembers(rng, k, B, n_gauss=n_gauss, wide=wide)
    if n_seeds is None:
        n_seeds = 8 * k
    if fractions is not None and len(fractions) != k:
        fractions = None
    truth = voronoi_labels(rng, H, W, k, n_seeds, fractions)
    cube = np.empty((B, H, W), dtype=np.float32)
    base = spectra.astype(np.float32)
    for band in range(B):
        noise = rng.standard_normal((H, W), dtype=np.float32) * np.float32(sigma)
        np.clip(base[truth, band] + noise, 0.0, 1.0, out=cube[band])
    # a one-band cube rescales every class spectrum to the same value: such a
    # frame serves the PCA alone and carries no SVM model
    distinct = all(np.linalg.norm(spectra[i] - spectra[j]) > 0.0 for i, j in ovo_pairs(k))
    return Frame(cube=cube, truth=truth, spectra=spectra,
                 model=svm_from_endmembers(spectra) if distinct else None, K=K,
                 window_rows=window_rows, lam=lam, sigma=sigma, seed=seed)


# The five workloads: tiny parity case, neurosurgery-scale frame, batched
# uneven snapshot frames, 1024x1024x256 mixed-precision frame, serving stream.
CONFIGS = {
    1: dict(name="tiny", H=32, W=32, B=16, k=4, sigma=0.01, n_seeds=6,
            fractions=None, K=8, window_rows=5, lam=1.0),
    2: dict(name="neuro", H=416, W=512, B=128, k=4, sigma=0.02, n_seeds=32,
            K=40, window_rows=14, lam=1.0),
    4: dict(name="mixed", H=1024, W=1024, B=256, k=4, sigma=0.01, n_seeds=32,
            n_gauss=2, wide=True, K=40, window_rows=14, lam=1.0),
}
SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}


def make_config(i: int, seed: Optional[int] = None) -> Frame:
    """Frame of single-frame config ``i`` (1 tiny, 2 neuro, 4 mixed)."""
    cfg = dict(CONFIGS[i])
    cfg.pop("name")
    return make_frame(SEEDS[i] if seed is None else seed, **cfg)


def make_batch(n_frames: int = 256, seed: int = SEEDS[3], side_lo: int = 40,
               side_hi: int = 64, B: int = 125, k: int = 4,
               sigma: float = 0.03) -> List[Frame]:
    """Uneven square snapshot frames sharing one set of class spectra."""
    rng = np.random.Generator(np.random.PCG64(seed))
    spectra = endmembers(rng, k, B)
    sides = rng.integers(side_lo, side_hi + 1, size=n_frames)
    return [make_frame(seed * 1000 + f, int(s), int(s), B, k=k, sigma=sigma,
                       K=16, window_rows=7, lam=1.0, spectra=spectra)
            for f, s in enumerate(sides)]


def make_serving_pool(n_snapshot: int = 24, n_pushbroom: int = 6, seed: int = SEEDS[5],
                      k: int = 4, pushbroom_scale: float = 1.0) -> List[Frame]:
    """Request frames of the serving stream, each with its own class spectra
    (hence its own SVM model) and K drawn from {16, 40}: snapshot cubes
    (40-64 px square, 125 bands, sigma 0.03, window 7 rows) and pushbroom
    cubes (H 384-640 x W 320-512 px scaled by ``pushbroom_scale``, 128 bands,
    sigma 0.02, window 14 rows). The first ``n_snapshot`` are snapshots."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_snapshot + n_pushbroom):
        K = int(rng.choice([16, 40]))
        if i < n_snapshot:
            s = int(rng.integers(40, 65))
            out.append(make_frame(seed * 1000 + i, s, s, 125, k=k, sigma=0.03, K=K,
                                  window_rows=7, lam=1.0))
        else:
            H = max(16, int(round(int(rng.integers(384, 641)) * pushbroom_scale)))
            W = max(16, int(round(int(rng.integers(320, 513)) * pushbroom_scale)))
            out.append(make_frame(seed * 1000 + i, H, W, 128, k=k, sigma=0.02, K=K,
                                  window_rows=14, lam=1.0))
    return out


def serving_arrivals(n_requests: int, rate_hz: float, n_snapshot: int, n_pushbroom: int,
                     snapshot_share: float = 0.7, seed: int = SEEDS[5]):
    """Poisson arrival times (seconds from 0) at ``rate_hz`` and, per request,
    the index of its frame in a serving pool: a snapshot with probability
    ``snapshot_share``, else a pushbroom cube, uniform within each kind."""
    rng = np.random.Generator(np.random.PCG64(seed + 17))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    snap = rng.random(n_requests) < snapshot_share
    idx = np.where(snap, rng.integers(0, n_snapshot, size=n_requests),
                   n_snapshot + rng.integers(0, max(1, n_pushbroom), size=n_requests))
    if n_pushbroom == 0:
        idx = rng.integers(0, n_snapshot, size=n_requests)
    return t, idx
