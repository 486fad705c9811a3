"""Seeded synthetic hyperspectral inputs shared by the tests, the bench and smoke().

This package holds input generation only: spectra, label maps, noisy cubes and
the linear one-vs-one SVM model built from the class spectra. None of the
classifier's arithmetic (PCA, Platt scaling, coupling, KNN) lives here, so the
FP64 oracle and the CUDA path can both draw their inputs from it without
sharing any of the method.
"""

from .hsi import (  # noqa: F401
    CONFIGS,
    SEEDS,
    Frame,
    SvmModel,
    endmembers,
    make_batch,
    make_frame,
    make_config,
    make_serving_pool,
    ovo_pairs,
    serving_arrivals,
    svm_from_endmembers,
    voronoi_labels,
)
