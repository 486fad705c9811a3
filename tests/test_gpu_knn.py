"""KNN filter (Eq. 1, Eq. 2) on the GPU through the C ABI against the
oracle on the same float inputs: neighbour sets identical to the oracle's
float-key selection at every pixel, O within 1e-5 of the FP64 mean, labels
exact (and exact against the FP64 selection outside the task's near-ties)."""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from parity import check_knn, check_knn_outputs, sample_rows

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEARCHES = [1, 2, 3]  # full-window scan, pruned walk, heap selection


def run_knn(hsc, ctx, I, P, K, R, lam, search=1):
    import torch
    dev = torch.device("cuda")
    It = torch.as_tensor(np.ascontiguousarray(I, dtype=np.float32), device=dev)
    Pt = torch.as_tensor(np.ascontiguousarray(P, dtype=np.float32), device=dev)
    k, H, W = Pt.shape
    O = torch.full((k, H, W), -1.0, dtype=torch.float32, device=dev)
    lab = torch.full((H, W), -1, dtype=torch.int32, device=dev)
    nbr = torch.full((H, W, K), -1, dtype=torch.int32, device=dev)
    hsc.hsc_knn_filter(ctx, It, Pt, K, R, lam, out_probs=O, labels=lab, nbr_idx=nbr,
                       search=search)
    ctx.sync()
    return nbr.cpu().numpy(), O.cpu().numpy(), lab.cpu().numpy()


def rand_maps(H, W, k, seed, dyadic=False):
    rng = np.random.default_rng(seed)
    if dyadic:
        I = (rng.integers(0, 64, size=(H, W)) / 64.0).astype(np.float32)
    else:
        I = rng.random((H, W)).astype(np.float32)
    P = rng.random((k, H, W))
    P = (P / P.sum(axis=0)).astype(np.float32)
    return I, P


@pytest.mark.parametrize("name", ["knn_line5.json", "knn_window_ties.json"])
@pytest.mark.parametrize("search", SEARCHES)
def test_golden_hand_examples(hsc, ctx, name, search):
    g = json.load(open(os.path.join(GOLDEN, name)))
    I = np.asarray(g["I"], dtype=np.float32)
    P = np.asarray(g["P"], dtype=np.float32)
    nbr, O, lab = run_knn(hsc, ctx, I, P, g["K"], g["R"], g["lambda"], search)
    np.testing.assert_array_equal(nbr.reshape(-1, g["K"]), g["nbr"])
    np.testing.assert_allclose(O, g["O"], atol=1e-7)
    np.testing.assert_array_equal(lab, g["labels"])


@pytest.mark.parametrize("search", SEARCHES)
@pytest.mark.parametrize("H,W,K,R,lam,k", [
    (32, 32, 8, 5, 1.0, 4),      # the tiny configuration's sizes
    (37, 45, 40, 14, 1.0, 4),    # paper's K and window, ragged width
    (20, 130, 64, 32, 1.0, 3),   # maximum K and window
    (9, 600, 17, 7, 0.5, 5),     # two shared-memory chunks, lambda != 1
    (5, 1030, 3, 3, 2.0, 2),     # three chunks, ragged tail
    (1, 70, 4, 1, 1.0, 8),       # one row, eight classes
    (40, 7, 12, 4, 1.0, 4),      # narrower than a warp, even window
    (6, 50, 150, 9, 1.0, 3),     # K above 64 is rejected (checked below)
])
def test_random_maps_against_oracle(hsc, ctx, H, W, K, R, lam, k, search):
    I, P = rand_maps(H, W, k, seed=H * 1000 + W + K)
    if K > hsc.HSC_MAX_K:
        with pytest.raises(hsc.HscError) as e:
            run_knn(hsc, ctx, I, P, K, R, lam, search)
        assert e.value.status == hsc.HSC_ERR_UNSUPPORTED
        return
    nbr, O, lab = run_knn(hsc, ctx, I, P, K, R, lam, search)
    st = check_knn(I, P, K, R, lam, nbr, O, lab)
    assert st["pixels"] == H * W


@pytest.mark.parametrize("search", SEARCHES)
def test_k1_window1_returns_own_probabilities(hsc, ctx, search):
    I, P = rand_maps(33, 71, 4, seed=3)
    nbr, O, lab = run_knn(hsc, ctx, I, P, 1, 1, 1.0, search)
    np.testing.assert_array_equal(O, P)
    np.testing.assert_array_equal(lab, np.argmax(P, axis=0))
    np.testing.assert_array_equal(nbr.reshape(-1), np.arange(33 * 71))


def test_lambda0_constant_image_tie_rule(hsc, ctx):
    """All distances 0: the K smallest linear indices of the window win."""
    H, W, R, K = 12, 40, 5, 30
    I = np.full((H, W), 0.25, dtype=np.float32)
    _, P = rand_maps(H, W, 3, seed=4)
    nbr, O, lab = run_knn(hsc, ctx, I, P, K, R, 0.0)
    for p in range(H * W):
        lo = max(0, p // W - R // 2)
        np.testing.assert_array_equal(nbr.reshape(-1, K)[p], lo * W + np.arange(K))


@pytest.mark.parametrize("search", SEARCHES)
def test_dyadic_image_exact_ties(hsc, ctx, search):
    """Coarse grey levels make many exactly equal distances: the tie rule
    (smaller linear index) must match the oracle everywhere."""
    I, P = rand_maps(24, 50, 3, seed=5, dyadic=True)
    nbr, O, lab = run_knn(hsc, ctx, I, P, 20, 6, 1.0, search)
    st = check_knn(I, P, 20, 6, 1.0, nbr, O, lab)
    assert st["official_near_ties"] > 0 and st["fp64_set_differs"] == 0


@pytest.mark.parametrize("search", SEARCHES)
def test_whole_window_box_filter(hsc, ctx, search):
    H, W = 3, 21
    I, P = rand_maps(H, W, 4, seed=6)
    nbr, O, lab = run_knn(hsc, ctx, I, P, H * W, 6, 1.0, search)
    mean = P.astype(np.float64).reshape(4, -1).mean(axis=1)
    np.testing.assert_allclose(O.reshape(4, -1), np.repeat(mean[:, None], H * W, axis=1), atol=1e-6)


@pytest.mark.parametrize("search", SEARCHES)
def test_neuro_size_sampled_rows(hsc, ctx, search):
    """416 x 512 frame, K = 40, 14-row window: the oracle's own normalised
    one-band image and probabilities as inputs, rows at both borders and
    inside checked pixel by pixel."""
    f = synth.make_config(2)
    pca = oracle.pca_one_band(f.cube)
    P, _, _ = oracle.svm_probs(f.cube, f.model)
    I32 = pca["I_norm"].astype(np.float32)
    P32 = P.astype(np.float32)
    nbr, O, lab = run_knn(hsc, ctx, I32, P32, 40, 14, 1.0, search)
    H, W = I32.shape
    st = check_knn(I32, P32, 40, 14, 1.0, nbr, O, lab,
                   pixels=sample_rows(H, W, [0, 1, 6, 7, 200, 408, 409, 415]))
    assert st["pixels"] == 8 * W


def test_pruned_and_heap_equal_full_window(hsc, ctx):
    """All three searches select the same sets: identical outputs bit for bit
    (neighbour lists nearest first, so O sums in the same order)."""
    f = synth.make_config(2)
    pca = oracle.pca_one_band(f.cube)
    P, _, _ = oracle.svm_probs(f.cube, f.model)
    I32 = pca["I_norm"].astype(np.float32)
    P32 = P.astype(np.float32)
    a = run_knn(hsc, ctx, I32, P32, 40, 14, 1.0, 1)
    for search in (2, 3):
        b = run_knn(hsc, ctx, I32, P32, 40, 14, 1.0, search)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_pruned_search_rejects_lambda_zero(hsc, ctx):
    I, P = rand_maps(8, 40, 3, seed=9)
    with pytest.raises(hsc.HscError) as e:
        run_knn(hsc, ctx, I, P, 4, 3, 0.0, 2)
    assert e.value.status == hsc.HSC_ERR_INVALID_ARG
    run_knn(hsc, ctx, I, P, 4, 3, 0.0, 0)  # auto falls back to the full scan


# ---- the path the classifier runs: no neighbour-index output. The pruned
# walk then finishes most pixels itself (keys below its lower bound summed
# as they are found, the rest from its undecided-key buffer); only the
# pixels it cannot finish go to the redo pass, which the counter shows.

def run_knn_outputs(hsc, ctx, I, P, K, R, lam, search):
    """O and labels of hsc_knn_filter without nbr_idx, and the pixels the
    pruned walk handed to its redo pass."""
    import torch
    dev = torch.device("cuda")
    It = torch.as_tensor(np.ascontiguousarray(I, dtype=np.float32), device=dev)
    Pt = torch.as_tensor(np.ascontiguousarray(P, dtype=np.float32), device=dev)
    k, H, W = Pt.shape
    O = torch.full((k, H, W), -1.0, dtype=torch.float32, device=dev)
    lab = torch.full((H, W), -1, dtype=torch.int32, device=dev)
    ctx.knn_diagnostics()  # reset the counters
    hsc.hsc_knn_filter(ctx, It, Pt, K, R, lam, out_probs=O, labels=lab, search=search)
    ctx.sync()
    _, redo = ctx.knn_diagnostics()
    return O.cpu().numpy(), lab.cpu().numpy(), redo


def rand_probs(k, H, W, seed):
    """Probability maps independent of the image: any neighbour taken in
    place of another moves O by about 0.3 / K, far above the O tolerance, so
    O fingerprints the selected set."""
    rng = np.random.default_rng(seed)
    P = rng.random((k, H, W))
    return (P / P.sum(axis=0)).astype(np.float32)


@pytest.mark.parametrize("search", [0, 2])  # AUTO (pruned for lambda > 0), PRUNED
@pytest.mark.parametrize("H,W,K,R,lam,k", [
    (32, 32, 8, 5, 1.0, 4),      # the tiny configuration's sizes
    (37, 45, 40, 14, 1.0, 4),    # paper's K and window, ragged width
    (20, 130, 64, 32, 1.0, 3),   # maximum K and window
    (9, 600, 17, 7, 0.5, 5),     # lambda below 1
    (5, 1030, 3, 3, 2.0, 2),     # lambda above 1, ragged tail
    (1, 70, 4, 1, 1.0, 8),       # one row, eight classes
    (40, 7, 12, 4, 1.0, 4),      # narrower than a warp, even window
    (48, 300, 40, 14, 0.5, 4),   # the paper's K and window, lambda 0.5
    (48, 300, 40, 14, 2.0, 4),   # and lambda 2
    (64, 512, 40, 14, 0.25, 4),  # small lambda: the FP64 rule decides most pixels
])
def test_fast_path_random_maps_against_oracle(hsc, ctx, H, W, K, R, lam, k, search):
    I, P = rand_maps(H, W, k, seed=H * 1000 + W + K + int(lam * 8))
    O, lab, redo = run_knn_outputs(hsc, ctx, I, P, K, R, lam, search)
    st = check_knn_outputs(I, P, K, R, lam, O, lab)
    assert st["pixels"] == H * W
    if lam == 0.25:
        print("\nrandom %dx%d map, lambda %.2f: FP64 rule decided %d of %d pixels, "
              "%d handed to the redo pass" % (H, W, lam, st["fp64_checked"], H * W, redo))
        assert st["fp64_checked"] >= 0.9 * H * W


@pytest.fixture(scope="module")
def neuro_map():
    """The oracle's normalised one-band image of the 416 x 512 x 128 frame
    with probability maps independent of it (see rand_probs)."""
    f = synth.make_config(2)
    I32 = oracle.pca_one_band(f.cube)["I_norm"].astype(np.float32)
    return I32, rand_probs(4, *I32.shape, seed=2024)


@pytest.mark.parametrize("lam", [1.0, 0.5, 2.0])
def test_fast_path_neuro_full_map(hsc, ctx, neuro_map, lam):
    """Every pixel of the 416 x 512 map (K = 40, 14-row window) through the
    classifier's KNN call against the oracle; the pruned walk must have
    finished nearly all of them itself."""
    I, P = neuro_map
    H, W = I.shape
    O, lab, redo = run_knn_outputs(hsc, ctx, I, P, 40, 14, lam, 0)
    st = check_knn_outputs(I, P, 40, 14, lam, O, lab)
    print("\n416x512 map, lambda %.1f: O max error %.2e; FP64 rule decided %d of %d pixels "
          "(the rest are its near-ties); %d pixels handed to the redo pass"
          % (lam, st["o_max_err"], st["fp64_checked"], H * W, redo))
    assert st["pixels"] == H * W
    assert redo <= 0.05 * H * W
