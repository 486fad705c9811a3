"""hsc_server_*: continuous batching of requests with host cubes.

Every result must be bit-identical to hsc_classify on the same frame, both
when the request runs alone and when it shares the GPU with others; the HBM
budget must bound what admitted requests hold; a failing request must not
disturb the others."""

import numpy as np
import pytest

import synth
from parity import e2e_labels, sample_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    # snapshot cubes plus pushbroom cubes at a quarter of their size, each
    # with its own model and K
    return synth.make_serving_pool(n_snapshot=10, n_pushbroom=3, pushbroom_scale=0.25)


def pinned(a):
    import torch
    t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
    t.numpy()[...] = a
    return t


def reference(hsc, ctx, f, model):
    """hsc_classify on the device, the result every server request must equal."""
    import torch
    cube = torch.as_tensor(f.cube, device="cuda")
    k = f.model.n_classes
    lab = torch.empty(f.cube.shape[1:], dtype=torch.int32, device="cuda")
    O = torch.empty((k,) + f.cube.shape[1:], device="cuda")
    hsc.hsc_classify(ctx, cube, model, f.K, f.window_rows, f.lam, labels=lab, out_probs=O)
    ctx.sync()
    return lab.cpu().numpy(), O.cpu().numpy()


def outputs(f):
    k = f.model.n_classes
    lab = pinned(np.full(f.cube.shape[1:], -1, np.int32))
    O = pinned(np.full((k,) + f.cube.shape[1:], -1.0, np.float32))
    return lab, O


def test_server_same_alone_and_in_mix(hsc, ctx, pool):
    models = [hsc.Model.from_host(f.model) for f in pool]
    cubes = [pinned(f.cube) for f in pool]
    ref = [reference(hsc, ctx, f, m) for f, m in zip(pool, models)]
    with hsc.Server(0, max_inflight=8) as srv:
        # alone: one request on the GPU at a time
        for i, f in enumerate(pool):
            lab, O = outputs(f)
            srv.wait(srv.submit(cubes[i], models[i], f.K, f.window_rows, f.lam, lab, O))
            np.testing.assert_array_equal(lab.numpy(), ref[i][0])
            np.testing.assert_array_equal(O.numpy(), ref[i][1])
        # in the mix: every request submitted before any completes, twice over
        order = list(range(len(pool))) * 2
        outs = [outputs(pool[i]) for i in order]
        tickets = [srv.submit(cubes[i], models[i], pool[i].K, pool[i].window_rows, pool[i].lam,
                              *outs[j]) for j, i in enumerate(order)]
        for t in tickets:
            assert srv.wait(t) > 0.0
        for j, i in enumerate(order):
            np.testing.assert_array_equal(outs[j][0].numpy(), ref[i][0])
            np.testing.assert_array_equal(outs[j][1].numpy(), ref[i][1])
        st = srv.stats()
        n = len(pool) + len(order)
        assert st["submitted"] == n and st["completed"] == n and st["failed"] == 0
        assert st["pixels"] == sum(int(np.prod(pool[i].cube.shape[1:]))
                                   for i in list(range(len(pool))) + order)
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert 1 < st["peak_inflight"] <= 8  # the mix did overlap on the GPU


def test_server_budget_bounds_admission(hsc, pool):
    snaps = pool[:6]
    models = [hsc.Model.from_host(f.model) for f in snaps]
    cubes = [pinned(f.cube) for f in snaps]
    budget = 3 << 20  # below any quarter-size pushbroom cube (>= 3.9 MB)
    with hsc.Server(0, hbm_budget_bytes=budget, max_inflight=8) as srv:
        outs = [outputs(f) for f in snaps]
        tickets = [srv.submit(cubes[i], models[i], f.K, f.window_rows, f.lam, *outs[i])
                   for i, f in enumerate(snaps)]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
        assert st["completed"] == len(snaps)
        assert 0 < st["peak_bytes"] <= budget
        # a request that alone exceeds the budget is refused at submit
        big = pool[-1]
        with pytest.raises(hsc.HscError) as e:
            srv.submit(pinned(big.cube), hsc.Model.from_host(big.model), big.K, big.window_rows,
                       big.lam, *outputs(big))
        assert e.value.status == hsc.HSC_ERR_OOM


def test_server_failed_request_is_isolated(hsc, ctx, pool):
    f = pool[0]
    model = hsc.Model.from_host(f.model)
    bad = f.cube.copy()
    bad[3, 5, 7] = np.nan
    ref = reference(hsc, ctx, f, model)
    with hsc.Server(0, max_inflight=4) as srv:
        o1, o2, o3 = outputs(f), outputs(f), outputs(f)
        t1 = srv.submit(pinned(f.cube), model, f.K, f.window_rows, f.lam, *o1)
        t2 = srv.submit(pinned(bad), model, f.K, f.window_rows, f.lam, *o2)
        t3 = srv.submit(pinned(f.cube), model, f.K, f.window_rows, f.lam, *o3)
        srv.wait(t1)
        with pytest.raises(hsc.HscError) as e:
            srv.wait(t2)
        assert e.value.status == hsc.HSC_ERR_NONFINITE
        srv.wait(t3)
        for o in (o1, o3):
            np.testing.assert_array_equal(o[0].numpy(), ref[0])
            np.testing.assert_array_equal(o[1].numpy(), ref[1])
        st = srv.stats()
        assert st["completed"] == 2 and st["failed"] == 1


def test_server_rejects_bad_requests(hsc, pool):
    f = pool[0]
    model = hsc.Model.from_host(f.model)
    with hsc.Server(0, max_inflight=2) as srv:
        lab, O = outputs(f)
        with pytest.raises(hsc.HscError):  # K above the smallest window
            srv.submit(pinned(f.cube), model, 10 ** 6, f.window_rows, f.lam, lab, O)
        with pytest.raises(hsc.HscError):  # model for another band count
            srv.submit(pinned(f.cube[:100].copy()), model, f.K, f.window_rows, f.lam, lab, O)
        with pytest.raises(hsc.HscError):  # unknown ticket
            srv.wait(12345)
    with pytest.raises(hsc.HscError):
        hsc.Server(0, max_inflight=0)


def test_server_full_size_pushbroom_against_oracle(hsc):
    """Two full-size pushbroom requests of the serving stream (128 bands,
    H 384-640 x W 320-512, their own models and K) in the mix with snapshot
    requests: labels and O read back to the host checked against the FP64
    oracle on rows at both edges and inside (near-tie margin for a one-band
    image within 2e-5 of the oracle's, the bound the PCA tests assert)."""
    full = synth.make_serving_pool()
    push = [f for f in full if f.cube.shape[0] == 128][:2]
    snaps = full[:6]
    assert all(f.cube.shape[1] >= 384 and f.cube.shape[2] >= 320 for f in push)
    reqs = push + snaps
    models = [hsc.Model.from_host(f.model) for f in reqs]
    cubes = [pinned(f.cube) for f in reqs]
    with hsc.Server(0, max_inflight=8) as srv:
        outs = [outputs(f) for f in reqs]
        tickets = [srv.submit(cubes[i], models[i], f.K, f.window_rows, f.lam, *outs[i])
                   for i, f in enumerate(reqs)]
        for t in tickets:
            srv.wait(t)
    for i, f in enumerate(push):
        _, H, W = f.cube.shape
        lab, O = outs[i][0].numpy(), outs[i][1].numpy()
        rows = [0, 1, 6, 7, H // 3, H // 2, H - 8, H - 7, H - 1]
        n, agree, ties = e2e_labels(f, lab, O, 2e-5, sample_rows(H, W, rows))
        print("\npushbroom %dx%d K=%d: %d pixels, %d labels agree, %d near-ties"
              % (H, W, f.K, n, agree, ties))
        assert agree >= n - ties
        assert (lab == f.truth).mean() > 0.99
