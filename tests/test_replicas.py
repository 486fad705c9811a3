"""The multi-GPU form of the path (replicas: one process per GPU, each on its
own frames, no data-path exchange) on two CPU ranks over gloo.

The helpers in paper_2404_10631_gb300.replicas are what bench.py runs under
torchrun (there over NCCL): the barrier around a timed region, the maximum
of the ranks' times, the whole-job rate, and which rank reports. Each rank
here also runs one replica step of the tiny frame through the FP64 oracle
(standing in for the GPU path, which needs a GPU) and the job's rate is
formed the way bench.py forms it."""

import json
import os
import socket
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2404_10631_gb300 import replicas
    import oracle
    import synth

    w, r, lr = replicas.env_ranks()
    replicas.init(w, lr, backend="gloo")
    res = {"env": [w, r, lr]}
    # the slowest rank's time, element by element
    res["max"] = replicas.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5], w)
    # a replica step: this rank's frame through the whole path, timed between
    # two barriers like bench.py's timed region
    f = synth.make_config(1)
    B, H, W = f.cube.shape
    replicas.barrier(w)
    t0 = time.perf_counter()
    out = oracle.classify(f.cube, f.model, f.K, f.window_rows, f.lam)
    dt = time.perf_counter() - t0
    replicas.barrier(w)
    (dt_max,) = replicas.max_over_ranks([dt], w)
    res["dt"] = dt
    res["dt_max"] = dt_max
    res["rate"] = replicas.whole_job_rate(H * W, w, dt_max)
    res["labels"] = out["labels"].astype(int).ravel().tolist()
    res["reports"] = replicas.reports(rank)
    if rank == 1:
        # the reference arm on a rank other than 0 returns without work or output
        import contextlib
        import io
        import bench
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            t1 = time.perf_counter()
            bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "gpus": w})(), f)
            res["ref_seconds"] = time.perf_counter() - t1
        res["ref_output"] = buf.getvalue()
    replicas.finalize(w)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as fh:
        json.dump(res, fh)


@pytest.mark.timeout(300)
def test_two_gloo_ranks_run_replicas(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r, d in enumerate(res):
        assert d["env"] == [world, r, r]
        assert d["max"] == [2.0, 10.0, 0.5]
        assert d["reports"] == (r == 0)
        # every rank sees the slowest rank's time
        assert d["dt_max"] == max(x["dt"] for x in res)
        # weak scaling: both ranks' pixels over the slowest rank's time
        assert d["rate"] == pytest.approx(2 * 32 * 32 / d["dt_max"], rel=1e-12)
    # replicas of the same frame give the same labels
    assert res[0]["labels"] == res[1]["labels"]
    assert len(set(res[0]["labels"])) > 1
    assert res[1]["ref_output"] == "" and res[1]["ref_seconds"] < 5.0


def test_single_rank_helpers_need_no_process_group():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2404_10631_gb300 import replicas
    replicas.init(1)
    replicas.barrier(1)
    assert replicas.max_over_ranks([3, 1.5], 1) == [3.0, 1.5]
    assert replicas.whole_job_rate(212992 * 64, 1, 0.5) == pytest.approx(212992 * 128)
    assert replicas.whole_job_rate(10, 4, 2.0) == 20.0
    with pytest.raises(ValueError):
        replicas.whole_job_rate(10, 1, 0.0)
    assert replicas.reports(0) and not replicas.reports(3)
    replicas.finalize(1)
    assert np.isfinite(replicas.whole_job_rate(1, 1, 1e-9))
