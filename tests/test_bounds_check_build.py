"""The debug build with index checks (-DHSC_BOUNDS_CHECK): the translation
units whose kernels carry the checks compile with them (CPU), and on the GPU
the checked library gives the normal library's outputs with every check
passing (the status word stays clear)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import json, os, sys
sys.path.insert(0, %r)
import numpy as np, torch
import paper_2404_10631_gb300 as hsc
import synth
out = {}
for cfg in (1, 2):
    f = synth.make_config(cfg)
    ctx = hsc.Context(0)
    c = torch.as_tensor(f.cube, device="cuda")
    m = hsc.Model.from_host(f.model)
    k = f.model.n_classes
    O = torch.empty((k,) + f.cube.shape[1:], device="cuda")
    lab = hsc.hsc_classify(ctx, c, m, f.K, f.window_rows, f.lam, out_probs=O)
    ctx.sync()
    out[cfg] = [int(v) for v in lab.cpu().numpy().ravel()[::97]] + [float(O.sum())]
    ctx.close()
print(json.dumps(out))
"""


def test_checked_translation_units_compile():
    from paper_2404_10631_gb300 import build
    out = build.build(bounds_check=True, sources_only=("k_knn.cu", "k_gram_tc.cu"))
    for name in ("k_knn.o", "k_gram_tc.o"):
        assert os.path.exists(os.path.join(out, name))


@pytest.mark.gpu
def test_checked_build_matches_and_passes_its_checks(hsc):
    from paper_2404_10631_gb300 import build
    lib = build.build(bounds_check=True)
    res = {}
    for name, path in (("checked", lib), ("normal", build.LIB)):
        env = dict(os.environ, HSC_LIBRARY=path)
        r = subprocess.run([sys.executable, "-c", RUN % ROOT], env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[name] = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["checked"] == res["normal"]
