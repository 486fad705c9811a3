"""Summaries of ncu CSV logs for the profiles folder.

    python ncu_summary.py launches LOG.csv
        per kernel: launches, total time, time per launch, share (markdown)
    python ncu_summary.py traffic LOG.csv STAGE_LAUNCHES HxWxB [FIRST-LAST]
        per pipeline stage: DRAM bytes (read + write) per stage launch, as
        "stage source_sha bytes HxWxB" lines (the format bench.py reads), with
        STAGE_LAUNCHES the number of times each stage ran in the captured
        launches counted (all of them, or the capture's launch IDs FIRST to
        LAST) and HxWxB the frame it ran on

LOG.csv comes from ``ncu --csv --log-file LOG.csv --metrics ...``.
"""

from __future__ import annotations

import collections
import csv
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))

# kernel name prefix -> pipeline stage, and the source file each stage's
# kernels live in (its hash tags the numbers with the code they measured)
STAGE_OF = (("pilot_", "moments"), ("gram_tc_kernel", "moments"),
            ("gram_tc_items_kernel", "moments"), ("gram_tc_wide_kernel", "moments"),
            ("gram_partial_kernel", "moments"),
            ("gram_reduce_kernel", "moments"), ("jacobi_kernel", "jacobi"),
            ("jacobi_cluster_kernel", "jacobi"),
            ("project_svm_kernel", "project_svm"), ("project_svm_batch_kernel", "project_svm"),
            ("normalize_kernel", "normalize"), ("normalize_batch_kernel", "normalize"),
            ("knn_pruned_kernel", "knn"), ("knn_redo_kernel", "knn"),
            ("svm_knn_batch_kernel", "knn"),
            ("knn_redo_batch_kernel", "knn"), ("knn_kernel", "knn_full"))
SOURCE_OF = {"moments": ("k_moments.cu", "k_gram_tc.cu", "dfloat.cuh"),
             "jacobi": ("k_jacobi.cu", "k_jacobi_cluster.cu", "jacobi_rot.cuh", "dfloat.cuh"),
             "project_svm": ("k_project_svm.cu", "svm_pixel.cuh"),
             "normalize": ("k_project_svm.cu", "svm_pixel.cuh"),
             "knn": ("k_knn.cu", "svm_pixel.cuh"), "knn_full": ("k_knn.cu", "svm_pixel.cuh")}


def source_sha(stage: str) -> str:
    h = hashlib.sha256()
    for f in SOURCE_OF[stage]:
        h.update(open(os.path.join(HERE, "paper_2404_10631_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_base(name: str) -> str:
    """'void (anonymous namespace)::knn_kernel<16>(...)' -> 'knn_kernel<16>'"""
    n = name.split("(")[0] if "(" in name and not name.startswith("(") else name
    n = n.replace("void ", "")
    if "::" in n:
        n = n.split("::")[-1]
    return n.strip()


def read(path: str):
    rows = [r for r in csv.reader(open(path)) if len(r) > 5]
    hdr = rows[0]
    ki, mi, vi = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value")
    idi = hdr.index("ID")
    launches = collections.OrderedDict()
    for r in rows[1:]:
        key = int(r[idi])
        d = launches.setdefault(key, {"kernel": kernel_base(r[ki]), "id": key})
        d[r[mi]] = float(r[vi].replace(",", ""))
    return list(launches.values())


def stage_of(kernel: str):
    for prefix, st in STAGE_OF:
        if kernel.startswith(prefix):
            return st
    return None


def launches_table(path: str) -> str:
    tot = collections.OrderedDict()
    cnt = collections.Counter()
    for d in read(path):
        t = d.get("gpu__time_duration.sum")
        if t is None:
            continue
        tot[d["kernel"]] = tot.get(d["kernel"], 0.0) + t
        cnt[d["kernel"]] += 1
    all_t = sum(tot.values())
    out = ["| kernel | launches | total us | us / launch | share |", "|---|---|---|---|---|"]
    for k, t in sorted(tot.items(), key=lambda x: -x[1]):
        out.append("| %s | %d | %.1f | %.1f | %.1f%% |" % (k, cnt[k], t / 1e3, t / 1e3 / cnt[k],
                                                          100.0 * t / all_t))
    return "\n".join(out)


def traffic_lines(path: str, stage_launches: int, tag: str, ids=None) -> str:
    tot = collections.defaultdict(float)
    for d in read(path):
        if ids is not None and not ids[0] <= d["id"] <= ids[1]:
            continue
        st = stage_of(d["kernel"])
        if st is None:
            continue
        tot[st] += d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0)
    return "\n".join("%s %s %.0f %s" % (st, source_sha(st), b / stage_launches, tag)
                     for st, b in sorted(tot.items()))


def main(argv):
    if len(argv) >= 2 and argv[0] == "launches":
        print(launches_table(argv[1]))
    elif len(argv) >= 4 and argv[0] == "traffic":
        ids = tuple(int(v) for v in argv[4].split("-")) if len(argv) >= 5 else None
        print(traffic_lines(argv[1], int(argv[2]), argv[3], ids))
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
