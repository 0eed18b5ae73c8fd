"""The bench's full-size batched checks (host logic, CPU only): keys that equal
the oracle's pass, a changed key or a removed plant is caught."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _batch():
    bw = synth.batch_workload(seed=51, n_images=4, n_templates=5, area_range=(60 * 45, 240 * 180),
                              r_range=(3, 10), max_scales=4, plants_per_image=2)
    keys, counts = [], []
    for p, (i, t) in enumerate(bw.pairs):
        ts = bw.templates[t]
        res = oracle.screen_workload(bw.images[i], ts.template, ts.r, max(ts.t_min, 2), ts.radii, bw.features,
                                     bw.tol)
        lst = res["list"]
        s = (lst >> np.uint64(48)) & np.uint64(0xFFFF)
        y = (lst >> np.uint64(24)) & np.uint64(0xFFFFFF)
        x = lst & np.uint64(0xFFFFFF)
        keys.append((np.uint64(p) << np.uint64(37)) | (s << np.uint64(32)) | (y << np.uint64(16)) | x)
        counts.append(len(lst))
    keys = np.concatenate(keys).astype(np.uint64)
    counts = np.array(counts, np.uint64)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.uint64)
    as_t = lambda a: torch.from_numpy(a.view(np.int64).copy())   # noqa: E731
    return bw, as_t(keys), as_t(counts), as_t(offsets)


def test_batched_checks_pass_on_oracle_keys_and_catch_changes():
    bw, keys, counts, offsets = _batch()
    r = bench.batched_checks(bw, bw.pairs, counts, offsets, keys, n_sample=8)
    assert r["pairs_compared_with_oracle"] >= 4 and r["pairs_with_mismatch"] == 0
    pl = r["plants"]
    assert pl["total"] == sum(len(p) for p in bw.plants) > 0
    # a plant the oracle keeps is reported as surviving; move its keys and it is missed
    assert pl["survive_exact"] > 0 and pl["survive_within_90pct_overlap"] >= pl["survive_exact"]
    bad = keys.clone()
    bad[:] = bad ^ 1                                            # every key moved by one column
    r2 = bench.batched_checks(bw, bw.pairs, counts, offsets, bad, n_sample=8)
    compared_nonempty = sum(1 for d in r2["sample"] if d["keys"] > 0)
    assert r2["pairs_with_mismatch"] == compared_nonempty > 0
    gone = keys | 0xFFFF                                          # every survivor moved to column 65535
    r3 = bench.batched_checks(bw, bw.pairs, counts, offsets, gone, n_sample=4)
    assert r3["plants"]["survive_exact"] == r3["plants"]["survive_within_90pct_overlap"] == 0
