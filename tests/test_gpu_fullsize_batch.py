"""Full-size batched workload (64 images of 640x480 .. 4096x3072 x 256 templates
of radius 8..64 with 1..16 scales, every pair in one CUDA-graph run): the
complete key lists of pairs sampled over image size and template radius equal
the oracle's, per-pair counts equal the per-request path's, and every planted
copy has a survivor at a covering scale whose square overlaps the copy's by at
least 90% (the paper's success criterion, Sec. 6).  Integer results, tolerance 0."""
import argparse

import pytest

import bench

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_full_batched_workload_against_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = bench.batched_leg(argparse.Namespace(images=64, templates=256, steps=1, warmup=0), check=True)
    assert r["keys_complete"] and r["counts_identical"]
    oc = r["oracle_check"]
    assert oc["pairs_compared_with_oracle"] >= 12 and oc["keys_compared"] > 0
    assert oc["pairs_with_mismatch"] == 0, oc["sample"]
    pl = oc["plants"]
    assert pl["total"] >= 200
    # the paper's success criterion (a survivor whose square overlaps the copy's
    # by >= 90%) holds for every copy; the exact candidate for nearly all
    assert pl["survive_within_90pct_overlap"] == pl["total"], pl["not_both"]
    assert pl["survive_exact"] >= pl["total"] - 2, pl["not_both"]
