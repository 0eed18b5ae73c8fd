"""Full-size serving workload (Poisson 2000 req/s for 2 s: uploads of 256..8192
pixel images under a 120 GiB table budget with LRU eviction, screens with radius
8..96, 1..16 scales, 2-3 features), replayed through a batched and a plain
server: every screen succeeds, both modes return the same counts, and the lists
of 12 sampled screens (two of them on images above 4096 pixels a side) equal
the oracle's key for key in both modes.  Integer results, tolerance 0.  The
latencies are the bench's concern, not asserted here."""
import argparse

import pytest

import bench

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_full_serving_stream_against_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = bench.serve_leg(argparse.Namespace(duration=2.0), [2000.0], check=True, seed=1004)
    assert r["counts_identical"]
    for mode in ("batched", "plain"):
        assert r[mode]["errors"] == 0, mode
    oc = r["oracle_check"]
    assert oc["screens_compared_with_oracle"] == 12 and oc["keys_compared"] > 0
    assert oc["lists_with_mismatch"] == 0, oc["sample"]
