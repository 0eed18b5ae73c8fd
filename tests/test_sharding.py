"""Row-band sharding of one image over ranks (the multi-GPU design), checked on
the CPU with the oracle and a gloo process group of world size 2.

Each rank owns a band of output rows and computes the screen on the image rows
of its band plus a halo of R_max + 1 rows: the square and cone four-corner
identities hold for any image, so band-local tables give exact window sums for
every window inside band + halo.  Rank 0 gathers the bands and compares them
with the whole-image result."""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import synth
    img = synth.random_image(77, 180, 150, "blobs")
    r = 9
    tmpl = img[60:60 + 2 * r + 1, 40:40 + 2 * r + 1].copy()
    tol = synth.Tolerances(Fraction(1, 4), Fraction(1, 2), Fraction(1, 2), Fraction(8))
    return img, tmpl, r, 6, [5, 7, 9, 12], 7, tol


def _band(rank, world, H):
    per = (H + world - 1) // world
    return rank * per, min(H, (rank + 1) * per)


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    img, tmpl, r, t_min, radii, feats, tol = _workload()
    H, W = img.shape
    y0, y1 = _band(rank, world, H)
    halo = max(radii) + 1
    a, b = max(0, y0 - halo), min(H, y1 + halo)
    res = oracle.screen_workload(img[a:b], tmpl, r, t_min, radii, feats, tol)
    mine = res["mask"][:, y0 - a:y1 - a, :]
    parts = [None] * world
    dist.all_gather_object(parts, (y0, y1, mine))
    if rank == 0:
        np.save(os.path.join(out_dir, "stitched.npy"),
                np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])], axis=1))
    dist.barrier()
    dist.destroy_process_group()


def test_row_band_sharding_matches_whole_image(tmp_path):
    import oracle
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    img, tmpl, r, t_min, radii, feats, tol = _workload()
    whole = oracle.screen_workload(img, tmpl, r, t_min, radii, feats, tol)["mask"]
    stitched = np.load(os.path.join(tmp_path, "stitched.npy"))
    assert whole.any()
    assert np.array_equal(stitched, whole)
