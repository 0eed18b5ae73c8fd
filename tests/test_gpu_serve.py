"""Serving loop: every screen's list against the oracle; a request served alone,
mixed into a batch of others, and in plain (one launch pair per request) mode
gives the same bytes; LRU eviction under a table budget and rebuild from the
host copy; forgotten images; list overflow; budget errors.  Integer results,
tolerance 0."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
import paper_1707_05647_gb300 as scr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = synth.Tolerances(Fraction(1, 6), Fraction(1, 3), Fraction(1, 3), Fraction(8))
FEATS = [3, 7, 1, 7, 5]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


@pytest.fixture(scope="module")
def work(ctx):
    bw = synth.batch_workload(seed=41, n_images=4, n_templates=5, area_range=(60 * 45, 400 * 300),
                              r_range=(3, 18), max_scales=5, plants_per_image=2)
    tmpls, params = [], []
    for t, ts in enumerate(bw.templates):
        tmpls.append(scr.template_features(ctx, ts.template, ts.r, max(ts.t_min, 2), 7))
        params.append(scr.Params(ts.radii, FEATS[t % len(FEATS)], TOL.mean_rel, TOL.std_rel, TOL.grad_rel,
                                 TOL.grad_abs))
    tabs = [oracle.Tables(im) for im in bw.images]
    want = {}
    for i in range(len(bw.images)):
        for t, ts in enumerate(bw.templates):
            res = oracle.screen_workload(bw.images[i], ts.template, ts.r, max(ts.t_min, 2), list(ts.radii),
                                         FEATS[t % len(FEATS)], TOL, tables=tabs[i])
            want[(i, t)] = res["list"].astype(np.uint64)
    return bw, tmpls, params, want


def _serve(ctx, bw, tmpls, params, requests, mode=scr.SERVE_BATCHED, held=True, cap=1 << 16, **kw):
    """Upload every image, queue the (image, template) screens (while held, so
    they form one batch), release, collect."""
    s = scr.server_create(ctx, mode=mode, **kw)
    try:
        ids = []
        for im in bw.images:
            iid, rid = scr.server_upload(s, im)
            assert scr.server_wait(s, rid)["status"] == scr.SCR_OK
            ids.append(iid)
        if held:
            scr.server_hold(s, True)
        rids, bufs = [], []
        for (i, t) in requests:
            buf = np.zeros(cap, np.uint64)
            rids.append(scr.server_screen(s, ids[i], tmpls[t], params[t], buf))
            bufs.append(buf)
        scr.server_hold(s, False)
        out = []
        for rid, buf in zip(rids, bufs):
            r = scr.server_wait(s, rid, 60_000_000)
            out.append((r, buf[:min(r["count"], cap)].copy()))
        return out, scr.server_stats(s)
    finally:
        scr.server_destroy(s)


def test_every_screen_matches_the_oracle_in_one_batch(ctx, work):
    bw, tmpls, params, want = work
    reqs = [(i, t) for i in range(len(bw.images)) for t in range(len(bw.templates))]
    out, st = _serve(ctx, bw, tmpls, params, reqs)
    assert st["batches"] >= 1
    sizes = {r["batch_size"] for r, _ in out}
    assert max(sizes) >= len(reqs)            # served together
    for (i, t), (r, lst) in zip(reqs, out):
        assert r["status"] == scr.SCR_OK
        assert r["count"] == len(want[(i, t)])
        assert np.array_equal(lst, want[(i, t)])


def test_alone_mixed_and_plain_are_identical(ctx, work):
    bw, tmpls, params, want = work
    probe = (2, 3)
    alone, _ = _serve(ctx, bw, tmpls, params, [probe])
    mix = [(0, 1), (2, 3), (1, 4), (3, 0), (2, 3), (0, 2), (1, 1)]
    mixed, _ = _serve(ctx, bw, tmpls, params, mix)
    plain, st = _serve(ctx, bw, tmpls, params, mix, mode=scr.SERVE_PLAIN)
    assert alone[0][0]["batch_size"] == 1 and mixed[1][0]["batch_size"] == len(mix)
    for k in (1, 4):
        assert np.array_equal(mixed[k][1], alone[0][1])
    for (i, t), (rb, lb), (rp, lp) in zip(mix, mixed, plain):
        assert rb["count"] == rp["count"] == len(want[(i, t)])
        assert np.array_equal(lb, lp) and np.array_equal(lb, want[(i, t)])
    assert st["launches"] > 0


def test_unheld_stream_of_requests(ctx, work):
    """Requests submitted while the worker is running form several batches."""
    bw, tmpls, params, want = work
    reqs = [(k % 4, (3 * k) % 5) for k in range(40)]
    out, st = _serve(ctx, bw, tmpls, params, reqs, held=False, max_batch=6)
    assert st["batches"] >= 40 // 6
    for (i, t), (r, lst) in zip(reqs, out):
        assert r["status"] == scr.SCR_OK and r["batch_size"] <= 6
        assert r["arrival_ns"] <= r["start_ns"] <= r["done_ns"]
        assert np.array_equal(lst, want[(i, t)])


def test_lru_eviction_and_rebuild(ctx, work):
    bw, tmpls, params, want = work
    sizes = [scr_table_bytes(im.shape) for im in bw.images]
    budget = sizes[0] + sizes[1] + 4096          # room for images 0 and 1 only
    s = scr.server_create(ctx, table_budget_bytes=budget)
    try:
        ids = []
        for im in bw.images[:2]:
            iid, rid = scr.server_upload(s, im)
            assert scr.server_wait(s, rid)["status"] == scr.SCR_OK
            ids.append(iid)
        assert scr.server_resident(s, ids[0]) and scr.server_resident(s, ids[1])
        # touch image 0 so image 1 is the least recently used
        buf = np.zeros(1 << 16, np.uint64)
        r = scr.server_wait(s, scr.server_screen(s, ids[0], tmpls[0], params[0], buf))
        assert r["status"] == scr.SCR_OK and r["built"] == 0
        if sizes[2] <= sizes[1] + 4096:
            iid, rid = scr.server_upload(s, bw.images[2])
            assert scr.server_wait(s, rid)["status"] == scr.SCR_OK
            assert not scr.server_resident(s, ids[1]) and scr.server_resident(s, ids[0])
            assert scr.server_stats(s)["evictions"] >= 1
        else:
            rid = scr.server_evict(s, ids[1])
            assert scr.server_wait(s, rid)["status"] == scr.SCR_OK
            assert not scr.server_resident(s, ids[1])
        # a screen on the evicted image rebuilds its tables from the host copy
        r = scr.server_wait(s, scr.server_screen(s, ids[1], tmpls[1], params[1], buf))
        assert r["status"] == scr.SCR_OK and r["built"] == 1
        assert np.array_equal(buf[:r["count"]], want[(1, 1)])
        st = scr.server_stats(s)
        assert st["rebuilds"] >= 1 and st["resident_bytes"] <= budget
    finally:
        scr.server_destroy(s)


def test_forget_overflow_and_budget_errors(ctx, work):
    bw, tmpls, params, want = work
    # room for the tables of image 0 or image 1, one at a time
    budget = max(scr_table_bytes(bw.images[0].shape), scr_table_bytes(bw.images[1].shape)) + 4096
    s = scr.server_create(ctx, start_held=True, table_budget_bytes=budget)
    try:
        i0, _ = scr.server_upload(s, bw.images[0])
        small = np.zeros(3, np.uint64)
        rid = scr.server_screen(s, i0, tmpls[0], params[0], small)
        second = scr.server_screen(s, i0, tmpls[1], params[1], np.zeros(16, np.uint64))
        big = np.zeros((1200, 1600), np.uint8)                 # tables larger than the budget
        _, rbig = scr.server_upload(s, big)
        scr.server_hold(s, False)
        r = scr.server_wait(s, rid)
        n = len(want[(0, 0)])
        assert r["count"] == n
        assert r["status"] == (scr.SCR_EOVERFLOW if n > 3 else scr.SCR_OK)
        assert np.array_equal(small[:min(n, 3)], want[(0, 0)][:3])
        assert scr.server_wait(s, second)["status"] in (scr.SCR_OK, scr.SCR_EOVERFLOW)
        assert scr.server_wait(s, rbig)["status"] == scr.SCR_EBUDGET
        scr.server_forget(s, i0)
        with pytest.raises(scr.ScreenError) as e:
            scr.server_screen(s, i0, tmpls[0], params[0], small)
        assert e.value.code == scr.SCR_EEVICTED
        # forgotten while a screen on it is queued: that screen reports SCR_EEVICTED
        i1, rup = scr.server_upload(s, bw.images[1])
        assert scr.server_wait(s, rup)["status"] == scr.SCR_OK
        scr.server_hold(s, True)
        q = scr.server_screen(s, i1, tmpls[0], params[0], small)
        scr.server_forget(s, i1)
        scr.server_hold(s, False)
        assert scr.server_wait(s, q)["status"] == scr.SCR_EEVICTED
        with pytest.raises(scr.ScreenError):
            scr.server_wait(s, q)                               # already collected
    finally:
        scr.server_destroy(s)


def scr_table_bytes(shape, sum_bits=32, sq_bits=64):
    """Device bytes the server charges for one image's four tables: (H + 1) rows
    at the padded pitch per u32 plane, one plane per 32 bits (the library's
    layout; a multiple of 256 bytes)."""
    H, W = shape
    pitch = ((W + 16 + 31) // 32) * 32
    plane = (((H + 1) * pitch + 63) // 64) * 64
    return plane * 4 * (2 * (sum_bits // 32) + 2 * (sq_bits // 32))


def test_completion_queue_returns_each_request_once(ctx, work):
    bw, tmpls, params, want = work
    s = scr.server_create(ctx, max_batch=3)
    try:
        ids = []
        for im in bw.images:
            iid, rid = scr.server_upload(s, im)
            ids.append(iid)
        reqs, bufs = {}, {}
        for k in range(12):
            i, t = k % 4, (2 * k) % 5
            buf = np.zeros(1 << 16, np.uint64)
            rid = scr.server_screen(s, ids[i], tmpls[t], params[t], buf)
            reqs[rid], bufs[rid] = (i, t), buf
        seen = []
        for _ in range(len(reqs) + len(bw.images)):
            rid, r = scr.server_next(s, 60_000_000)
            seen.append(rid)
            if rid in reqs:
                i, t = reqs[rid]
                assert r["status"] == scr.SCR_OK and r["kind"] == 1
                assert np.array_equal(bufs[rid][:r["count"]], want[(i, t)])
            else:
                assert r["kind"] == 0                       # the uploads
        assert len(set(seen)) == len(seen) and set(reqs) <= set(seen)
        with pytest.raises(scr.ScreenError) as e:
            scr.server_next(s, 1000)
        assert e.value.code == scr.SCR_ETIMEOUT
    finally:
        scr.server_destroy(s)


def test_concurrent_clients(ctx, work):
    """Four client threads upload and screen at once, one collector drains the
    completion queue; every list equals the oracle's."""
    import threading
    bw, tmpls, params, want = work
    s = scr.server_create(ctx, max_batch=5)
    try:
        ids = {}
        for i, im in enumerate(bw.images):
            iid, rid = scr.server_upload(s, im)
            assert scr.server_wait(s, rid)["status"] == scr.SCR_OK
            ids[i] = iid
        lock = threading.Lock()
        submitted, errors = {}, []

        def client(c):
            try:
                for k in range(15):
                    i, t = (c + k) % 4, (c * 3 + k) % 5
                    buf = np.zeros(1 << 16, np.uint64)
                    rid = scr.server_screen(s, ids[i], tmpls[t], params[t], buf)
                    with lock:
                        submitted[rid] = (i, t, buf)
            except Exception as e:   # surfaced below
                errors.append(e)

        threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errors
        got = {}
        for _ in range(len(submitted)):
            rid, r = scr.server_next(s, 60_000_000)
            got[rid] = r
        assert set(got) == set(submitted)
        for rid, (i, t, buf) in submitted.items():
            r = got[rid]
            assert r["status"] == scr.SCR_OK
            assert np.array_equal(buf[:r["count"]], want[(i, t)])
    finally:
        scr.server_destroy(s)
