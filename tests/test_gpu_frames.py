"""The frame pipeline (frames_create / frames_submit / frames_wait) against the
oracle: a synthetic video (panning scene, drifting target) screened frame by
frame with the copy of the next frame overlapping the current one's tables,
screen and compaction.  Every frame's list equals the oracle's key for key, at
every pipeline depth; the pipeline's contract errors are reported, not
faulted on.  Integer results, tolerance 0."""
import numpy as np
import pytest

import oracle
import synth
import paper_1707_05647_gb300 as scr
from paper_1707_05647_gb300 import ScreenError

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENTINEL = np.uint64(2**64 - 1)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _params(fs):
    return scr.Params(fs.radii, fs.features, fs.tol.mean_rel, fs.tol.std_rel, fs.tol.grad_rel, fs.tol.grad_abs)


def _pinned(n, dtype=torch.int64):
    return torch.full((n,), -1, dtype=dtype).pin_memory().numpy()


def _oracle_lists(fs, frames=None):
    frames = fs.frames if frames is None else frames
    return [oracle.screen_workload(f, fs.template, fs.r, fs.t_min, fs.radii, fs.features, fs.tol)["list"]
            for f in frames]


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("pinned_img", [True, False])
def test_frames_equal_the_oracle(ctx, depth, pinned_img):
    fs = synth.frame_sequence(5001, n_frames=7)
    want = _oracle_lists(fs)
    cap = max(len(w) for w in want) + 16
    tm = scr.template_features(ctx, fs.template, fs.r, fs.t_min, fs.features)
    H, W = fs.frames[0].shape
    f = scr.frames_create(ctx, H, W, fs.sum_bits, fs.sq_bits, tm, _params(fs), cap, depth)
    try:
        imgs = [torch.from_numpy(im).pin_memory().numpy() if pinned_img else im for im in fs.frames]
        lists = [_pinned(cap).view(np.uint64) for _ in range(depth)]
        got, inflight = [], []
        for k, im in enumerate(imgs):
            if len(inflight) == depth:
                t, lst = inflight.pop(0)
                n, over = scr.frames_wait(f, t)
                assert not over
                got.append(lst[:n].copy())
                lst[:] = SENTINEL
            lst = lists[k % depth]
            inflight.append((scr.frames_submit(f, im, lst), lst))
        for t, lst in inflight:
            n, over = scr.frames_wait(f, t)
            got.append(lst[:n].copy())
        assert len(got) == len(want)
        for k, (g, w) in enumerate(zip(got, want)):
            assert len(w) > 0
            assert np.array_equal(g, w), f"frame {k}: {len(g)} keys against {len(w)}"
    finally:
        scr.frames_destroy(f)
        scr.template_release(ctx, tm)


def test_frames_pitched_ragged_image(ctx):
    """Host frames with a pitch above the width and a width that is not a
    multiple of 16 or 32 (a cropped view of a wider array)."""
    fs = synth.frame_sequence(5002, n_frames=3, H=203, W=333)
    crop = 301
    frames = [np.ascontiguousarray(f)[:, :crop] for f in fs.frames]
    want = _oracle_lists(fs, [np.ascontiguousarray(f) for f in frames])
    cap = max(len(w) for w in want) + 4
    tm = scr.template_features(ctx, fs.template, fs.r, fs.t_min, fs.features)
    f = scr.frames_create(ctx, 203, crop, fs.sum_bits, fs.sq_bits, tm, _params(fs), cap, 2)
    try:
        lists = [_pinned(cap).view(np.uint64) for _ in range(3)]
        tickets = []
        for k, im in enumerate(frames):
            assert im.strides[0] == 333
            if len(tickets) == 2:
                t0, l0 = tickets.pop(0)
                n, _ = scr.frames_wait(f, t0)
                assert np.array_equal(l0[:n], want[t0])
            tickets.append((scr.frames_submit(f, im, lists[k]), lists[k]))
        for t, lst in tickets:
            n, _ = scr.frames_wait(f, t)
            assert np.array_equal(lst[:n], want[t])
    finally:
        scr.frames_destroy(f)
        scr.template_release(ctx, tm)


def test_frames_overflow_reports_true_count(ctx):
    fs = synth.frame_sequence(5003, n_frames=2)
    want = _oracle_lists(fs)
    cap = 40
    assert min(len(w) for w in want) > cap
    tm = scr.template_features(ctx, fs.template, fs.r, fs.t_min, fs.features)
    H, W = fs.frames[0].shape
    f = scr.frames_create(ctx, H, W, fs.sum_bits, fs.sq_bits, tm, _params(fs), cap, 2)
    try:
        lists = [_pinned(cap + 8).view(np.uint64) for _ in range(2)]
        ts = [scr.frames_submit(f, im, lst) for im, lst in zip(fs.frames, lists)]
        for t, lst, w in zip(ts, lists, want):
            n, over = scr.frames_wait(f, t)
            assert over and n == len(w)
            assert np.array_equal(lst[:cap], w[:cap])
            assert np.all(lst[cap:] == SENTINEL)
    finally:
        scr.frames_destroy(f)
        scr.template_release(ctx, tm)


def test_frames_count_only(ctx):
    fs = synth.frame_sequence(5001, n_frames=2)
    want = _oracle_lists(fs)
    tm = scr.template_features(ctx, fs.template, fs.r, fs.t_min, fs.features)
    H, W = fs.frames[0].shape
    f = scr.frames_create(ctx, H, W, fs.sum_bits, fs.sq_bits, tm, _params(fs), 0, 2)
    try:
        ts = [scr.frames_submit(f, im, None) for im in fs.frames]
        for t, w in zip(ts, want):
            n, over = scr.frames_wait(f, t)
            assert n == len(w) and (over == (n > 0))
    finally:
        scr.frames_destroy(f)
        scr.template_release(ctx, tm)


def test_frames_contract_errors(ctx):
    fs = synth.frame_sequence(5001, n_frames=3)
    tm = scr.template_features(ctx, fs.template, fs.r, fs.t_min, fs.features)
    H, W = fs.frames[0].shape
    p = _params(fs)
    base = scr.screen_stats(ctx)["bytes_in_use"]
    for bad in (dict(depth=0), dict(depth=5), dict(H=0), dict(W=70000)):
        kw = dict(H=H, W=W, depth=2)
        kw.update(bad)
        with pytest.raises(ScreenError) as e:
            scr.frames_create(ctx, kw["H"], kw["W"], fs.sum_bits, fs.sq_bits, tm, p, 100, kw["depth"])
        assert e.value.code == scr.SCR_EINVAL
    f = scr.frames_create(ctx, H, W, fs.sum_bits, fs.sq_bits, tm, p, 1 << 16, 2)
    try:
        assert scr.screen_stats(ctx)["bytes_in_use"] > base
        pageable = np.zeros(1 << 16, np.uint64)
        with pytest.raises(ScreenError) as e:
            scr.frames_submit(f, fs.frames[0], pageable)
        assert e.value.code == scr.SCR_EINVAL
        lists = [_pinned(1 << 16).view(np.uint64) for _ in range(3)]
        t0 = scr.frames_submit(f, fs.frames[0], lists[0])
        t1 = scr.frames_submit(f, fs.frames[1], lists[1])
        assert (t0, t1) == (0, 1)
        with pytest.raises(ScreenError) as e:   # depth 2: full
            scr.frames_submit(f, fs.frames[2], lists[2])
        assert e.value.code == scr.SCR_EINVAL
        with pytest.raises(ScreenError) as e:   # not the oldest
            scr.frames_wait(f, t1)
        assert e.value.code == scr.SCR_EINVAL
        scr.frames_wait(f, t0)
        t2 = scr.frames_submit(f, fs.frames[2], lists[0])
        assert t2 == 2
        # destroy with two frames in flight: it waits for them
    finally:
        scr.frames_destroy(f)
    assert scr.screen_stats(ctx)["bytes_in_use"] == base
    scr.template_release(ctx, tm)


def test_shutdown_frees_live_pipelines():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    fs = synth.frame_sequence(5002, n_frames=1)
    tm = scr.template_features(c, fs.template, fs.r, fs.t_min, fs.features)
    H, W = fs.frames[0].shape
    f = scr.frames_create(c, H, W, fs.sum_bits, fs.sq_bits, tm, _params(fs), 1 << 14, 2)
    lst = _pinned(1 << 14).view(np.uint64)
    scr.frames_submit(f, fs.frames[0], lst)
    scr.screen_shutdown(c)   # frees the pipeline after its frame completes


def test_frames_full_size_against_the_oracle():
    """Configuration 2 (4096 x 4096, 8 scales, u32/u64 tables) as a three-frame
    stream (the image, its mirror image, the image again) through a depth-2
    pipeline: every frame's complete list equals the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.config2()
    frames = [wl.image, np.ascontiguousarray(wl.image[:, ::-1]), wl.image]
    ref = {}
    for k in (0, 1):
        ref[k] = oracle.screen_workload(frames[k], wl.template, wl.r, wl.t_min, wl.radii, wl.features,
                                        wl.tol)["list"]
    want = [ref[0], ref[1], ref[0]]
    cap = max(len(w) for w in want) + 64
    c = scr.screen_init(0, 0)
    try:
        tm = scr.template_features(c, wl.template, wl.r, wl.t_min, wl.features)
        p = scr.Params(wl.radii, wl.features, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel, wl.tol.grad_abs)
        H, W = wl.image.shape
        f = scr.frames_create(c, H, W, wl.sum_bits, wl.sq_bits, tm, p, cap, 2)
        imgs = [torch.from_numpy(im).pin_memory().numpy() for im in frames]
        lists = [_pinned(cap).view(np.uint64) for _ in range(3)]
        t0 = scr.frames_submit(f, imgs[0], lists[0])
        t1 = scr.frames_submit(f, imgs[1], lists[1])
        n0, _ = scr.frames_wait(f, t0)
        t2 = scr.frames_submit(f, imgs[2], lists[2])
        n1, _ = scr.frames_wait(f, t1)
        n2, _ = scr.frames_wait(f, t2)
        for n, lst, w in zip((n0, n1, n2), lists, want):
            assert n == len(w)
            assert np.array_equal(lst[:n], w)
        scr.frames_destroy(f)
    finally:
        scr.screen_shutdown(c)
