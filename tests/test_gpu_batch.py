"""Batched screening (many images x many templates in one persistent launch):
every pair's survivor list, the per-pair counts and offsets, and the per-image
union mask against the oracle run pair by pair.  Integer results, tolerance 0."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
import paper_1707_05647_gb300 as scr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FEATURE_SETS = [7, 7, 3, 1, 5, 2, 6]
TOLS = [synth.Tolerances(),
        synth.Tolerances(Fraction(1, 6), Fraction(1, 3), Fraction(1, 3), Fraction(8)),
        synth.Tolerances(Fraction(1, 10), Fraction(1, 5), Fraction(1, 5), Fraction(6))]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _setup(ctx, seed, n_images, n_templates, pairs=None):
    bw = synth.batch_workload(seed=seed, n_images=n_images, n_templates=n_templates,
                              area_range=(40 * 30, 480 * 360), r_range=(3, 20), max_scales=6,
                              plants_per_image=2)
    pairs = pairs if pairs is not None else bw.pairs
    feats = [FEATURE_SETS[t % len(FEATURE_SETS)] for t in range(n_templates)]
    tols = [TOLS[t % len(TOLS)] for t in range(n_templates)]
    tables = [scr.build_tables(ctx, torch.from_numpy(im).cuda(), 32, 64) for im in bw.images]
    tmpls, params = [], []
    for t, ts in enumerate(bw.templates):
        tmin = max(ts.t_min, 2)
        tmpls.append(scr.template_features(ctx, ts.template, ts.r, tmin, 7))
        params.append(scr.Params(ts.radii, feats[t], tols[t].mean_rel, tols[t].std_rel,
                                 tols[t].grad_rel, tols[t].grad_abs))
    return bw, pairs, feats, tols, tables, tmpls, params


def _oracle(bw, pairs, feats, tols):
    keys, counts, unions = [], [], [np.zeros((im.shape[0], (im.shape[1] + 31) // 32), np.uint32)
                                    for im in bw.images]
    tabs = [oracle.Tables(im) for im in bw.images]
    for p, (i, t) in enumerate(pairs):
        ts = bw.templates[t]
        radii = [R for R in ts.radii]
        res = oracle.screen_workload(bw.images[i], ts.template, ts.r, max(ts.t_min, 2), radii, feats[t], tols[t],
                                     tables=tabs[i])
        lst = res["list"]
        s = (lst >> np.uint64(48)) & np.uint64(0xFFFF)
        y = (lst >> np.uint64(24)) & np.uint64(0xFFFFFF)
        x = lst & np.uint64(0xFFFFFF)
        keys.append((np.uint64(p) << np.uint64(37)) | (s << np.uint64(32)) | (y << np.uint64(16)) | x)
        counts.append(res["count"])
        unions[i] |= np.bitwise_or.reduce(res["mask"], axis=0)
    return np.concatenate(keys) if keys else np.zeros(0, np.uint64), np.array(counts, np.uint64), unions


def _run(ctx, bw, pairs, tables, tmpls, params, cap, tuning=None):
    n = len(pairs)
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    offsets = torch.zeros(n, dtype=torch.int64, device="cuda")
    uw = sum(im.shape[0] * ((im.shape[1] + 31) // 32) for im in bw.images)
    union = torch.zeros(uw, dtype=torch.int32, device="cuda")
    keys = torch.zeros(cap, dtype=torch.int64, device="cuda")
    nk = torch.zeros(2, dtype=torch.int64, device="cuda")
    b = scr.screen_batch_create(ctx, tables, tmpls, params, pairs, counts, keys, nk, offsets=offsets,
                                union_mask=union, tuning=tuning)
    return b, counts, offsets, union, keys, nk


def _check(bw, got, want):
    b, counts, offsets, union, keys, nk = got
    wkeys, wcounts, wunions = want
    torch.cuda.synchronize()
    n, slots = int(nk[0].item()), int(nk[1].item())
    assert n == len(wkeys)
    assert n <= slots <= keys.numel()
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), wcounts)
    off = np.concatenate([[0], np.cumsum(wcounts)[:-1]]).astype(np.uint64)
    assert np.array_equal(offsets.cpu().numpy().view(np.uint64), off)
    assert np.array_equal(keys[:n].cpu().numpy().view(np.uint64), wkeys)
    u = union.cpu().numpy().view(np.uint32)
    o = 0
    for wu in wunions:
        assert np.array_equal(u[o:o + wu.size].reshape(wu.shape), wu)
        o += wu.size


def test_batch_matches_oracle_pair_by_pair(ctx):
    bw, pairs, feats, tols, tables, tmpls, params = _setup(ctx, 31, 5, 7)
    want = _oracle(bw, pairs, feats, tols)
    assert len(want[0]) > 0
    got = _run(ctx, bw, pairs, tables, tmpls, params, cap=1 << 22)
    scr.screen_batch_run(got[0])
    _check(bw, got, want)
    info = scr.screen_batch_info(got[0])
    assert info["n_records"] > 0 and info["candidates"] > 0
    scr.screen_batch_run(got[0])          # graph replay gives the same result
    _check(bw, got, want)
    scr.screen_batch_release(ctx, got[0])


@pytest.mark.parametrize("wpw", [2, 4, 8])
def test_batch_every_launch_shape(ctx, wpw):
    bw, pairs, feats, tols, tables, tmpls, params = _setup(ctx, 32, 3, 5)
    want = _oracle(bw, pairs, feats, tols)
    got = _run(ctx, bw, pairs, tables, tmpls, params, cap=1 << 21, tuning=(wpw, 2))
    scr.screen_batch_run(got[0])
    _check(bw, got, want)
    assert scr.screen_batch_info(got[0])["words_per_warp"] == wpw
    scr.screen_batch_release(ctx, got[0])


def test_batch_subset_and_repeated_pairs(ctx):
    bw, _, feats, tols, tables, tmpls, params = _setup(ctx, 33, 4, 6)
    pairs = [(3, 1), (0, 5), (0, 5), (2, 0), (1, 4), (3, 3), (0, 0)]
    want = _oracle(bw, pairs, feats, tols)
    got = _run(ctx, bw, pairs, tables, tmpls, params, cap=1 << 20)
    scr.screen_batch_run(got[0])
    _check(bw, got, want)
    scr.screen_batch_release(ctx, got[0])


@pytest.mark.parametrize("n_pairs", [7, 8, 9, 40])
def test_batch_sort_pass_parity(ctx, n_pairs):
    """The packed sort key's width (column, row, scale and pair bits) sets the
    number of 8-bit passes; odd counts start from the scratch buffer.  Both
    parities end with the canonical order in the caller's buffer."""
    bw, _, feats, tols, tables, tmpls, params = _setup(ctx, 35, 4, 10)
    pairs = [(k % 4, (3 * k) % 10) for k in range(n_pairs)]
    want = _oracle(bw, pairs, feats, tols)
    got = _run(ctx, bw, pairs, tables, tmpls, params, cap=1 << 20)
    scr.screen_batch_run(got[0])
    _check(bw, got, want)
    H = max(im.shape[0] for im in bw.images)
    W = max(im.shape[1] for im in bw.images)
    S = max(len(ts.radii) for ts in bw.templates)
    bits = (W - 1).bit_length() + (H - 1).bit_length() + max(1, (S - 1).bit_length()) + n_pairs.bit_length()
    assert scr.screen_batch_info(got[0])["sort_passes"] == (bits + 7) // 8
    scr.screen_batch_release(ctx, got[0])


def test_batch_key_overflow_keeps_counts_exact(ctx):
    bw, pairs, feats, tols, tables, tmpls, params = _setup(ctx, 34, 3, 4)
    want = _oracle(bw, pairs, feats, tols)
    assert len(want[0]) > 20
    got = _run(ctx, bw, pairs, tables, tmpls, params, cap=8)
    scr.screen_batch_run(got[0])
    torch.cuda.synchronize()
    assert int(got[5][0].item()) == len(want[0])
    assert np.array_equal(got[1].cpu().numpy().view(np.uint64), want[1])
    scr.screen_batch_release(ctx, got[0])
