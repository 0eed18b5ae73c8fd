"""Compaction of constructed masks into key lists, through the C ABI.

The list is by definition the ascending keys (s << 48) | (y << 24) | x of the
mask's set bits (Algorithm 1's result set in mask order), derived here on the
host.  The masks mix the patterns the scatter kernel treats differently:
clusters of fully or densely set words (a warp then writes each word's bits
together, one bit per lane), sparse scattered bits (each lane walks its own
bits) and fully set stretches; the shapes make a thread's 16 consecutive words
run across rows and scale planes and leave a partial last chunk; the list
capacities end inside dense words."""
import numpy as np
import pytest

import paper_1707_05647_gb300 as scr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = scr.screen_init(0, 0)
    yield c
    scr.screen_shutdown(c)


def _mask(seed, S, H, W, pattern):
    rng = np.random.default_rng(seed)
    Ww = (W + 31) // 32
    bits = np.zeros((S, H, Ww * 32), bool)
    if pattern in ("clusters", "mixed"):
        for _ in range(max(1, S * H // 8)):
            s, y, x = rng.integers(S), rng.integers(H), rng.integers(Ww * 32)
            h, w = rng.integers(1, 12), rng.integers(1, 80)
            bits[s, y:y + h, x:x + w] = rng.random((min(h, H - y), min(w, Ww * 32 - x))) < rng.choice([0.6, 1.0])
    if pattern in ("sparse", "mixed"):
        bits |= rng.random(bits.shape) < 0.002
    if pattern == "full":
        bits[:] = True
    if pattern == "band":   # fully set rows in the middle of otherwise empty planes
        bits[:, H // 3:H // 3 + 3, :] = True
    bits[:, :, W:] = False
    weights = np.left_shift(np.uint64(1), np.arange(32, dtype=np.uint64))
    words = (bits.reshape(S, H, Ww, 32).astype(np.uint64) * weights).sum(-1).astype(np.uint32)
    s, y, x = np.nonzero(bits)
    keys = (s.astype(np.uint64) << np.uint64(48)) | (y.astype(np.uint64) << np.uint64(24)) | x.astype(np.uint64)
    return torch.from_numpy(words.reshape(-1).view(np.int32)).cuda(), keys


# (S, H, W): 16 words per thread cross rows (Ww = 1, 3, 33, 7, 256, 4) and scale
# planes; totals that are not multiples of the 4096-word chunk
SHAPES = [(1, 1, 1), (2, 5, 70), (3, 37, 1050), (4, 129, 200), (2, 300, 8192), (5, 61, 97)]


PATTERNS = ["clusters", "sparse", "mixed", "full", "band"]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("pattern", PATTERNS)
def test_compact_mask_keys(ctx, shape, pattern):
    S, H, W = shape
    mask, keys = _mask(100 * SHAPES.index(shape) + PATTERNS.index(pattern), S, H, W, pattern)
    n = len(keys)
    lst = torch.full((max(n, 1) + 5,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    scr.compact_mask(ctx, mask, S, H, W, lst, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == n
    got = lst.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[:n], keys)
    assert np.all(lst.cpu().numpy()[n:] == -1)          # nothing written past the count


@pytest.mark.parametrize("pattern", ["clusters", "full", "mixed"])
def test_compact_mask_capacity_inside_dense_words(ctx, pattern):
    """Capacities that end inside a dense word: exactly the first cap keys are
    written, nothing beyond, and the true count is reported."""
    S, H, W = 3, 90, 1000
    mask, keys = _mask(7, S, H, W, pattern)
    n = len(keys)
    assert n > 100
    for cap in (1, 17, 31, 33, n // 3 + 5, n - 1):
        lst = torch.full((cap + 8,), -1, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        scr.compact_mask(ctx, mask, S, H, W, lst[:cap], cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == n
        got = lst.cpu().numpy()
        assert np.array_equal(got[:cap].view(np.uint64), keys[:cap]), cap
        assert np.all(got[cap:] == -1), cap
