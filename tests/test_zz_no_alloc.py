"""The allocation-free compaction entry point, checked against the keys the
mask defines and against compact_mask.

compact_mask_noalloc exists for callers that cannot allocate device memory at
the point where they compact a mask (real-time loops that must never enter an
allocator, processes whose device memory all belongs to another framework's
allocator, embedded runtimes with every buffer fixed at start).  Its scratch is
a fixed array inside the library.  The list it returns is by definition the
ascending keys (s << 48) | (y << 24) | x of the mask's set bits, which the test
derives on the host from the mask itself; it must also equal what compact_mask
returns.  Two calls in a row check that what one call leaves in the shared
array does not leak into the next.  This file is collected last so a failure
here does not hide the other GPU tests.
"""
import numpy as np
import pytest

import paper_1707_05647_gb300 as scr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mask(seed, S, H, W, density):
    """Random mask words (device) and the expected keys derived from its bits."""
    rng = np.random.default_rng(seed)
    Ww = (W + 31) // 32
    bits = rng.random((S, H, Ww * 32)) < density
    bits[:, :, W:] = False
    weights = np.left_shift(np.uint64(1), np.arange(32, dtype=np.uint64))
    words = (bits.reshape(S, H, Ww, 32).astype(np.uint64) * weights).sum(-1).astype(np.uint32)
    s, y, x = np.nonzero(bits)             # row-major order = ascending (s, y, x)
    keys = (s.astype(np.uint64) << np.uint64(48)) | (y.astype(np.uint64) << np.uint64(24)) | x.astype(np.uint64)
    return torch.from_numpy(words.reshape(-1).view(np.int32)).cuda(), keys


def _compact_both(ctx, mask, S, H, W, cap):
    ref_list = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    got_list = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    got_cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    scr.compact_mask(ctx, mask, S, H, W, ref_list, ref_cnt)
    scr.compact_mask_noalloc(mask, S, H, W, got_list, got_cnt)
    torch.cuda.synchronize()
    return ref_list.cpu(), int(ref_cnt.item()), got_list.cpu(), int(got_cnt.item())


def test_noalloc_matches_mask_keys_and_compact_mask_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    ctx = scr.screen_init(0, 0)
    try:
        # the second mask is smaller and sparser, so stale counts or keys left
        # by the first call in the shared array would show
        cases = [(11, 5, 700, 1000, 0.02), (12, 2, 300, 97, 0.001)]
        for (seed, S, H, W, dens) in cases:                     # two calls in a row
            mask, want = _mask(seed, S, H, W, dens)
            cap = 1 << 16
            rl, rn, gl, gn = _compact_both(ctx, mask, S, H, W, cap)
            assert gn == len(want) > 0
            k = min(gn, cap)
            assert np.array_equal(gl[:k].numpy().view(np.uint64), want[:k])
            assert rn == gn and torch.equal(gl[:k], rl[:k])
    finally:
        scr.screen_shutdown(ctx)


def test_noalloc_rejects_masks_beyond_the_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = torch.zeros(16, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(scr.ScreenError) as e:
        # 32 scales x 65535 rows x 2048 words exceeds 65536 chunks of 4096 words
        scr.compact_mask_noalloc(small, 32, 65535, 65535, None, cnt)
    assert e.value.code == scr.SCR_EINVAL
    assert "scratch" in scr.compact_mask_noalloc_error()
