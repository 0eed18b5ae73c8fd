"""Row-band sharding on the CUDA path (the multi-GPU design, run here on one
device): each band of output rows is screened from tables built over the band's
image rows plus a halo of R_max + 1 rows on each side, as a rank would build
them from its own slice of the image.  The square and cone four-corner
identities hold for any image, so every window inside band + halo has its
exact sum, and the stitched masks and key lists must equal the whole-image
result bit for bit.  Integer results, tolerance 0."""
import numpy as np
import pytest

import synth
import paper_1707_05647_gb300 as scr
from gpu_helpers import params_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _screen(ctx, img, wl):
    H, W = img.shape
    S = len(wl.radii)
    tb = scr.build_tables(ctx, torch.from_numpy(np.ascontiguousarray(img)).cuda(), wl.sum_bits, wl.sq_bits)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    mask = torch.full((scr.mask_words(S, H, W),), -1, dtype=torch.int32, device="cuda")
    lst = torch.zeros(S * H * W + 1, dtype=torch.int64, device="cuda")
    n, over = scr.screen_positions(ctx, tb, tm, params_of(wl), mask, lst)
    assert not over
    m = mask.cpu().numpy().view(np.uint32).reshape(S, H, (W + 31) // 32)
    keys = lst[:n].cpu().numpy().view(np.uint64)
    scr.tables_release(ctx, tb)
    scr.template_release(ctx, tm)
    return m, keys


@pytest.mark.parametrize("ranks", [2, 3])
def test_row_bands_with_halo_equal_the_whole_image(ranks):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.small_planted(4100 + ranks, H=700, r=24, n_scales=5, s_min=0.6, s_max=1.6, sum_bits=32,
                             sq_bits=64)
    img = wl.image
    H = img.shape[0]
    halo = max(wl.radii) + 1
    ctx = scr.screen_init(0, 0)
    try:
        full_mask, full_keys = _screen(ctx, img, wl)
        assert len(full_keys) > 0
        per = (H + ranks - 1) // ranks
        masks, keys = [], []
        for k in range(ranks):
            y0, y1 = k * per, min(H, (k + 1) * per)
            a, b = max(0, y0 - halo), min(H, y1 + halo)
            m, kk = _screen(ctx, img[a:b], wl)
            masks.append(m[:, y0 - a:y1 - a])
            # keys of the band's own rows, moved from sub-image rows to image rows
            y = (kk >> np.uint64(24)) & np.uint64(0xFFFFFF)
            own = (y >= np.uint64(y0 - a)) & (y < np.uint64(y1 - a))
            kk = kk[own]
            keys.append(kk + (np.uint64(a) << np.uint64(24)))
        stitched = np.concatenate(masks, axis=1)
        assert np.array_equal(stitched, full_mask)
        # concatenated band lists, merged per scale, equal the whole-image list
        merged = np.sort(np.concatenate(keys))
        assert np.array_equal(merged, full_keys)
    finally:
        scr.screen_shutdown(ctx)
