"""Full-size parity in the bench's launch configuration (build_tables ->
screen_features -> compact_mask on one stream): every table entry, mask word
and list key against the oracle, and the planted match present."""
import numpy as np
import pytest

import oracle
import synth
import paper_1707_05647_gb300 as scr
from gpu_helpers import params_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _covering(wl):
    return [wl.t_min - 1 <= R / wl.s_true <= wl.r + 1 for R in wl.radii]


@pytest.mark.parametrize("cfg", [2, 3])
def test_full_size_bit_exact(cfg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.CONFIGS[cfg]()
    H, W = wl.image.shape
    S = len(wl.radii)
    ctx = scr.screen_init(0, 0)
    try:
        stream = torch.cuda.current_stream()
        img = torch.from_numpy(wl.image).cuda()
        p = params_of(wl)
        tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
        mask = torch.empty(scr.mask_words(S, H, W), dtype=torch.int32, device="cuda")
        cap = 1 << 22
        lst = torch.empty(cap, dtype=torch.int64, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        tb = scr.build_tables(ctx, img, wl.sum_bits, wl.sq_bits, stream)
        scr.screen_features(ctx, tb, tm, p, mask, stream)
        scr.compact_mask(ctx, mask, S, H, W, lst, count, stream)
        torch.cuda.synchronize()
        ref = oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol)
        got = mask.cpu().numpy().view(np.uint32).reshape(ref["mask"].shape)
        assert np.array_equal(got, ref["mask"]), "mask differs"
        n = int(count.item())
        assert n == ref["count"] and n <= cap
        assert np.array_equal(lst[:n].cpu().numpy().view(np.uint64), ref["list"])
        tabs = ref["tables"]
        for which, want in enumerate((tabs.L1, tabs.L2, tabs.T1, tabs.T2)):
            bits = wl.sum_bits if which % 2 == 0 else wl.sq_bits
            g = scr.tables_copy_to_host(ctx, tb, which)
            if bits == 32:
                want = want & np.uint64(0xFFFFFFFF)
            assert np.array_equal(g, want), f"table {which}"
            del g
        y, x = wl.planted
        hit = [(got[s, y, x >> 5] >> (x & 31)) & 1 for s in range(S)]
        assert any(h and c for h, c in zip(hit, _covering(wl))), hit
        scr.tables_release(ctx, tb)
        scr.template_release(ctx, tm)
    finally:
        scr.screen_shutdown(ctx)
