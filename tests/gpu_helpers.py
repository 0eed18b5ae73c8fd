"""Helpers for the GPU tests: run a workload through the C ABI and through the oracle."""
import numpy as np

import oracle
import paper_1707_05647_gb300 as scr


def params_of(wl):
    return scr.Params(wl.radii, wl.features, wl.tol.mean_rel, wl.tol.std_rel, wl.tol.grad_rel, wl.tol.grad_abs)


def gpu_run(ctx, wl, cap=None, torch=None):
    import torch as _t
    torch = torch or _t
    H, W = wl.image.shape
    img = torch.from_numpy(np.ascontiguousarray(wl.image)).cuda()
    tb = scr.build_tables(ctx, img, wl.sum_bits, wl.sq_bits)
    tm = scr.template_features(ctx, wl.template, wl.r, wl.t_min, wl.features)
    p = params_of(wl)
    nw = scr.mask_words(len(wl.radii), H, W)
    mask = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    if cap is None:
        cap = len(wl.radii) * H * W
    lst = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    n, over = scr.screen_positions(ctx, tb, tm, p, mask, lst)
    out = dict(tables=tb, tmpl=tm, params=p,
               mask=mask.cpu().numpy().view(np.uint32).reshape(len(wl.radii), H, (W + 31) // 32),
               list=lst.cpu().numpy().view(np.uint64)[:min(n, cap)], count=n, overflow=over,
               bounds=scr.screen_bounds(tm, p))
    return out


def oracle_run(wl, tables=None):
    return oracle.screen_workload(wl.image, wl.template, wl.r, wl.t_min, wl.radii, wl.features, wl.tol,
                                  tables=tables)
