"""Helpers shared by the GPU parity tests: run the CUDA path (through the C ABI
binding) and the CPU oracle on the same seeded input and compare bit for bit."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
from paper_2312_05492_gb300 import ginterp as G


def bits(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a).view(np.uint32)


def gpu_roundtrip(x_np: np.ndarray, eb: float, cfg: G.Config, capacity: int | None = None, hist: bool = True):
    x = torch.from_numpy(np.ascontiguousarray(x_np, np.float32)).cuda()
    cap = x.numel() if capacity is None else capacity
    cf = G.compress(x, eb, cfg, capacity=cap, hist=hist, grow_on_overflow=False)
    xr = G.decompress(cf)
    torch.cuda.synchronize()
    h = cf.host_header(refresh=True)
    return cf, xr.cpu().numpy(), h


def oracle_cfg_from_header(h, radius: int) -> O.Config:
    return O.Config(order=tuple(h.cfg.dim_order), level_kind=tuple(h.cfg.level_kind),
                    cubic_kind=tuple(h.cfg.cubic_kind), radius=radius,
                    domain_x=32 if h.cfg.domain_x == 32 else 8, ndim=h.cfg.ndim if h.cfg.ndim in (1, 2) else 3)


def assert_parity(x_np: np.ndarray, eb: float, cfg: G.Config, capacity: int | None = None, check_hist=True):
    """Full element-by-element comparison of codes, anchors, outliers, histogram,
    header bounds and reconstruction; plus the hard bound |x - x'| <= e_l."""
    x_np = np.ascontiguousarray(x_np, np.float32)
    cf, xr, h = gpu_roundtrip(x_np, eb, cfg, capacity, hist=check_hist)
    mode = cfg.eb_mode
    ndim = cfg.ndim if cfg.ndim in (1, 2) else 3
    # bounds: range, alpha and level bounds identical to the oracle's (the header
    # holds the first three levels; the 1-D / 2-D kernels continue the sequence)
    eb_abs, e, twoe, inv2e = O.bounds_for(x_np, eb, mode, cfg.alpha if cfg.alpha > 0 else None, ndim=ndim)
    assert h.eb_abs == eb_abs, (h.eb_abs, eb_abs)
    assert np.array_equal(bits(np.array(h.e[:], np.float32)), bits(e[:3]))
    assert np.array_equal(bits(np.array(h.twoe[:], np.float32)), bits(twoe[:3]))
    assert np.array_equal(bits(np.array(h.inv2e[:], np.float32)), bits(inv2e[:3]))
    assert h.cfg.ndim == cfg.ndim
    # configuration: the oracle's own autotune decision when autotuning
    if cfg.autotune:
        ocfg = O.autotune(x_np, cfg.radius, ndim=ndim)
        ocfg.domain_x = 32 if cfg.domain_x == 32 else 8
        prof = O.profile(x_np, ndim)
        assert np.array_equal(np.array(h.profile[:], np.float64).view(np.uint64), prof.view(np.uint64))
    else:
        ocfg = O.Config(order=tuple(cfg.dim_order), level_kind=tuple(cfg.level_kind),
                        cubic_kind=tuple(cfg.cubic_kind), radius=cfg.radius,
                        domain_x=32 if cfg.domain_x == 32 else 8, ndim=ndim)
    assert tuple(h.cfg.dim_order) == tuple(ocfg.order)
    assert tuple(h.cfg.level_kind) == tuple(ocfg.level_kind)
    assert tuple(h.cfg.cubic_kind) == tuple(ocfg.cubic_kind)
    oc = O.compress(x_np, ocfg, e, twoe, inv2e, eb_abs)
    codes = cf.codes.cpu().numpy().view(np.uint16).reshape(x_np.shape)
    mism = np.flatnonzero(codes.reshape(-1) != oc.codes.reshape(-1))
    assert mism.size == 0, f"{mism.size} code mismatches, first at {np.unravel_index(mism[0], x_np.shape)}"
    assert np.array_equal(bits(cf.anchors.cpu().numpy()), bits(oc.anchors))
    assert h.n_outliers == oc.n_outliers
    k = min(int(h.n_outliers), cf.capacity)
    assert np.array_equal(cf.out_idx[:k].cpu().numpy().view(np.uint32), oc.out_idx[:k])
    assert np.array_equal(bits(cf.out_val[:k].cpu().numpy()), bits(oc.out_val[:k]))
    if check_hist:
        hist = cf.hist.cpu().numpy().view(np.uint32)
        assert np.array_equal(hist, O.histogram(oc.codes, cfg.radius))
    # decompression equals the oracle's reconstruction bit for bit
    if k == int(h.n_outliers):
        bad = np.flatnonzero(bits(xr).reshape(-1) != bits(oc.xrec).reshape(-1))
        assert bad.size == 0, f"{bad.size} reconstruction mismatches, first at {np.unravel_index(bad[0], x_np.shape)}"
        assert_bound(x_np, xr, ocfg, e)
    return cf, xr, h, oc


def assert_bound(x_np, xr, cfg: O.Config, e):
    pm, _ = O.schedule_maps(x_np.shape, cfg)
    L = O.levels(cfg.ndim)
    lvl = np.where(pm == 255, -1, L - 1 - pm.astype(np.int64) // 3)
    fin = np.isfinite(x_np)
    err = np.abs(xr.astype(np.float64) - x_np.astype(np.float64))
    for l in range(L):
        m = (lvl == l) & fin
        assert np.all(err[m] <= e[l]), (l, float(err[m].max()), float(e[l]))
    assert np.all(bits(xr)[~fin] == bits(x_np)[~fin])
    assert np.all(err[(lvl < 0) & fin] == 0)
