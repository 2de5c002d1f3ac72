"""CPU oracle for G-Interp (cuSZ-i, arXiv 2312.05492, Sec. IV).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA library never links, loads or calls it, and nothing here imports the
CUDA package: the two implementations share no code.

The arithmetic lives in ``ginterp_oracle.c`` (plain C, float32 with FMA
contraction off, float64 for the error-bound algebra); this module only
marshals numpy arrays through ctypes.  Every function cites the passage of
the paper it restates in the C source.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from .build import build as _build, library_path

_lib = None

# stencil kinds written by schedule_maps / predict_original
K_ANCHOR, K_COPY, K_LINEAR, K_QUAD_LEFT, K_QUAD_RIGHT, K_CUBIC_NAK, K_CUBIC_NATURAL = range(7)
PROFILE_LEN = 18


_libs = {}
_threads = 1


def set_threads(n: int) -> int:
    """Run the oracle on n host threads (the OpenMP build, which splits the points of
    each pass; its results are identical to the single-threaded build's), or on one
    (the plain build) for n <= 1.  Returns the number of threads in use."""
    global _lib, _threads
    if n <= 1:
        _lib, _threads = _open(False), 1
    else:
        _lib = _open(True)
        _threads = int(_lib.orc_threads(int(n)))
    return _threads


def threads() -> int:
    return _threads


def _load():
    global _lib
    if _lib is None:
        _lib = _open(False)
    return _lib


def _open(threaded: bool):
    if threaded in _libs:
        return _libs[threaded]
    path = library_path(threaded)
    if not os.path.exists(path) or not os.path.exists(library_path(not threaded)):
        _build()
    lib = ctypes.CDLL(path)
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.c_void_p
    lib.orc_alpha.restype = f64
    lib.orc_alpha.argtypes = [f64]
    lib.orc_level_bounds.restype = None
    lib.orc_level_bounds.argtypes = [f64, f64, i32, P, P, P]
    lib.orc_levels.restype = i32
    lib.orc_levels.argtypes = [i32]
    lib.orc_value_range.restype = i64
    lib.orc_value_range.argtypes = [P, i64, P, P]
    lib.orc_rel_to_abs.restype = f64
    lib.orc_rel_to_abs.argtypes = [f64, ctypes.c_float, ctypes.c_float]
    lib.orc_anchor_count.restype = i64
    lib.orc_anchor_count.argtypes = [i64, i64, i64, i32]
    lib.orc_spline.restype = ctypes.c_float
    lib.orc_spline.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    lib.orc_schedule_maps.restype = ctypes.c_int
    lib.orc_schedule_maps.argtypes = [i64, i64, i64, P, P, P, i32, i32, P, P]
    lib.orc_compress.restype = i64
    lib.orc_compress.argtypes = [P, i64, i64, i64, P, P, P, i32, i32, i32, P, P, P, P, P, P, P, i64, P]
    lib.orc_decompress.restype = ctypes.c_int
    lib.orc_decompress.argtypes = [i64, i64, i64, P, P, P, i32, i32, i32, P, P, P, P, P, i64, P]
    lib.orc_predict_original.restype = ctypes.c_int
    lib.orc_predict_original.argtypes = [P, i64, i64, i64, P, P, P, i32, i32, P, P]
    lib.orc_histogram.restype = None
    lib.orc_histogram.argtypes = [P, i64, i32, P]
    lib.orc_profile.restype = None
    lib.orc_profile.argtypes = [P, i64, i64, i64, i32, P]
    lib.orc_autotune_decide.restype = None
    lib.orc_autotune_decide.argtypes = [P, P, P, P]
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_threads.argtypes = [ctypes.c_int]
    _libs[threaded] = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


@dataclass
class Config:
    """Interpolation configuration (Sec. IV-B).

    order: axes (0=z, 1=y, 2=x) in processing order within every level.
    level_kind[l]: stride 2**l uses 0 = linear only, 1 = splines by neighbour count.
    cubic_kind[axis]: 0 = not-a-knot, 1 = natural.
    domain_x: neighbour domain along x, 8 (the closed 8^3 chunk, Sec. IV-A) or 32
      (the x-extended 32x8x8 block of Sec. IV-C).
    ndim: chunk geometry (Sec. IV-A): 3 = 8^3 chunks; 2 = 16^2 chunks over (y, x),
      every z-slice independent; 1 = 512-point chunks along x, every row independent.
      Levels coarser than stride 4 (2-D, 1-D) follow level_kind[2].
    """
    order: tuple = (0, 1, 2)
    level_kind: tuple = (1, 1, 1)
    cubic_kind: tuple = (0, 0, 0)
    radius: int = 512
    domain_x: int = 8
    ndim: int = 3


@dataclass
class Compressed:
    dims: tuple
    cfg: Config
    e: np.ndarray
    twoe: np.ndarray
    inv2e: np.ndarray
    eb_abs: float
    anchors: np.ndarray
    codes: np.ndarray
    out_idx: np.ndarray
    out_val: np.ndarray
    n_outliers: int
    xrec: np.ndarray = field(repr=False)


def alpha(eps: float) -> float:
    """Eq. 1: alpha = A(eps)."""
    return float(_load().orc_alpha(float(eps)))


def levels(ndim: int = 3) -> int:
    """Interpolation levels of the chunk geometry: 3 (8^3), 4 (16^2), 9 (512)."""
    return int(_load().orc_levels(int(ndim)))


def level_bounds(eb_abs: float, alpha_: float, nlev: int = 3):
    """e_l = eb / alpha^l for l = 0 .. nlev-1 (strides 1, 2, 4, ...), with 2e_l and 1/(2e_l)."""
    e = np.zeros(nlev, np.float32)
    twoe = np.zeros(nlev, np.float32)
    inv2e = np.zeros(nlev, np.float32)
    _load().orc_level_bounds(float(eb_abs), float(alpha_), int(nlev), _ptr(e), _ptr(twoe), _ptr(inv2e))
    return e, twoe, inv2e


def value_range(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float32)
    lo = np.zeros(1, np.float32)
    hi = np.zeros(1, np.float32)
    nonfinite = _load().orc_value_range(_ptr(x), x.size, _ptr(lo), _ptr(hi))
    return float(lo[0]), float(hi[0]), int(nonfinite)


def rel_to_abs(eps: float, vmin: float, vmax: float) -> float:
    return float(_load().orc_rel_to_abs(float(eps), float(vmin), float(vmax)))


def anchor_count(dims, ndim: int = 3) -> int:
    return int(_load().orc_anchor_count(*[int(d) for d in dims], int(ndim)))


def spline(kind: int, m3: float, m1: float, p1: float, p3: float) -> float:
    return float(_load().orc_spline(int(kind), m3, m1, p1, p3))


def schedule_maps(dims, cfg: Config):
    """Per-point pass id (0..8, coarse first; 255 = anchor) and stencil kind."""
    n = int(np.prod(dims))
    pm = np.zeros(n, np.uint8)
    km = np.zeros(n, np.uint8)
    rc = _load().orc_schedule_maps(*[int(d) for d in dims], _ptr(_i32(cfg.order)), _ptr(_i32(cfg.level_kind)),
                                   _ptr(_i32(cfg.cubic_kind)), int(cfg.domain_x), int(cfg.ndim), _ptr(pm),
                                   _ptr(km))
    if rc != 0:
        raise ValueError("bad configuration")
    return pm.reshape(dims), km.reshape(dims)


def predict_original(x: np.ndarray, cfg: Config):
    """Debug mode: each point predicted from the ORIGINAL neighbours (no quantization)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    pred = np.zeros_like(x)
    kind = np.zeros(x.shape, np.uint8)
    rc = _load().orc_predict_original(_ptr(x), *[int(d) for d in x.shape], _ptr(_i32(cfg.order)),
                                      _ptr(_i32(cfg.level_kind)), _ptr(_i32(cfg.cubic_kind)), int(cfg.domain_x),
                                      int(cfg.ndim), _ptr(pred), _ptr(kind))
    if rc != 0:
        raise ValueError("bad configuration")
    return pred, kind


def bounds_for(x: np.ndarray, eb: float, mode: str = "rel", alpha_override: float | None = None, ndim: int = 3):
    """Absolute bound and level bounds as the compressor derives them (Sec. IV-B)."""
    if mode == "rel":
        lo, hi, _ = value_range(x)
        eb_abs = rel_to_abs(eb, lo, hi)
        a = alpha(eb) if not alpha_override or alpha_override <= 0 else alpha_override
    else:
        eb_abs = float(eb)
        a = 1.0 if not alpha_override or alpha_override <= 0 else alpha_override
    e, twoe, inv2e = level_bounds(eb_abs, a, levels(ndim))
    return eb_abs, e, twoe, inv2e


def compress(x: np.ndarray, cfg: Config, e, twoe, inv2e, eb_abs: float = float("nan"),
             capacity: int | None = None) -> Compressed:
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = tuple(int(d) for d in x.shape)
    n = x.size
    cap = n if capacity is None else int(capacity)
    anchors = np.zeros(anchor_count(dims, cfg.ndim), np.float32)
    codes = np.zeros(n, np.uint16)
    out_idx = np.zeros(max(cap, 1), np.uint32)
    out_val = np.zeros(max(cap, 1), np.float32)
    xr = np.zeros(n, np.float32)
    e = np.ascontiguousarray(e, np.float32)
    twoe = np.ascontiguousarray(twoe, np.float32)
    inv2e = np.ascontiguousarray(inv2e, np.float32)
    if min(e.size, twoe.size, inv2e.size) < levels(cfg.ndim):
        raise ValueError(f"{levels(cfg.ndim)} level bounds needed")
    cnt = _load().orc_compress(_ptr(x), *dims, _ptr(_i32(cfg.order)), _ptr(_i32(cfg.level_kind)),
                               _ptr(_i32(cfg.cubic_kind)), int(cfg.domain_x), int(cfg.ndim), int(cfg.radius), _ptr(e),
                               _ptr(twoe), _ptr(inv2e),
                               _ptr(anchors), _ptr(codes), _ptr(out_idx), _ptr(out_val), cap, _ptr(xr))
    if cnt < 0:
        raise RuntimeError(f"oracle compress failed ({cnt})")
    k = min(int(cnt), cap)
    return Compressed(dims, cfg, e, twoe, inv2e, eb_abs, anchors, codes.reshape(dims), out_idx[:k].copy(),
                      out_val[:k].copy(), int(cnt), xr.reshape(dims))


def decompress(c: Compressed) -> np.ndarray:
    n = int(np.prod(c.dims))
    xr = np.zeros(n, np.float32)
    codes = np.ascontiguousarray(c.codes.reshape(-1), np.uint16)
    idx = np.ascontiguousarray(c.out_idx, np.uint32)
    val = np.ascontiguousarray(c.out_val, np.float32)
    rc = _load().orc_decompress(*c.dims, _ptr(_i32(c.cfg.order)), _ptr(_i32(c.cfg.level_kind)),
                                _ptr(_i32(c.cfg.cubic_kind)), int(c.cfg.domain_x), int(c.cfg.ndim), int(c.cfg.radius),
                                _ptr(np.ascontiguousarray(c.twoe, np.float32)),
                                _ptr(np.ascontiguousarray(c.anchors, np.float32)), _ptr(codes), _ptr(idx), _ptr(val),
                                int(idx.size), _ptr(xr))
    if rc != 0:
        raise RuntimeError(f"oracle decompress failed ({rc})")
    return xr.reshape(c.dims)


def histogram(codes: np.ndarray, radius: int) -> np.ndarray:
    codes = np.ascontiguousarray(codes.reshape(-1), np.uint16)
    hist = np.zeros(2 * int(radius), np.uint32)
    _load().orc_histogram(_ptr(codes), codes.size, int(radius), _ptr(hist))
    return hist


def profile(x: np.ndarray, ndim: int = 3) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    prof = np.zeros(PROFILE_LEN, np.float64)
    _load().orc_profile(_ptr(x), *[int(d) for d in x.shape], int(ndim), _ptr(prof))
    return prof


def autotune_decide(prof: np.ndarray, radius: int = 512, ndim: int = 3) -> Config:
    order = np.zeros(3, np.int32)
    lk = np.zeros(3, np.int32)
    ck = np.zeros(3, np.int32)
    _load().orc_autotune_decide(_ptr(np.ascontiguousarray(prof, np.float64)), _ptr(order), _ptr(lk), _ptr(ck))
    return Config(tuple(int(v) for v in order), tuple(int(v) for v in lk), tuple(int(v) for v in ck), radius,
                  ndim=int(ndim))


def autotune(x: np.ndarray, radius: int = 512, ndim: int = 3) -> Config:
    return autotune_decide(profile(x, ndim), radius, ndim)


def quality(hist: np.ndarray, radius: int, x: np.ndarray | None = None, xrec: np.ndarray | None = None) -> dict:
    """Quality report written from its definitions (Sec. IV-D: Fig. 4 counts the
    nonzero quant-codes; the PSNR comparison after it), in float64:

    - n = sum of the histogram, n_outliers = hist[0], n_nonzero = n - hist[R]
      (points whose quant-code q is not 0, outliers included),
      max_abs_q = max |c - R| over occupied bins c != 0;
    - entropy_bits = -sum_c p_c log2 p_c with p_c = hist[c] / n (Shannon);
    - over the finite points of x: sse = sum (x - x')^2, max_abs_err = max |x - x'|,
      vmin / vmax, psnr_db = 20 log10(vmax - vmin) - 10 log10(sse / n_finite).
    """
    h = np.asarray(hist, dtype=np.float64).reshape(-1)
    R = int(radius)
    n = float(h.sum())
    occ = np.nonzero(h)[0]
    kept = occ[(occ != 0) & (occ != R)]
    p = h[occ] / n if n else np.zeros(0)
    out = {
        "n": int(n), "n_outliers": int(h[0]), "n_nonzero": int(n - h[R]),
        "max_abs_q": int(np.abs(kept - R).max()) if kept.size else 0,
        "entropy_bits": float(-(p * np.log2(p)).sum()) if p.size else 0.0,
    }
    if x is None:
        out.update(n_finite=0, sse=float("nan"), max_abs_err=float("nan"), vmin=float("nan"), vmax=float("nan"),
                   psnr_db=float("nan"))
        return out
    a = np.asarray(x, dtype=np.float64).reshape(-1)
    b = np.asarray(xrec, dtype=np.float64).reshape(-1)
    fin = np.isfinite(a)
    a, b = a[fin], b[fin]
    d = a - b
    sse = float((d * d).sum())
    nf = int(a.size)
    vmin, vmax = (float(a.min()), float(a.max())) if nf else (float("nan"), float("nan"))
    if nf and sse > 0:
        psnr = 20.0 * np.log10(vmax - vmin) - 10.0 * np.log10(sse / nf)
    else:
        psnr = float("inf") if nf else float("nan")
    out.update(n_finite=nf, sse=sse, max_abs_err=float(np.abs(d).max()) if nf else float("nan"), vmin=vmin,
               vmax=vmax, psnr_db=float(psnr))
    return out
