"""One field split across ranks along z (one process per GPU).

Under the closed-8^3-chunk rule (Sec. IV-A) the outputs of a slab of planes
[z0, z1), with z0 and z1 multiples of 8, depend only on the original values of
planes [z0, z1]: the slab's own planes plus the closing anchor plane z1, which
the next slab owns.  Each rank therefore compresses the sub-field
x[z0 : z1 + 1] on its own GPU and keeps the outputs of its own planes.  The
ranks exchange only:
  - the value range (two scalars, one all-reduce) when the bound is relative,
    so that every rank quantizes against the same e_l;
  - the histogram of their owned codes (2R counters, one all-reduce);
  - for assembly into the single-field form only: their owned outputs, outlier
    indices offset by z0 * ny * nx (concatenated in rank order they are the
    whole field's ascending list).
Codes, anchors, outliers and reconstructions then equal a single-GPU run on
the whole field bit for bit.  The configuration must be explicit (the sampling
autotuner looks at the whole field); pick it once and pass the same one on
every rank.

The arithmetic stays in the library; this module decides slab bounds, agrees
on the bound and combines per-rank results.  The per-rank work goes through a
backend object (GpuBackend here) with value_range / compress / histogram /
decompress methods, so the same combining logic runs on any device.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import torch
import torch.distributed as dist


@dataclass(frozen=True)
class Slab:
    rank: int
    z0: int   # first owned plane (a multiple of 8)
    z1: int   # one past the last owned plane
    zc: int   # one past the last plane the rank reads: z1 + 1 (closing plane), or nz

    @property
    def owned_planes(self) -> int:
        return self.z1 - self.z0

    @property
    def empty(self) -> bool:
        return self.z1 <= self.z0


def slabs(nz: int, world: int) -> list[Slab]:
    """Contiguous z-ranges with boundaries on multiples of 8, split as evenly as the
    8-plane chunk grid allows; with more ranks than chunks the extra ranks get
    empty slabs."""
    if nz < 1 or world < 1:
        raise ValueError("nz and world must be positive")
    chunks = max(1, -(-(nz - 1) // 8))
    out = []
    for r in range(world):
        c0, c1 = chunks * r // world, chunks * (r + 1) // world
        z0 = min(nz, 8 * c0)
        z1 = nz if r == world - 1 else min(nz, 8 * c1)
        if z1 < z0:
            z1 = z0
        zc = min(nz, z1 + 1)
        out.append(Slab(r, z0, z1, zc))
    return out


def anchors_along(n: int) -> int:
    return (n - 1) // 8 + 1


@dataclass
class ShardField:
    """A rank's part of a sharded compression."""
    slab: Slab
    dims: tuple           # whole field (nz, ny, nx)
    eb_abs: float
    alpha: float
    local: object         # the backend's compressed form of x[z0:zc] (closing plane included)
    hist: torch.Tensor    # whole-field histogram (int64, 2R), identical on every rank
    n_owned_outliers: int

    @property
    def n_outliers(self) -> int:
        return int(self.hist[0])


def agree_on_bound(eps: float, eb_mode: str, local_range, backend, group=None):
    """(eb_abs, alpha) every rank uses.  Relative mode: eps * (vmax - vmin) over the
    whole field (finite values; one MAX all-reduce of (-vmin, vmax)) and alpha =
    A(eps) (Eq. 1); absolute mode: eps and alpha = 1."""
    if eb_mode == "abs":
        return float(eps), 1.0
    lo, hi = local_range
    t = torch.tensor([-lo, hi], dtype=torch.float64, device=backend.comm_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    lo, hi = -float(t[0]), float(t[1])
    if lo > hi:  # no finite value anywhere
        lo = hi = 0.0
    return eps * (hi - lo), backend.alpha(eps)


def compress(x_local, slab: Slab, dims, eps: float, cfg, backend, group=None, eb_mode: str = "rel") -> ShardField:
    """Compress this rank's sub-field x[z0:zc] (shape (zc - z0, ny, nx)) of a field of
    shape dims.  Collective: every rank of `group` calls it with its own slab."""
    nz, ny, nx = (int(d) for d in dims)
    if getattr(cfg, "autotune", False):
        raise ValueError("a sharded field needs an explicit configuration (autotune looks at the whole field)")
    if getattr(cfg, "ndim", 3) not in (0, 3):
        raise ValueError("slabs split the 8^3-chunk geometry; 1-D and 2-D fields are independent per slice or "
                         "row and are split by the caller")
    if not slab.empty and tuple(int(d) for d in x_local.shape) != (slab.zc - slab.z0, ny, nx):
        raise ValueError(f"rank {slab.rank}: sub-field shape {tuple(x_local.shape)} does not match {slab}")
    rng = backend.value_range(x_local) if not slab.empty else (float("inf"), float("-inf"))
    eb_abs, alpha = agree_on_bound(eps, eb_mode, rng, backend, group)
    R = int(cfg.radius)
    if slab.empty:
        local, owned_hist = None, torch.zeros(2 * R, dtype=torch.int64, device=backend.comm_device)
    else:
        local = backend.compress(x_local, eb_abs, alpha, cfg)
        owned_hist = backend.histogram(backend.codes(local)[: slab.owned_planes * ny * nx], R)
        owned_hist = owned_hist.to(device=backend.comm_device, dtype=torch.int64)
    n_owned = int(owned_hist[0])
    hist = owned_hist.clone()
    dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    return ShardField(slab, (nz, ny, nx), eb_abs, alpha, local, hist, n_owned)


def owned_outputs(sf: ShardField, backend) -> dict:
    """This rank's part of the single-field outputs, as CPU tensors: codes and anchors
    of its planes, its outliers with whole-field indices."""
    nz, ny, nx = sf.dims
    s = sf.slab
    if s.empty:
        z = torch.zeros(0)
        return {"codes": z.to(torch.int32), "anchors": z.float(), "out_idx": z.long(), "out_val": z.float()}
    plane_anchors = anchors_along(ny) * anchors_along(nx)
    a_planes = -(-s.owned_planes // 8)
    idx, val = backend.outliers(sf.local, sf.n_owned_outliers)
    return {
        "codes": backend.codes(sf.local)[: s.owned_planes * ny * nx].cpu().to(torch.int32),
        "anchors": backend.anchors(sf.local)[: a_planes * plane_anchors].cpu(),
        "out_idx": idx.cpu().to(torch.int64) + s.z0 * ny * nx,
        "out_val": val.cpu(),
    }


def assemble(sf: ShardField, backend, group=None, dst: int = 0):
    """Gather the single-field form on rank `dst` (None elsewhere): codes [N] int32,
    anchors, outlier indices (ascending) and values, histogram."""
    part = owned_outputs(sf, backend)
    world = dist.get_world_size(group)
    parts = [None] * world if dist.get_rank(group) == dst else None
    dist.gather_object(part, parts, dst=dst, group=group)
    if parts is None:
        return None
    return {
        "codes": torch.cat([p["codes"] for p in parts]),
        "anchors": torch.cat([p["anchors"] for p in parts]),
        "out_idx": torch.cat([p["out_idx"] for p in parts]),
        "out_val": torch.cat([p["out_val"] for p in parts]),
        "hist": sf.hist.cpu(),
    }


def decompress(sf: ShardField, backend):
    """Reconstruction of this rank's own planes (shape (z1 - z0, ny, nx)); the closing
    plane is decoded from the rank's own copy of it, so no exchange is needed."""
    if sf.slab.empty:
        return None
    xr = backend.decompress(sf.local)
    return xr[: sf.slab.owned_planes]


class GpuBackend:
    """Per-rank work on this process's GPU through the C ABI."""

    comm_device = "cuda"

    def __init__(self):
        from . import ginterp as G
        self.G = G
        G.load()

    def alpha(self, eps: float) -> float:
        return self.G.interp_alpha(eps)

    def value_range(self, x):
        lo, hi = self.G.value_range(x).tolist()
        return float(lo), float(hi)

    def compress(self, x, eb_abs: float, alpha: float, cfg):
        c = replace(cfg, eb_mode="abs", alpha=float(alpha), autotune=False)
        return self.G.compress(x, eb_abs, c)

    def codes(self, cf):
        return cf.codes.view(-1)

    def anchors(self, cf):
        return cf.anchors.view(-1)

    def histogram(self, codes, radius: int):
        return self.G.histogram(codes, radius).to(torch.int64) & 0xFFFFFFFF  # uint32 counters

    def outliers(self, cf, k: int):
        return cf.out_idx[:k], cf.out_val[:k]

    def decompress(self, cf):
        return self.G.decompress(cf)
