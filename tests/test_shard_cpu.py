"""Splitting one field across ranks along z (world size 2, gloo, CPU).

The per-rank work runs on the oracle, so these tests check the sharding logic
itself (slab bounds on the 8-plane chunk grid, the closing plane each slab
reads, agreement on the bound, owned-code histogram all-reduce, outlier
filtering and index offsets, assembly) and the claim it rests on: under the
closed-8^3-chunk rule (Sec. IV-A) the slabs' outputs concatenate to the
single-field result bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2312_05492_gb300 import fields, shard


def test_slab_bounds():
    for nz in (1, 2, 8, 9, 16, 17, 41, 64, 65, 100, 512):
        for world in (1, 2, 3, 4, 8):
            ss = shard.slabs(nz, world)
            assert len(ss) == world
            assert ss[0].z0 == 0 and ss[-1].z1 == nz
            for a, b in zip(ss, ss[1:]):
                assert a.z1 == b.z0
            for s in ss:
                assert s.z0 % 8 == 0 and s.z0 <= s.z1
                assert s.empty or s.z1 == nz or s.z1 % 8 == 0
                assert s.zc == min(nz, s.z1 + 1)
            sizes = [s.owned_planes for s in ss if s.z1 < nz]
            if sizes:  # interior slabs differ by at most one chunk
                assert max(sizes) - min(sizes) <= 8
    assert [s.empty for s in shard.slabs(9, 2)] == [True, False]


class OracleBackend:
    comm_device = "cpu"

    def alpha(self, eps):
        return O.alpha(eps)

    def value_range(self, x):
        lo, hi, _ = O.value_range(x)
        return lo, hi

    def compress(self, x, eb_abs, alpha, cfg):
        e, twoe, inv2e = O.level_bounds(eb_abs, alpha)
        return O.compress(x, cfg, e, twoe, inv2e, eb_abs)

    def codes(self, c):
        return torch.from_numpy(c.codes.reshape(-1).astype(np.int32))

    def anchors(self, c):
        return torch.from_numpy(c.anchors.copy())

    def histogram(self, codes, radius):
        return torch.from_numpy(O.histogram(codes.numpy().astype(np.uint16), radius).astype(np.int64))

    def outliers(self, c, k):
        return torch.from_numpy(c.out_idx[:k].astype(np.int64)), torch.from_numpy(c.out_val[:k].copy())

    def decompress(self, c):
        return torch.from_numpy(O.decompress(c))


CASES = {
    # (dims, field, eps, mode, config)
    "split": ((41, 20, 27), "shocks", 1e-4, "rel", O.Config((0, 1, 2), (1, 1, 1), (0, 0, 0), 512)),
    "order": ((48, 17, 33), "grf", 1e-3, "rel", O.Config((2, 0, 1), (1, 0, 1), (1, 0, 0), 64)),
    "empty": ((9, 24, 16), "grf", 1e-2, "abs", O.Config((1, 2, 0), (0, 1, 1), (0, 1, 1), 8)),
}


def _field(kind, dims):
    if kind == "shocks":
        return fields.shocks(dims, 6).numpy()
    return fields.grf(dims, 3.0, 0).numpy()


def _worker(rank, world, port, case, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, kind, eps, mode, cfg = CASES[case]
        x = _field(kind, dims)
        s = shard.slabs(dims[0], world)[rank]
        be = OracleBackend()
        sf = shard.compress(x[s.z0:s.zc] if not s.empty else None, s, dims, eps, cfg, be, eb_mode=mode)
        full = shard.assemble(sf, be)
        xr = shard.decompress(sf, be)
        parts = [None] * world if rank == 0 else None
        dist.gather_object(None if xr is None else xr.numpy(), parts, dst=0)
        if rank == 0:
            xr_all = np.concatenate([p for p in parts if p is not None])
            q.put((full, xr_all, sf.eb_abs, sf.alpha, sf.n_outliers))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_world(case, world=2):
    """One gloo job of `world` spawned ranks; None if the rendezvous or a rank failed
    (the free port can be taken by another process between its probe and its use)."""
    import queue
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = q.get(timeout=120)
    except queue.Empty:
        res = None
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
            p.join()
        if p.exitcode != 0:
            res = None
    return res


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_equals_single_field(case):
    res = _run_world(case)
    if res is None:  # one retry on a fresh port
        res = _run_world(case)
    assert res is not None, "the world-2 gloo job failed twice"
    full, xr_all, eb_abs, alpha, n_out = res
    dims, kind, eps, mode, cfg = CASES[case]
    x = _field(kind, dims)
    ref_eb, e, twoe, inv2e = O.bounds_for(x, eps, mode)
    assert eb_abs == ref_eb
    assert alpha == (O.alpha(eps) if mode == "rel" else 1.0)
    ref = O.compress(x, cfg, e, twoe, inv2e, ref_eb)
    assert np.array_equal(full["codes"].numpy().astype(np.uint16), ref.codes.reshape(-1))
    assert np.array_equal(full["anchors"].numpy().view(np.uint32), ref.anchors.view(np.uint32))
    assert np.array_equal(full["out_idx"].numpy(), ref.out_idx.astype(np.int64))
    assert np.array_equal(full["out_val"].numpy().view(np.uint32), ref.out_val.view(np.uint32))
    assert np.array_equal(full["hist"].numpy(), O.histogram(ref.codes, cfg.radius).astype(np.int64))
    assert n_out == ref.n_outliers
    assert np.array_equal(xr_all.view(np.uint32), ref.xrec.view(np.uint32))
    if case == "split":
        assert ref.n_outliers > 0  # the outlier offsets were exercised


def test_sharding_rejects_1d_2d_geometry():
    from paper_2312_05492_gb300 import shard
    sl = shard.slabs(64, 2)[0]
    for ndim in (1, 2):
        with pytest.raises(ValueError):
            shard.compress(torch.zeros(sl.zc - sl.z0, 8, 8), sl, (64, 8, 8), 1e-3, O.Config(ndim=ndim), backend=None)
