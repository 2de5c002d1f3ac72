"""The OpenMP build of the oracle (points of one pass on several threads) gives the
same results as the single-threaded build: codes, anchors, outliers, reconstruction
and decompression bit for bit, in every geometry and neighbour domain."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture()
def restore_threads():
    yield
    O.set_threads(1)


CASES = [
    ((33, 40, 57), O.Config(order=(0, 1, 2), level_kind=(1, 1, 1), cubic_kind=(0, 0, 0))),
    ((25, 17, 96), O.Config(order=(2, 0, 1), level_kind=(0, 1, 1), cubic_kind=(1, 0, 1), radius=8)),
    ((17, 33, 65), O.Config(order=(1, 2, 0), level_kind=(1, 0, 1), cubic_kind=(0, 1, 1), domain_x=32)),
    ((6, 40, 48), O.Config(order=(2, 1, 0), level_kind=(1, 1, 1), cubic_kind=(1, 1, 1), ndim=2)),
    ((5, 3, 1500), O.Config(order=(2, 1, 0), level_kind=(1, 1, 1), cubic_kind=(0, 0, 1), ndim=1)),
]


@pytest.mark.parametrize("shape,cfg", CASES)
def test_threaded_oracle_is_bit_identical(shape, cfg, restore_threads):
    rng = np.random.default_rng(sum(shape))
    x = np.cumsum(rng.standard_normal(shape), axis=2).astype(np.float32)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-3, "rel", ndim=cfg.ndim)
    O.set_threads(1)
    a = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    da = O.decompress(a)
    assert O.set_threads(4) == 4
    b = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    db = O.decompress(b)
    assert np.array_equal(a.codes, b.codes)
    assert np.array_equal(a.anchors.view(np.uint32), b.anchors.view(np.uint32))
    assert a.n_outliers == b.n_outliers
    assert np.array_equal(a.out_idx, b.out_idx) and np.array_equal(a.out_val.view(np.uint32), b.out_val.view(np.uint32))
    assert np.array_equal(a.xrec.view(np.uint32), b.xrec.view(np.uint32))
    assert np.array_equal(da.view(np.uint32), db.view(np.uint32))
    assert np.array_equal(da.view(np.uint32), a.xrec.view(np.uint32))
