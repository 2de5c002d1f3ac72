"""Python binding of libginterp.so (include/ginterp.h).

Argument marshalling only: torch supplies device memory and streams, every
computation runs in the library's CUDA kernels.  The low-level functions keep
the C names (interp_compress, interp_decompress, qcode_histogram,
interp_autotune, ...) and take raw pointers; ``compress`` / ``decompress``
wrap them for torch tensors.  There is no CPU fallback: if the library is
missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libginterp.so")

INTERP_OK, INTERP_EINVAL, INTERP_ECUDA, INTERP_EWORKSPACE, INTERP_ECAPACITY, INTERP_ENONFINITE = 0, -1, -2, -3, -4, -5
INTERP_ESCRATCH = -6
STATUS_CAPACITY, STATUS_NONFINITE, STATUS_TIMEOUT = 1, 2, 4

FUNCTIONS = ("interp_anchor_count", "interp_workspace_bytes", "interp_compress", "interp_decompress",
             "qcode_histogram", "interp_autotune", "interp_timing_enable", "interp_timing_read",
             "interp_compress_noalloc", "interp_noalloc_scratch_bytes", "interp_compress_batched",
             "interp_decompress_batched", "interp_status_string", "interp_alpha", "interp_value_range",
             "interp_quality_workspace_bytes", "interp_quality_report", "interp_huffman_codebook",
             "interp_huffman_chunks", "interp_huffman_capacity_words", "interp_huffman_workspace_bytes",
             "interp_huffman_encode", "interp_huffman_decode", "interp_anchor_count_nd", "interp_decompress_nd",
             "interp_compress_batched_scheduled", "interp_decompress_batched_scheduled", "interp_tune_batched")

# kernels each call launches, for one field or a whole batch: compress = zeroing +
# set-up (profile, range, bounds) + tiles + outlier scan + outlier write;
# decompress = outlier scatter + tiles
def launches_compress(cfg: "Config") -> int:
    return 5


LAUNCHES_DECOMPRESS = 2


class interp_config(ctypes.Structure):
    _fields_ = [("dim_order", ctypes.c_int32 * 3), ("level_kind", ctypes.c_int32 * 3),
                ("cubic_kind", ctypes.c_int32 * 3), ("eb_mode", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("domain_x", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("alpha", ctypes.c_double)]


class interp_header(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("cfg", interp_config), ("eb", ctypes.c_double),
                ("eb_abs", ctypes.c_double), ("alpha", ctypes.c_double), ("e", ctypes.c_float * 3),
                ("twoe", ctypes.c_float * 3), ("inv2e", ctypes.c_float * 3), ("vmin", ctypes.c_float),
                ("vmax", ctypes.c_float), ("n_outliers", ctypes.c_uint64), ("n_nonfinite", ctypes.c_uint64),
                ("status", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("profile", ctypes.c_double * 18)]


class interp_quality(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("n_outliers", ctypes.c_uint64), ("n_nonzero", ctypes.c_uint64),
                ("n_finite", ctypes.c_uint64), ("max_abs_q", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("entropy_bits", ctypes.c_double), ("sse", ctypes.c_double), ("max_abs_err", ctypes.c_double),
                ("vmin", ctypes.c_double), ("vmax", ctypes.c_double), ("psnr_db", ctypes.c_double)]


class interp_compress_item(ctypes.Structure):
    _fields_ = [("d_x", ctypes.c_void_p), ("dims", ctypes.c_int64 * 3), ("eb", ctypes.c_double),
                ("cfg", interp_config), ("d_anchors", ctypes.c_void_p), ("d_codes", ctypes.c_void_p),
                ("d_out_idx", ctypes.c_void_p), ("d_out_val", ctypes.c_void_p), ("out_capacity", ctypes.c_uint64),
                ("d_hist", ctypes.c_void_p), ("d_hdr", ctypes.c_void_p), ("d_ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t)]


class interp_tile_schedule(ctypes.Structure):
    _fields_ = [("run", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class interp_decompress_item(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("d_hdr", ctypes.c_void_p), ("d_anchors", ctypes.c_void_p),
                ("d_codes", ctypes.c_void_p), ("d_out_idx", ctypes.c_void_p), ("d_out_val", ctypes.c_void_p),
                ("out_capacity", ctypes.c_uint64), ("d_xrec", ctypes.c_void_p), ("ndim", ctypes.c_int32)]


MAX_BATCH = 16
HEADER_BYTES = ctypes.sizeof(interp_header)
_lib = None


class InterpError(RuntimeError):
    pass


def load() -> ctypes.CDLL:
    """Load libginterp.so (built by __graft_entry__.build() / build.py); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise InterpError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
    dims_t = ctypes.POINTER(ctypes.c_int64)
    cfg_p = ctypes.POINTER(interp_config)
    lib.interp_anchor_count.restype = ctypes.c_size_t
    lib.interp_anchor_count.argtypes = [dims_t]
    lib.interp_anchor_count_nd.restype = ctypes.c_size_t
    lib.interp_anchor_count_nd.argtypes = [dims_t, i32]
    lib.interp_decompress_nd.restype = ctypes.c_int
    lib.interp_decompress_nd.argtypes = [i32, dims_t, P, P, P, P, P, u64, P, P]
    lib.interp_workspace_bytes.restype = ctypes.c_size_t
    lib.interp_workspace_bytes.argtypes = [dims_t, cfg_p]
    lib.interp_compress.restype = ctypes.c_int
    lib.interp_compress.argtypes = [P, dims_t, ctypes.c_double, cfg_p, P, P, P, P, u64, P, P, P, ctypes.c_size_t, P]
    lib.interp_decompress.restype = ctypes.c_int
    lib.interp_decompress.argtypes = [dims_t, P, P, P, P, P, u64, P, P]
    lib.qcode_histogram.restype = ctypes.c_int
    lib.qcode_histogram.argtypes = [P, u64, i32, P, P]
    lib.interp_huffman_codebook.restype = ctypes.c_int
    lib.interp_huffman_codebook.argtypes = [P, i32, i32, P, P]
    lib.interp_huffman_chunks.restype = u64
    lib.interp_huffman_chunks.argtypes = [u64]
    lib.interp_huffman_capacity_words.restype = u64
    lib.interp_huffman_capacity_words.argtypes = [u64, i32]
    lib.interp_huffman_workspace_bytes.restype = ctypes.c_size_t
    lib.interp_huffman_workspace_bytes.argtypes = [u64, i32]
    lib.interp_huffman_encode.restype = ctypes.c_int
    lib.interp_huffman_encode.argtypes = [P, u64, i32, P, P, P, P, u64, P, ctypes.c_size_t, P]
    lib.interp_huffman_decode.restype = ctypes.c_int
    lib.interp_huffman_decode.argtypes = [P, P, u64, i32, P, P, P, P, ctypes.c_size_t, P]
    lib.interp_quality_workspace_bytes.restype = ctypes.c_size_t
    lib.interp_quality_workspace_bytes.argtypes = []
    lib.interp_quality_report.restype = ctypes.c_int
    lib.interp_quality_report.argtypes = [P, i32, P, P, u64, P, P, ctypes.c_size_t, P]
    lib.interp_alpha.restype = ctypes.c_double
    lib.interp_alpha.argtypes = [ctypes.c_double]
    lib.interp_value_range.restype = ctypes.c_int
    lib.interp_value_range.argtypes = [P, dims_t, P, P, ctypes.c_size_t, P]
    lib.interp_autotune.restype = ctypes.c_int
    lib.interp_autotune.argtypes = [P, dims_t, cfg_p, P, P, ctypes.c_size_t, P]
    lib.interp_timing_enable.restype = ctypes.c_int
    lib.interp_timing_enable.argtypes = [ctypes.c_int]
    lib.interp_timing_read.restype = ctypes.c_int
    lib.interp_timing_read.argtypes = [P, P, P, P]
    lib.interp_compress_noalloc.restype = ctypes.c_int
    lib.interp_compress_noalloc.argtypes = [P, dims_t, ctypes.c_double, cfg_p, P, P, P, P, u64, P, P, P]
    lib.interp_noalloc_scratch_bytes.restype = ctypes.c_size_t
    lib.interp_noalloc_scratch_bytes.argtypes = []
    lib.interp_compress_batched.restype = ctypes.c_int
    lib.interp_compress_batched.argtypes = [ctypes.POINTER(interp_compress_item), ctypes.c_int, P]
    lib.interp_decompress_batched.restype = ctypes.c_int
    lib.interp_decompress_batched.argtypes = [ctypes.POINTER(interp_decompress_item), ctypes.c_int, P]
    sched_p = ctypes.POINTER(interp_tile_schedule)
    lib.interp_compress_batched_scheduled.restype = ctypes.c_int
    lib.interp_compress_batched_scheduled.argtypes = [ctypes.POINTER(interp_compress_item), ctypes.c_int, sched_p, P]
    lib.interp_decompress_batched_scheduled.restype = ctypes.c_int
    lib.interp_decompress_batched_scheduled.argtypes = [ctypes.POINTER(interp_decompress_item), ctypes.c_int,
                                                        sched_p, P]
    lib.interp_tune_batched.restype = ctypes.c_int
    lib.interp_tune_batched.argtypes = [ctypes.POINTER(interp_compress_item), ctypes.POINTER(interp_decompress_item),
                                        ctypes.c_int, i32, sched_p, sched_p, P]
    lib.interp_status_string.restype = ctypes.c_char_p
    lib.interp_status_string.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def _dims(dims) -> ctypes.Array:
    return (ctypes.c_int64 * 3)(*[int(d) for d in dims])


def _check(rc: int, what: str):
    if rc != INTERP_OK:
        msg = load().interp_status_string(rc).decode()
        raise InterpError(f"{what} failed: {msg} ({rc})")


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ----------------------------------------------------------- C-name entry points
def interp_anchor_count(dims) -> int:
    return int(load().interp_anchor_count(_dims(dims)))


def interp_anchor_count_nd(dims, ndim: int) -> int:
    return int(load().interp_anchor_count_nd(_dims(dims), int(ndim)))


def interp_decompress_nd(ndim, dims, d_hdr, d_anchors, d_codes, d_out_idx, d_out_val, out_capacity, d_xrec,
                         stream) -> int:
    return load().interp_decompress_nd(int(ndim), _dims(dims), d_hdr, d_anchors, d_codes, d_out_idx, d_out_val,
                                       int(out_capacity), d_xrec, stream)


def interp_workspace_bytes(dims, cfg: interp_config) -> int:
    return int(load().interp_workspace_bytes(_dims(dims), ctypes.byref(cfg)))


def interp_compress(d_x, dims, eb, cfg, d_anchors, d_codes, d_out_idx, d_out_val, out_capacity, d_hist, d_hdr,
                    d_ws, ws_bytes, stream) -> int:
    return load().interp_compress(d_x, _dims(dims), float(eb), ctypes.byref(cfg), d_anchors, d_codes, d_out_idx,
                                  d_out_val, int(out_capacity), d_hist, d_hdr, d_ws, int(ws_bytes), stream)


def interp_decompress(dims, d_hdr, d_anchors, d_codes, d_out_idx, d_out_val, out_capacity, d_xrec, stream) -> int:
    return load().interp_decompress(_dims(dims), d_hdr, d_anchors, d_codes, d_out_idx, d_out_val, int(out_capacity),
                                    d_xrec, stream)


def qcode_histogram(d_codes, n, radius, d_hist, stream) -> int:
    return load().qcode_histogram(d_codes, int(n), int(radius), d_hist, stream)


def interp_quality_workspace_bytes() -> int:
    return int(load().interp_quality_workspace_bytes())


def interp_quality_report(d_hist, radius, d_x, d_xrec, n, d_out, d_ws, ws_bytes, stream) -> int:
    return load().interp_quality_report(d_hist, int(radius), d_x, d_xrec, int(n), d_out, d_ws, int(ws_bytes), stream)


def interp_alpha(eps: float) -> float:
    return float(load().interp_alpha(float(eps)))


def interp_value_range(d_x, dims, d_range, d_ws, ws_bytes, stream) -> int:
    return load().interp_value_range(d_x, _dims(dims), d_range, d_ws, int(ws_bytes), stream)


def interp_autotune(d_x, dims, cfg: interp_config, h_profile, d_ws, ws_bytes, stream) -> int:
    return load().interp_autotune(d_x, _dims(dims), ctypes.byref(cfg), h_profile, d_ws, int(ws_bytes), stream)


def interp_timing_enable(on: bool) -> int:
    return load().interp_timing_enable(1 if on else 0)


def interp_timing_read():
    """(compress_ms, compress_launches, decompress_ms, decompress_launches) of the tile kernels."""
    cm, dm = ctypes.c_double(), ctypes.c_double()
    cn, dn = ctypes.c_int32(), ctypes.c_int32()
    _check(load().interp_timing_read(ctypes.byref(cm), ctypes.byref(cn), ctypes.byref(dm), ctypes.byref(dn)),
           "interp_timing_read")
    return cm.value, cn.value, dm.value, dn.value


def interp_compress_noalloc(d_x, dims, eb, cfg, d_anchors, d_codes, d_out_idx, d_out_val, out_capacity, d_hist,
                            d_hdr, stream) -> int:
    """interp_compress for callers that cannot allocate device memory: the scratch is the
    library's built-in array (interp_noalloc_scratch_bytes()), shared by all calls."""
    return load().interp_compress_noalloc(d_x, _dims(dims), float(eb), ctypes.byref(cfg), d_anchors, d_codes,
                                          d_out_idx, d_out_val, int(out_capacity), d_hist, d_hdr, stream)


def interp_noalloc_scratch_bytes() -> int:
    return int(load().interp_noalloc_scratch_bytes())


def interp_compress_batched(items, stream) -> int:
    arr = (interp_compress_item * len(items))(*items)
    return load().interp_compress_batched(arr, len(items), stream)


def interp_decompress_batched(items, stream) -> int:
    arr = (interp_decompress_item * len(items))(*items)
    return load().interp_decompress_batched(arr, len(items), stream)


def interp_compress_batched_scheduled(items, sched, stream) -> int:
    arr = (interp_compress_item * len(items))(*items)
    return load().interp_compress_batched_scheduled(arr, len(items), ctypes.byref(sched) if sched else None, stream)


def interp_decompress_batched_scheduled(items, sched, stream) -> int:
    arr = (interp_decompress_item * len(items))(*items)
    return load().interp_decompress_batched_scheduled(arr, len(items), ctypes.byref(sched) if sched else None, stream)


def interp_tune_batched(citems, ditems, stream, force: bool = False):
    """(compression schedule, decompression schedule) the library's autotuner picks."""
    ca = (interp_compress_item * len(citems))(*citems)
    da = (interp_decompress_item * len(ditems))(*ditems)
    cs, ds = interp_tile_schedule(), interp_tile_schedule()
    _check(load().interp_tune_batched(ca, da, len(citems), int(force), ctypes.byref(cs), ctypes.byref(ds), stream),
           "interp_tune_batched")
    return cs, ds


def interp_status_string(rc: int) -> str:
    return load().interp_status_string(int(rc)).decode()


# ---------------------------------------------------------------- torch API
@dataclass
class Config:
    """Interpolation configuration (Sec. IV-B); mirrors interp_config.

    level_kind is indexed by level l (stride 2**l): 0 = linear only, 1 = splines.
    cubic_kind is indexed by axis (0=z, 1=y, 2=x): 0 = not-a-knot, 1 = natural.
    domain_x: neighbour domain along x, 8 (the 8^3 chunk) or 32 (the x-extended block).
    ndim: chunk geometry (Sec. IV-A): 3 = 8^3 chunks; 2 = 16^2 chunks over (y, x) of
      every z-slice; 1 = 512-point chunks along x of every row.  Levels coarser than
      stride 4 follow level_kind[2].
    """
    dim_order: tuple = (0, 1, 2)
    level_kind: tuple = (1, 1, 1)
    cubic_kind: tuple = (0, 0, 0)
    eb_mode: str = "rel"
    autotune: bool = False
    radius: int = 512
    alpha: float = 0.0
    domain_x: int = 8
    ndim: int = 3

    def to_c(self) -> interp_config:
        c = interp_config()
        c.dim_order[:] = [int(v) for v in self.dim_order]
        c.level_kind[:] = [int(v) for v in self.level_kind]
        c.cubic_kind[:] = [int(v) for v in self.cubic_kind]
        c.eb_mode = 1 if self.eb_mode == "rel" else 0
        c.autotune = 1 if self.autotune else 0
        c.radius = int(self.radius)
        c.domain_x = int(self.domain_x)
        c.ndim = int(self.ndim)
        c.alpha = float(self.alpha)
        return c


@dataclass
class CompressedField:
    """Device-resident result of compress(): the header, anchors, quant-codes,
    outlier list (capacity entries, the first n_outliers valid) and histogram."""
    dims: tuple
    cfg: Config
    header: torch.Tensor      # uint8[HEADER_BYTES]
    anchors: torch.Tensor     # float32
    codes: torch.Tensor       # int16 storage of uint16 codes
    out_idx: torch.Tensor     # int32 storage of uint32 indices
    out_val: torch.Tensor     # float32
    hist: torch.Tensor | None  # int32 storage of uint32 counts
    capacity: int
    _host_header: interp_header | None = field(default=None, repr=False)

    def host_header(self, refresh: bool = False) -> interp_header:
        """Copy the device header to the host (synchronises the current stream)."""
        if self._host_header is None or refresh:
            h = interp_header()
            buf = self.header.cpu().numpy().tobytes()
            ctypes.memmove(ctypes.addressof(h), buf, HEADER_BYTES)
            self._host_header = h
        return self._host_header

    @property
    def n_outliers(self) -> int:
        return int(self.host_header().n_outliers)

    @property
    def status(self) -> int:
        return int(self.host_header().status)

    def nbytes(self) -> int:
        n = min(self.n_outliers, self.capacity)
        return HEADER_BYTES + self.anchors.numel() * 4 + self.codes.numel() * 2 + n * 8


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else int(t.data_ptr())


def _check_field(x: torch.Tensor):
    if not isinstance(x, torch.Tensor) or x.dtype != torch.float32 or x.dim() != 3 or not x.is_cuda:
        raise InterpError("expected a float32 3-D CUDA tensor")
    if not x.is_contiguous():
        raise InterpError("expected a contiguous tensor")


class Workspace:
    """Reusable device scratch for compress(); grows on demand."""

    def __init__(self, device=None):
        self.device = device
        self.buf: torch.Tensor | None = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
        return self.buf


_default_ws: dict = {}


def default_capacity(n: int) -> int:
    """Initial outlier capacity: N/64 entries (grown on overflow by compress)."""
    return max(1024, n // 64)


def allocate(dims, cfg: Config, device, capacity: int | None = None, hist: bool = True):
    n = int(dims[0]) * int(dims[1]) * int(dims[2])
    cap = default_capacity(n) if capacity is None else int(capacity)
    return dict(
        header=torch.zeros(HEADER_BYTES, dtype=torch.uint8, device=device),
        anchors=torch.empty(interp_anchor_count_nd(dims, cfg.ndim), dtype=torch.float32, device=device),
        codes=torch.empty(n, dtype=torch.int16, device=device),
        out_idx=torch.empty(max(cap, 1), dtype=torch.int32, device=device),
        out_val=torch.empty(max(cap, 1), dtype=torch.float32, device=device),
        hist=torch.empty(2 * int(cfg.radius), dtype=torch.int32, device=device) if hist else None,
        capacity=cap,
    )


def compress_into(x: torch.Tensor, eb: float, cfg: Config, bufs: dict, ws: torch.Tensor, stream=None) -> None:
    """Enqueue interp_compress on preallocated buffers (no synchronisation)."""
    dims = tuple(x.shape)
    rc = interp_compress(_ptr(x), dims, eb, cfg.to_c(), _ptr(bufs["anchors"]), _ptr(bufs["codes"]),
                         _ptr(bufs["out_idx"]), _ptr(bufs["out_val"]), bufs["capacity"], _ptr(bufs["hist"]),
                         _ptr(bufs["header"]), _ptr(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "interp_compress")


def decompress_into(cf: CompressedField, out: torch.Tensor, stream=None) -> None:
    if cf.cfg.ndim in (1, 2):
        rc = interp_decompress_nd(cf.cfg.ndim, cf.dims, _ptr(cf.header), _ptr(cf.anchors), _ptr(cf.codes),
                                  _ptr(cf.out_idx), _ptr(cf.out_val), cf.capacity, _ptr(out), _stream_ptr(stream))
    else:
        rc = interp_decompress(cf.dims, _ptr(cf.header), _ptr(cf.anchors), _ptr(cf.codes), _ptr(cf.out_idx),
                               _ptr(cf.out_val), cf.capacity, _ptr(out), _stream_ptr(stream))
    _check(rc, "interp_decompress")


def compress(x: torch.Tensor, eb: float, cfg: Config | None = None, capacity: int | None = None,
             hist: bool = True, workspace: Workspace | None = None, stream=None,
             grow_on_overflow: bool = True) -> CompressedField:
    """Compress a float32 CUDA field.  With grow_on_overflow the call checks the
    outlier count (one device-to-host read) and recompresses with a larger
    outlier buffer if the first capacity was too small."""
    _check_field(x)
    cfg = cfg or Config()
    dims = tuple(int(d) for d in x.shape)
    ccfg = cfg.to_c()
    wsb = interp_workspace_bytes(dims, ccfg)
    if wsb == 0:
        raise InterpError("invalid dims or configuration")
    ws_obj = workspace or _default_ws.setdefault(x.device, Workspace())
    ws = ws_obj.get(wsb, x.device)
    bufs = allocate(dims, cfg, x.device, capacity, hist)
    compress_into(x, eb, cfg, bufs, ws, stream)
    cf = CompressedField(dims, cfg, bufs["header"], bufs["anchors"], bufs["codes"], bufs["out_idx"],
                         bufs["out_val"], bufs["hist"], bufs["capacity"])
    if grow_on_overflow:
        h = cf.host_header(refresh=True)
        if h.status & STATUS_CAPACITY:
            return compress(x, eb, cfg, capacity=int(h.n_outliers), hist=hist, workspace=ws_obj, stream=stream,
                            grow_on_overflow=False)
    return cf


def decompress(cf: CompressedField, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(cf.dims, dtype=torch.float32, device=cf.codes.device)
    decompress_into(cf, out, stream)
    return out


def histogram(codes: torch.Tensor, radius: int, stream=None) -> torch.Tensor:
    hist = torch.empty(2 * int(radius), dtype=torch.int32, device=codes.device)
    rc = qcode_histogram(_ptr(codes), codes.numel(), radius, _ptr(hist), _stream_ptr(stream))
    _check(rc, "qcode_histogram")
    return hist


def value_range(x: torch.Tensor, workspace: Workspace | None = None, stream=None) -> torch.Tensor:
    """{vmin, vmax} over the finite values of x, as a 2-float CUDA tensor (no sync)."""
    _check_field(x)
    dims = tuple(int(d) for d in x.shape)
    wsb = interp_workspace_bytes(dims, Config().to_c())
    ws = (workspace or _default_ws.setdefault(x.device, Workspace())).get(wsb, x.device)
    out = torch.empty(2, dtype=torch.float32, device=x.device)
    _check(interp_value_range(_ptr(x), dims, _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream)),
           "interp_value_range")
    return out


def quality(cf: "CompressedField", x: torch.Tensor | None = None, xrec: torch.Tensor | None = None,
            stream=None) -> dict:
    """Quality report of a compressed field (histogram entropy and code counts; with x
    and xrec also the error statistics and PSNR).  Synchronises the stream."""
    if cf.hist is None:
        raise InterpError("the field was compressed without a histogram")
    dev = cf.codes.device
    out = torch.zeros(ctypes.sizeof(interp_quality), dtype=torch.uint8, device=dev)
    ws = torch.empty(interp_quality_workspace_bytes(), dtype=torch.uint8, device=dev)
    if (x is None) != (xrec is None):
        raise InterpError("give both x and xrec, or neither")
    n = int(x.numel()) if x is not None else 0
    rc = interp_quality_report(_ptr(cf.hist), cf.cfg.radius, _ptr(x), _ptr(xrec), n, _ptr(out), _ptr(ws),
                               ws.numel(), _stream_ptr(stream))
    _check(rc, "interp_quality_report")
    host = out.cpu().numpy().tobytes()
    q = interp_quality.from_buffer_copy(host)
    return {name: getattr(q, name) for name, _ in interp_quality._fields_ if name != "reserved"}


def huffman_codebook(hist, radius: int, max_len: int = 16):
    """Canonical Huffman codebook (host) from a 2R-bin histogram (numpy array or tensor):
    (lengths uint8[2R], codewords uint32[2R]) as numpy arrays."""
    import numpy as np
    a = np.asarray(hist.cpu().numpy() if isinstance(hist, torch.Tensor) else hist)
    h = np.ascontiguousarray(a.view(np.uint32) if a.dtype.itemsize == 4 and a.dtype.kind in "iu" else a.astype(np.uint32))
    lengths = np.zeros(2 * radius, np.uint8)
    codewords = np.zeros(2 * radius, np.uint32)
    rc = load().interp_huffman_codebook(h.ctypes.data, int(radius), int(max_len), lengths.ctypes.data,
                                        codewords.ctypes.data)
    _check(rc, "interp_huffman_codebook")
    return lengths, codewords


@dataclass
class HuffmanStream:
    """Device-resident Huffman stream of n codes (chunks of 1024 codes)."""
    n: int
    radius: int
    lengths: torch.Tensor    # uint8 [2R] (device)
    codewords: torch.Tensor  # int32 storage of uint32 [2R] (device)
    offsets: torch.Tensor    # int32 storage of uint32 [chunks + 1]
    words: torch.Tensor      # int32 storage of uint32 [capacity]
    flag: torch.Tensor       # workspace; its first word is the error flag

    def total_words(self) -> int:
        return int(self.offsets[-1].item()) & 0xFFFFFFFF

    def nbytes(self) -> int:
        return 4 * self.total_words() + 4 * self.offsets.numel()


def huffman_encode(codes: torch.Tensor, radius: int, lengths, codewords, max_len: int = 16, stream=None,
                   ws: torch.Tensor | None = None) -> HuffmanStream:
    """Encode uint16 codes (an int16 tensor) on the device with a host codebook."""
    import numpy as np
    dev = codes.device
    n = int(codes.numel())
    d_len = torch.from_numpy(np.ascontiguousarray(lengths, np.uint8)).to(dev)
    d_cw = torch.from_numpy(np.ascontiguousarray(codewords, np.uint32).view(np.int32)).to(dev)
    nch = int(load().interp_huffman_chunks(n))
    cap = int(load().interp_huffman_capacity_words(n, int(max_len)))
    offsets = torch.empty(nch + 1, dtype=torch.int32, device=dev)
    words = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    wsb = int(load().interp_huffman_workspace_bytes(n, int(radius)))
    if ws is None or ws.numel() < wsb:
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    rc = load().interp_huffman_encode(_ptr(codes), n, int(radius), _ptr(d_len), _ptr(d_cw), _ptr(offsets),
                                      _ptr(words), cap, _ptr(ws), ws.numel(), _stream_ptr(stream))
    _check(rc, "interp_huffman_encode")
    return HuffmanStream(n, int(radius), d_len, d_cw, offsets, words, ws)


def huffman_reencode(hs: HuffmanStream, codes: torch.Tensor, stream=None) -> HuffmanStream:
    """Encode codes again into an existing stream's buffers with its codebook (no
    allocation, no host work: only the encoder's launches)."""
    n = int(codes.numel())
    if n != hs.n:
        raise ValueError(f"stream holds {hs.n} codes, got {n}")
    rc = load().interp_huffman_encode(_ptr(codes), n, hs.radius, _ptr(hs.lengths), _ptr(hs.codewords),
                                      _ptr(hs.offsets), _ptr(hs.words), hs.words.numel(), _ptr(hs.flag),
                                      hs.flag.numel(), _stream_ptr(stream))
    _check(rc, "interp_huffman_encode")
    return hs


def huffman_decode(hs: HuffmanStream, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Decode a stream back into uint16 codes (an int16 tensor)."""
    dev = hs.words.device
    if out is None:
        out = torch.empty(hs.n, dtype=torch.int16, device=dev)
    rc = load().interp_huffman_decode(_ptr(hs.words), _ptr(hs.offsets), hs.n, hs.radius, _ptr(hs.lengths),
                                      _ptr(hs.codewords), _ptr(out), _ptr(hs.flag), hs.flag.numel(),
                                      _stream_ptr(stream))
    _check(rc, "interp_huffman_decode")
    return out


def autotune(x: torch.Tensor, radius: int = 512, stream=None, ndim: int = 3):
    """Sampling profile + decision on the device; returns (Config, profile sums)."""
    _check_field(x)
    c = interp_config()
    c.radius = radius
    c.ndim = int(ndim)
    prof = (ctypes.c_double * 18)()
    ws = torch.empty(HEADER_BYTES, dtype=torch.uint8, device=x.device)
    rc = interp_autotune(_ptr(x), tuple(x.shape), c, ctypes.addressof(prof), _ptr(ws), ws.numel(),
                         _stream_ptr(stream))
    _check(rc, "interp_autotune")
    cfg = Config(dim_order=tuple(c.dim_order), level_kind=tuple(c.level_kind), cubic_kind=tuple(c.cubic_kind),
                 radius=radius, ndim=int(ndim))
    return cfg, [float(v) for v in prof]


# ------------------------------------------------------------ batched torch API
def compress_item(x: torch.Tensor, eb: float, cfg: Config, bufs: dict, ws: torch.Tensor) -> interp_compress_item:
    it = interp_compress_item()
    it.d_x = _ptr(x)
    it.dims[:] = [int(d) for d in x.shape]
    it.eb = float(eb)
    it.cfg = cfg.to_c()
    it.d_anchors = _ptr(bufs["anchors"])
    it.d_codes = _ptr(bufs["codes"])
    it.d_out_idx = _ptr(bufs["out_idx"])
    it.d_out_val = _ptr(bufs["out_val"])
    it.out_capacity = int(bufs["capacity"])
    it.d_hist = _ptr(bufs["hist"])
    it.d_hdr = _ptr(bufs["header"])
    it.d_ws = _ptr(ws)
    it.ws_bytes = int(ws.numel())
    return it


def decompress_item(cf: CompressedField, out: torch.Tensor) -> interp_decompress_item:
    it = interp_decompress_item()
    it.dims[:] = [int(d) for d in cf.dims]
    it.d_hdr = _ptr(cf.header)
    it.d_anchors = _ptr(cf.anchors)
    it.d_codes = _ptr(cf.codes)
    it.d_out_idx = _ptr(cf.out_idx)
    it.d_out_val = _ptr(cf.out_val)
    it.out_capacity = int(cf.capacity)
    it.d_xrec = _ptr(out)
    it.ndim = int(cf.cfg.ndim)
    return it


class Batch:
    """Preallocated buffers for compressing / decompressing a fixed set of fields
    together: one persistent tile launch per call for all fields.  Reusable, and
    capturable into a CUDA graph once it has run once (no host synchronisation)."""

    def __init__(self, xs, ebs, cfgs, capacities=None, hist=True):
        if not 1 <= len(xs) <= MAX_BATCH:
            raise InterpError(f"a batch holds 1..{MAX_BATCH} fields")
        for x in xs:
            _check_field(x)
        self.xs = list(xs)
        self.ebs = [float(e) for e in ebs]
        self.cfgs = list(cfgs)
        caps = capacities or [None] * len(xs)
        self.bufs = [allocate(tuple(x.shape), c, x.device, capacity=cap, hist=hist)
                     for x, c, cap in zip(self.xs, self.cfgs, caps)]
        self.ws = [torch.empty(max(1, interp_workspace_bytes(tuple(x.shape), c.to_c())), dtype=torch.uint8,
                               device=x.device) for x, c in zip(self.xs, self.cfgs)]
        self.fields = [CompressedField(tuple(x.shape), c, b["header"], b["anchors"], b["codes"], b["out_idx"],
                                       b["out_val"], b["hist"], b["capacity"])
                       for x, c, b in zip(self.xs, self.cfgs, self.bufs)]
        self.outs = [torch.empty_like(x) for x in self.xs]
        self._citems = [compress_item(x, e, c, b, w) for x, e, c, b, w in
                        zip(self.xs, self.ebs, self.cfgs, self.bufs, self.ws)]
        self._ditems = [decompress_item(cf, o) for cf, o in zip(self.fields, self.outs)]
        self.csched = self.dsched = None  # tile schedules (None: the library's cost model)

    def tune(self, stream=None, force: bool = False):
        """Let the library's autotuner pick the tile schedules of this batch (times the
        candidates on the device; cached by the batch's shapes).  Synchronises."""
        self.csched, self.dsched = interp_tune_batched(self._citems, self._ditems, _stream_ptr(stream), force)
        return self.csched, self.dsched

    def compress(self, stream=None):
        _check(interp_compress_batched_scheduled(self._citems, self.csched, _stream_ptr(stream)),
               "interp_compress_batched")

    def decompress(self, stream=None):
        _check(interp_decompress_batched_scheduled(self._ditems, self.dsched, _stream_ptr(stream)),
               "interp_decompress_batched")

    def round_trip(self, stream=None):
        self.compress(stream)
        self.decompress(stream)
