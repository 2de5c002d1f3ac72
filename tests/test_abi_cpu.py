"""Host-side checks of the C ABI (no GPU needed): the shared library loads,
exports every function declared in include/ginterp.h, its struct layouts match
the binding, and argument errors are rejected before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2312_05492_gb300 import build, ginterp
    build.build()
    return ginterp


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "sizeof", "return"):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("interp_compress", "interp_decompress", "qcode_histogram", "interp_autotune"):
        assert required in names


def test_library_exports_every_declared_function(G):
    lib = ctypes.CDLL(G.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(G.FUNCTIONS) <= set(_declared_functions())


def test_struct_layouts(G):
    assert ctypes.sizeof(G.interp_config) == 64
    assert ctypes.sizeof(G.interp_header) == 328
    assert G.interp_header.profile.offset == 184


def test_struct_layouts_match_the_c_header(G, tmp_path):
    """Every field offset and size of the structs the binding declares, against a C
    program compiled from include/ginterp.h (catches a field the binding lacks, or a
    type of the wrong width)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [G.interp_config, G.interp_header, G.interp_compress_item, G.interp_decompress_item,
               G.interp_tile_schedule]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ginterp.h"', 'int main(void) {']
    for st in structs:
        lines.append(f'printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            lines.append(f'printf("{st.__name__} {name} %zu\\n", offsetof({st.__name__}, {name}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert got[(st.__name__, name)] == getattr(st, name).offset, (st.__name__, name)


def test_anchor_count_and_workspace(G):
    assert G.interp_anchor_count((64, 64, 64)) == 512
    assert G.interp_anchor_count((449, 449, 235)) == 57 * 57 * 30
    assert G.interp_anchor_count((0, 4, 4)) == 0
    cfg = G.Config().to_c()
    ws = G.interp_workspace_bytes((512, 512, 512), cfg)
    assert ws >= 512 * 512 * 16 * 4  # one bitmap word per 32 x-positions
    bad = G.Config(dim_order=(0, 0, 1)).to_c()
    assert G.interp_workspace_bytes((8, 8, 8), bad) == 0
    assert G.interp_workspace_bytes((1 << 11, 1 << 11, 1 << 11), cfg) == 0  # N >= 2^32


@pytest.mark.parametrize("change", [
    dict(radius=1), dict(radius=40000), dict(dim_order=(0, 1, 1)), dict(level_kind=(2, 1, 1)),
    dict(cubic_kind=(0, 3, 0)),
])
def test_compress_rejects_bad_config(G, change):
    cfg = G.Config(**change).to_c()
    rc = G.interp_compress(1, (8, 8, 8), 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, 1, 1 << 20, None)
    assert rc == G.INTERP_EINVAL


def test_compress_rejects_bad_arguments(G):
    cfg = G.Config().to_c()
    ok = dict(d_x=1, dims=(8, 8, 8), eb=1e-3)
    assert G.interp_compress(1, (8, 8, 8), 0.0, cfg, 1, 1, 1, 1, 16, None, 1, 1, 1 << 20, None) == G.INTERP_EINVAL
    assert G.interp_compress(1, (8, 8, 8), float("nan"), cfg, 1, 1, 1, 1, 16, None, 1, 1, 1 << 20,
                             None) == G.INTERP_EINVAL
    assert G.interp_compress(None, (8, 8, 8), 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, 1, 1 << 20,
                             None) == G.INTERP_EINVAL
    assert G.interp_compress(1, (8, 0, 8), 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, 1, 1 << 20, None) == G.INTERP_EINVAL
    assert G.interp_compress(1, (8, 8, 8), 1e-3, cfg, 1, 1, None, 1, 16, None, 1, 1, 1 << 20,
                             None) == G.INTERP_EINVAL
    assert G.interp_compress(1, (8, 8, 8), 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, 1, 16, None) == G.INTERP_EWORKSPACE
    assert ok  # argument errors above never reached CUDA
    assert G.qcode_histogram(1, 10, 1, 1, None) == G.INTERP_EINVAL
    assert G.interp_decompress((8, 8, 8), None, 1, 1, 1, 1, 4, 1, None) == G.INTERP_EINVAL
    assert G.interp_status_string(G.INTERP_EWORKSPACE) == "workspace too small"


def test_binding_refuses_cpu_tensors(G):
    import torch
    with pytest.raises(G.InterpError):
        G.compress(torch.zeros(8, 8, 8), 1e-3)


def test_anchor_count_nd_matches_oracle(G):
    import oracle as O
    for dims in [(1, 17, 17), (3, 33, 40), (2, 3, 1025), (1, 1, 512), (5, 100, 7), (64, 1, 1 << 21)]:
        for ndim in (1, 2, 3):
            assert G.interp_anchor_count_nd(dims, ndim) == O.anchor_count(dims, ndim), (dims, ndim)
    assert G.interp_anchor_count_nd((8, 8, 8), 0) == G.interp_anchor_count((8, 8, 8))
    assert G.interp_anchor_count_nd((8, 8, 8), 4) == 0
    assert G.interp_anchor_count_nd((0, 8, 8), 2) == 0


@pytest.mark.parametrize("change", [dict(ndim=2, domain_x=32), dict(ndim=1, domain_x=32), dict(ndim=4),
                                    dict(ndim=-1)])
def test_nd_configuration_errors(G, change):
    cfg = G.Config(**change).to_c()
    assert G.interp_workspace_bytes((8, 8, 8), cfg) == 0
    rc = G.interp_compress(1, (8, 8, 8), 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, 1, 1 << 20, None)
    assert rc == G.INTERP_EINVAL


def test_decompress_nd_argument_errors(G):
    # rejected on the host, before anything is enqueued
    assert G.interp_decompress_nd(5, (8, 8, 8), 1, 1, 1, 1, 1, 16, 1, None) == G.INTERP_EINVAL
    assert G.interp_decompress_nd(2, (0, 8, 8), 1, 1, 1, 1, 1, 16, 1, None) == G.INTERP_EINVAL
    assert G.interp_decompress_nd(2, (8, 8, 8), None, 1, 1, 1, 1, 16, 1, None) == G.INTERP_EINVAL
    assert G.interp_decompress_nd(1, (8, 8, 8), 1, 1, 1, None, None, 16, 1, None) == G.INTERP_EINVAL


def test_huffman_sizes(G):
    lib = G.load()
    assert lib.interp_huffman_chunks(0) == 0 and lib.interp_huffman_chunks(1025) == 2
    assert lib.interp_huffman_capacity_words(1024, 16) >= 1024 * 16 // 32
    assert lib.interp_huffman_capacity_words(1024, 25) == 0
    assert lib.interp_huffman_workspace_bytes(1 << 27, 512) > lib.interp_huffman_workspace_bytes(1024, 512) > 0
    assert lib.interp_huffman_workspace_bytes(1024, 1) == 0
    assert lib.interp_huffman_workspace_bytes(1 << 32, 512) == 0
