"""The library's host codebook builder (interp_huffman_codebook) against the Huffman
oracle, on the CPU: identical lengths and canonical codewords whenever no codeword
exceeds the limit; a valid limited prefix code otherwise."""
import numpy as np
import pytest

from oracle import huffman as H


@pytest.fixture(scope="module")
def G():
    from paper_2312_05492_gb300 import build, ginterp
    build.build()
    ginterp.load()
    return ginterp


def test_codebook_matches_oracle(G):
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(150):
        R = int(rng.choice([2, 8, 64, 512, 4096]))
        hist = (rng.integers(0, 1 << 20, 2 * R) * (rng.random(2 * R) < rng.uniform(0.01, 1))).astype(np.uint32)
        lengths, cw = G.huffman_codebook(hist, R, 24)
        ol = H.huffman_lengths(hist)
        if ol.max() > 24:
            continue
        assert np.array_equal(lengths.astype(np.int64), ol)
        assert np.array_equal(cw.astype(np.uint64), H.canonical_codewords(ol))
        checked += 1
    assert checked > 100


def _fibonacci_hist(k):
    f = [1, 1]
    while len(f) < k:
        f.append(f[-1] + f[-2])
    return np.array(f, np.uint32)


@pytest.mark.parametrize("max_len", [8, 12, 16])
def test_length_limit_gives_a_valid_prefix_code(G, max_len):
    """Fibonacci weights make Huffman's tree as deep as the alphabet: the limit is hit."""
    hist = np.zeros(64, np.uint32)
    hist[:30] = _fibonacci_hist(30)
    assert H.huffman_lengths(hist).max() > max_len
    lengths, cw = G.huffman_codebook(hist, 32, max_len)
    assert lengths.max() <= max_len and np.all(lengths[:30] > 0) and np.all(lengths[30:] == 0)
    assert H.kraft_sum(lengths) <= 1.0
    assert np.array_equal(cw.astype(np.uint64), H.canonical_codewords(lengths.astype(np.int64)))
    words = [format(int(cw[s]), f"0{int(lengths[s])}b") for s in range(30)]
    for a in range(30):
        for b in range(30):
            assert a == b or not words[b].startswith(words[a])


def test_codebook_argument_errors(G):
    h = np.ones(16, np.uint32)
    with pytest.raises(G.InterpError):
        G.huffman_codebook(h, 8, 25)
    with pytest.raises(G.InterpError):
        G.huffman_codebook(h, 8, 0)
    l, c = G.huffman_codebook(np.zeros(16, np.uint32), 8, 16)
    assert not l.any()
