"""The library's host codebook builder (interp_huffman_codebook) against the Huffman
oracle, on the CPU: identical lengths and canonical codewords, with and without the
length limit (the oracle's limited_lengths restates the limiting rule)."""
import numpy as np
import pytest

from oracle import huffman as H


@pytest.fixture(scope="module")
def G():
    from paper_2312_05492_gb300 import build, ginterp
    build.build()
    ginterp.load()
    return ginterp


def _skewed_hist(rng, R):
    """Two-sided geometric counts around the central code (the shape of quant-code
    histograms) with a random decay, so that deep trees and the limit occur."""
    k = np.abs(np.arange(2 * R) - R).astype(np.float64)
    w = np.floor((1 << 24) * np.exp(-k * rng.uniform(0.05, 3.0))) + (rng.random(2 * R) < 0.05)
    return w.astype(np.uint32)


@pytest.mark.parametrize("max_len", [24, 16, 12])
def test_codebook_matches_oracle(G, max_len):
    rng = np.random.default_rng(11 + max_len)
    limited = 0
    for i in range(120):
        R = int(rng.choice([2, 8, 64, 512, 4096]))
        if i % 2:
            hist = (rng.integers(0, 1 << 20, 2 * R) * (rng.random(2 * R) < rng.uniform(0.01, 1))).astype(np.uint32)
        else:
            hist = _skewed_hist(rng, R)
        if not hist.any():
            continue
        if np.count_nonzero(hist) > (1 << max_len):  # no code of max_len bits exists
            with pytest.raises(G.InterpError):
                G.huffman_codebook(hist, R, max_len)
            with pytest.raises(ValueError):
                H.limited_lengths(hist, max_len)
            continue
        lengths, cw = G.huffman_codebook(hist, R, max_len)
        ol = H.limited_lengths(hist, max_len)
        limited += int(H.huffman_lengths(hist).max() > max_len)
        assert np.array_equal(lengths.astype(np.int64), ol), (R, max_len)
        assert np.array_equal(cw.astype(np.uint64), H.canonical_codewords(ol))
        assert ol.max() <= max_len and H.kraft_sum(ol) <= 1.0
    if max_len < 24:
        assert limited > 10


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
    assert np.array_equal(lengths.astype(np.int64), H.limited_lengths(hist, max_len))
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
