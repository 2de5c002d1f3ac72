"""Pins of the Huffman oracle (Sec. V-A lossless stage): closed forms and the
properties every optimal prefix code has, independent of its implementation."""
import math

import numpy as np

from oracle import huffman as H


def test_dyadic_frequencies_give_exact_lengths():
    # probabilities 1/2, 1/4, 1/8, 1/16, 1/16: the optimal code lengths are -log2 p
    hist = np.array([0, 8, 0, 4, 2, 1, 1], np.uint32)
    l = H.huffman_lengths(hist)
    assert list(l) == [0, 1, 0, 2, 3, 4, 4]
    assert H.kraft_sum(l) == 1.0


def test_single_and_two_symbols():
    assert list(H.huffman_lengths([0, 5, 0])) == [0, 1, 0]
    assert list(H.huffman_lengths([3, 0, 7])) == [1, 0, 1]
    assert list(H.huffman_lengths([0, 0])) == [0, 0]


def test_shannon_bound_and_complete_code():
    """Huffman's average length L satisfies H <= L < H + 1, and its code is complete
    (Kraft sum exactly 1) whenever two or more symbols occur."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        k = int(rng.integers(2, 300))
        hist = rng.integers(0, 1000, k).astype(np.uint32) * (rng.random(k) < 0.7)
        if np.count_nonzero(hist) < 2:
            continue
        l = H.huffman_lengths(hist)
        p = hist[hist > 0] / hist.sum()
        ent = float(-(p * np.log2(p)).sum())
        avg = float((hist * l).sum() / hist.sum())
        assert ent - 1e-12 <= avg < ent + 1
        assert math.isclose(H.kraft_sum(l), 1.0, rel_tol=0, abs_tol=1e-12)


def test_canonical_code_is_prefix_free():
    rng = np.random.default_rng(6)
    hist = rng.integers(1, 50, 40)
    l = H.huffman_lengths(hist)
    cw = H.canonical_codewords(l)
    words = [format(int(cw[s]), f"0{int(l[s])}b") for s in range(l.size)]
    for a in range(len(words)):
        for b in range(len(words)):
            if a != b:
                assert not words[b].startswith(words[a])


def test_encode_decode_roundtrip_and_sizes():
    rng = np.random.default_rng(7)
    R = 16
    codes = np.clip(np.rint(rng.standard_normal(5000) * 2) + R, 0, 2 * R - 1).astype(np.int64)
    hist = np.bincount(codes, minlength=2 * R)
    l = H.huffman_lengths(hist)
    cw = H.canonical_codewords(l)
    words, offs = H.encode_chunks(codes, l, cw, chunk=256)
    for k in range(len(offs) - 1):
        bits = int(l[codes[256 * k:256 * (k + 1)]].sum())
        assert offs[k + 1] - offs[k] == (bits + 31) // 32
    assert np.array_equal(H.decode_chunks(words, offs, codes.size, l, cw, chunk=256), codes)


def test_length_limit_worked_example():
    """Weights 1, 1, 2, 3, 5, 8: Huffman's lengths are 5, 5, 4, 3, 2, 1 (Kraft sum 1).
    Limited to 3 bits: cut to 3, 3, 3, 3, 2, 1 (Kraft 5/4); lengthen the longest code
    below 3 bits, symbol 4 (2 -> 3, Kraft 9/8); then symbol 5 (1 -> 2, Kraft 7/8)."""
    hist = np.array([1, 1, 2, 3, 5, 8], np.uint32)
    assert list(H.huffman_lengths(hist)) == [5, 5, 4, 3, 2, 1]
    l = H.limited_lengths(hist, 3)
    assert list(l) == [3, 3, 3, 3, 3, 2]
    assert H.kraft_sum(l) == 0.875
    assert list(H.limited_lengths(hist, 5)) == [5, 5, 4, 3, 2, 1]  # no length above the limit
    # ties on length go to the lighter symbol: weights 5, 4, 2, 3, 1, 1, 1 have Huffman
    # lengths 2, 2, 3, 3, 4, 4, 3; cut to 3 bits the Kraft sum is 9/8, and of the two
    # 2-bit codes the lighter one (symbol 1) is lengthened, which makes it exactly 1
    t = np.array([5, 4, 2, 3, 1, 1, 1], np.uint32)
    assert list(H.huffman_lengths(t)) == [2, 2, 3, 3, 4, 4, 3]
    assert list(H.limited_lengths(t, 3)) == [2, 3, 3, 3, 3, 3, 3]
