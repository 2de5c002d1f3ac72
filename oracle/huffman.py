"""Canonical Huffman coding of quant-codes, written from its definition (the
lossless stage after the histogram, Sec. V-A: a codebook built on the host from
the histogram, then the codes encoded with it).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python and numpy; no
code shared with the CUDA library.

Stream format (the one the library's encoder writes): the codes are cut into
chunks of `chunk` consecutive codes; each chunk's codewords are concatenated
most-significant bit first into 32-bit words (the first bit of the chunk is
bit 31 of its first word) and the chunk is padded with zero bits to a whole
word; offsets[k] is the first word of chunk k and offsets[-1] the total.
"""
from __future__ import annotations

import heapq

import numpy as np


def huffman_lengths(hist) -> np.ndarray:
    """Code lengths of an optimal prefix code (Huffman's construction): repeatedly
    merge the two lightest subtrees; a symbol's length is its leaf depth.  Ties are
    broken by creation order (symbols by index first, merged nodes after), so the
    result is deterministic.  Unused symbols get length 0; a single used symbol
    gets length 1."""
    h = np.asarray(hist, dtype=np.int64).reshape(-1)
    used = [int(s) for s in np.flatnonzero(h)]
    lengths = np.zeros(h.size, np.int64)
    if not used:
        return lengths
    if len(used) == 1:
        lengths[used[0]] = 1
        return lengths
    heap = [(int(h[s]), s, [s]) for s in used]
    heapq.heapify(heap)
    seq = h.size
    while len(heap) > 1:
        w1, _, a = heapq.heappop(heap)
        w2, _, b = heapq.heappop(heap)
        for s in a + b:
            lengths[s] += 1
        heapq.heappush(heap, (w1 + w2, seq, a + b))
        seq += 1
    return lengths


def limited_lengths(hist, max_len: int) -> np.ndarray:
    """Huffman's lengths (huffman_lengths) limited to max_len bits.  The paper builds
    the codebook on the host and names no limit; the reading taken here: when some
    length exceeds max_len, every length above it is cut to max_len; then, while the
    Kraft sum of the used symbols exceeds 1, the codeword that is longest among those
    shorter than max_len is lengthened by one bit (on equal lengths the lighter
    symbol, on equal weights the higher symbol index).  The Kraft sum is kept as an
    exact rational."""
    from fractions import Fraction
    h = np.asarray(hist, dtype=np.int64).reshape(-1)
    lengths = huffman_lengths(h)
    used = [int(s) for s in np.flatnonzero(h)]
    if not used or int(lengths.max()) <= max_len:
        return lengths
    if len(used) > (1 << max_len):
        raise ValueError("more symbols than codewords of max_len bits")
    for s in used:
        lengths[s] = min(int(lengths[s]), max_len)
    kraft = sum(Fraction(1, 1 << int(lengths[s])) for s in used)
    while kraft > 1:
        shorter = [s for s in used if lengths[s] < max_len]
        s = max(shorter, key=lambda t: (int(lengths[t]), -int(h[t]), t))
        kraft -= Fraction(1, 1 << (int(lengths[s]) + 1))
        lengths[s] += 1
    return lengths


def kraft_sum(lengths) -> float:
    l = np.asarray(lengths)
    l = l[l > 0]
    return float(np.sum(2.0 ** (-l.astype(np.float64))))


def canonical_codewords(lengths) -> np.ndarray:
    """Canonical prefix code for the given lengths: symbols ordered by (length,
    symbol) receive consecutive codewords, shifted left whenever the length grows."""
    l = np.asarray(lengths, dtype=np.int64)
    cw = np.zeros(l.size, np.uint64)
    order = sorted((int(l[s]), s) for s in np.flatnonzero(l))
    code, prev = 0, 0
    for length, s in order:
        code <<= (length - prev)
        cw[s] = code
        code += 1
        prev = length
    return cw


def encode_chunks(codes, lengths, codewords, chunk: int = 1024):
    """The stream of the module docstring: (words uint32[], offsets uint32[nchunks + 1])."""
    c = np.asarray(codes, dtype=np.int64).reshape(-1)
    nch = (c.size + chunk - 1) // chunk
    words, offsets = [], [0]
    for k in range(nch):
        acc, nbits = 0, 0
        for s in c[k * chunk:(k + 1) * chunk]:
            acc = (acc << int(lengths[s])) | int(codewords[s])
            nbits += int(lengths[s])
        nw = (nbits + 31) // 32
        acc <<= nw * 32 - nbits
        for i in range(nw):
            words.append((acc >> (32 * (nw - 1 - i))) & 0xFFFFFFFF)
        offsets.append(offsets[-1] + nw)
    return np.array(words, np.uint32), np.array(offsets, np.uint32)


def decode_chunks(words, offsets, n: int, lengths, codewords, chunk: int = 1024) -> np.ndarray:
    """Inverse of encode_chunks: read each chunk's bits from its first word and match
    codewords (prefix-free, so the first match is the symbol)."""
    table = {(int(lengths[s]), int(codewords[s])): s for s in np.flatnonzero(np.asarray(lengths))}
    maxlen = int(np.max(lengths)) if np.any(lengths) else 0
    out = np.zeros(n, np.int64)
    w = np.asarray(words, dtype=np.uint64)
    for k in range((n + chunk - 1) // chunk):
        bitpos = 32 * int(offsets[k])
        for i in range(k * chunk, min(n, (k + 1) * chunk)):
            code, length = 0, 0
            while True:
                word = int(w[bitpos // 32])
                code = (code << 1) | ((word >> (31 - bitpos % 32)) & 1)
                bitpos += 1
                length += 1
                if (length, code) in table:
                    out[i] = table[(length, code)]
                    break
                if length > maxlen:
                    raise ValueError("invalid stream")
    return out
