"""Digests the checkers compare -- TEST INFRASTRUCTURE ONLY.

The paper defines no digest; these are checking devices of this project.

word digest   D(w_0 .. w_{m-1}) = sum_j w_j * (2j + 1)   (mod 2**64)

Every multiplier is odd, hence invertible modulo 2**64, so changing any single
word changes D; the multiplier depends on the position, so moving a word
changes D too (unless the two words are equal modulo a power of two that the
position difference fixes, which random 64-bit words essentially never are).

byte digest   the word digest of the little-endian 8-byte words of a byte
              string, the last word zero-padded.

The sum is written as a plain loop over Python integers for small inputs
(``word_digest_loop``) and as a numpy reduction for large ones
(``word_digest``); the two are compared in the oracle's own tests.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1


def word_digest_loop(words, first_index: int = 0) -> int:
    d = 0
    for j, w in enumerate(words):
        d = (d + (int(w) & MASK) * (2 * (first_index + j) + 1)) & MASK
    return d


def word_digest(words: np.ndarray, first_index: int = 0) -> int:
    w = np.asarray(words, dtype=np.uint64)
    if len(w) == 0:
        return 0
    j = np.arange(first_index, first_index + len(w), dtype=np.uint64)
    with np.errstate(over="ignore"):
        terms = w * (np.uint64(2) * j + np.uint64(1))
    # uint64 sums wrap modulo 2**64
    return int(np.add.reduce(terms, dtype=np.uint64))


def bytes_to_words(b: np.ndarray) -> np.ndarray:
    b = np.asarray(b, dtype=np.uint8)
    pad = (-len(b)) % 8
    if pad:
        b = np.concatenate([b, np.zeros(pad, dtype=np.uint8)])
    return b.view("<u8").astype(np.uint64)


def byte_digest(b: np.ndarray) -> int:
    return word_digest(bytes_to_words(b))


def combine(digests) -> int:
    """Ordered combination of part digests: sum_k D_k * (2k + 1) mod 2**64."""
    return word_digest(np.array([int(x) & MASK for x in digests], dtype=np.uint64))


def block_digests(b: np.ndarray, block: int) -> np.ndarray:
    """Byte digest of each consecutive ``block``-byte piece of ``b`` (a
    multiple of 8; the last piece may be shorter), word positions counted
    from each piece's start."""
    b = np.asarray(b, dtype=np.uint8)
    if block % 8:
        raise ValueError("block must be a multiple of 8")
    nfull = len(b) // block
    out = np.zeros(nfull + (1 if len(b) % block else 0), dtype=np.uint64)
    if nfull:
        w = b[:nfull * block].view("<u8").reshape(nfull, block // 8)
        j = np.uint64(2) * np.arange(block // 8, dtype=np.uint64) + np.uint64(1)
        with np.errstate(over="ignore"):
            out[:nfull] = (w * j).sum(axis=1, dtype=np.uint64)
    if len(b) % block:
        out[nfull] = np.uint64(byte_digest(b[nfull * block:]))
    return out


def segment_digests(words: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """Word digest of each consecutive segment of ``words`` (segment k has
    ``counts[k]`` words; positions counted from the segment's start)."""
    w = np.asarray(words, dtype=np.uint64)
    counts = np.asarray(counts, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    j = (np.arange(len(w), dtype=np.int64) - np.repeat(starts, counts)).astype(np.uint64)
    with np.errstate(over="ignore"):
        terms = w * (np.uint64(2) * j + np.uint64(1))
    out = np.zeros(len(counts), dtype=np.uint64)
    nz = counts > 0
    if nz.any():
        out[nz] = np.add.reduceat(terms, starts[nz], dtype=np.uint64)
    return out
