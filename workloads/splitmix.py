"""SplitMix64 as a counter-based generator of synthetic inputs.

SplitMix64 is the generator of Steele, Lea and Flood ("Fast splittable
pseudorandom number generators", OOPSLA 2014), in the public-domain form
published by S. Vigna: the state advances by the odd constant GAMMA and each
output is the state passed through a 64-bit finaliser (xor-shift by 30, multiply,
xor-shift by 27, multiply, xor-shift by 31).

Everything here describes INPUTS (slot bytes, channel payloads, random draws
for the operation tables). None of it is part of the HiCR operations that are
being computed, so both the oracle and the GPU path may consume these values;
the CUDA kernels carry their own implementation of the same published
definition for the payloads they generate on the device.

All arithmetic is on numpy uint64 arrays, which wrap modulo 2**64.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)

_U64 = np.uint64


def _finalise(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def H(keys) -> np.ndarray:
    """First output of a SplitMix64 generator whose state is ``keys``.

    H(k) = finalise(k + GAMMA).  H is a bijection on 64-bit words.
    """
    k = np.asarray(keys, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _finalise(k + GAMMA)


def H_int(key: int) -> int:
    """Scalar H on a Python int (wrapped to 64 bits)."""
    return int(H(np.array([key & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0])


def sequence(state: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 started from ``state``.

    Output k is finalise(state + (k+1)*GAMMA): the generator is counter
    based, so any window can be produced without running the prefix.
    """
    ks = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & 0xFFFFFFFFFFFFFFFF) + ks * GAMMA
    return _finalise(z)


class Stream:
    """A named random stream: SplitMix64 started from H((seed << 32) | stream_id).

    ``uniform(count)`` returns doubles in [0, 1) built from the top 53 bits
    of consecutive outputs; each call continues where the previous stopped.
    """

    def __init__(self, seed: int, stream_id: int):
        self.state = H_int(((seed & 0xFFFFFFFF) << 32) | (stream_id & 0xFFFFFFFF))
        self.pos = 0

    def raw(self, count: int) -> np.ndarray:
        out = sequence(self.state, count, self.pos)
        self.pos += count
        return out

    def uniform(self, count: int) -> np.ndarray:
        return (self.raw(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers uniform on the closed range [lo, hi] (int64)."""
        u = self.uniform(count)
        span = float(hi - lo + 1)
        v = np.floor(u * span).astype(np.int64)
        return np.minimum(v, hi - lo) + lo

    def log_uniform(self, lo: int, hi: int, count: int) -> np.ndarray:
        """floor(exp(ln lo + U * (ln(hi+1) - ln lo))) clamped to [lo, hi] (int64)."""
        u = self.uniform(count)
        a = np.log(float(lo))
        b = np.log(float(hi) + 1.0)
        v = np.floor(np.exp(a + u * (b - a))).astype(np.int64)
        return np.clip(v, lo, hi)


# ---------------------------------------------------------------------------
# Slot fill: byte i of slot s under seed q is byte (i mod 8), little endian, of
# H(q * 2**56 + s * 2**40 + floor(i / 8)).
# ---------------------------------------------------------------------------

def fill_key_base(seed: int, slot: int) -> int:
    return ((seed & 0xFF) << 56) | ((slot & 0xFFFF) << 40)


def fill_words(seed: int, slot: int, first_word: int, n_words: int) -> np.ndarray:
    base = fill_key_base(seed, slot)
    keys = np.uint64(base) + np.arange(first_word, first_word + n_words, dtype=np.uint64)
    return H(keys)


def fill_bytes(seed: int, slot: int, start: int, length: int) -> np.ndarray:
    """Bytes [start, start+length) of the seeded fill of ``slot`` (uint8 array)."""
    if length <= 0:
        return np.zeros(0, dtype=np.uint8)
    w0 = start // 8
    w1 = (start + length + 7) // 8
    words = fill_words(seed, slot, w0, w1 - w0).astype("<u8")
    b = words.view(np.uint8)
    off = start - w0 * 8
    return b[off:off + length].copy()


def fill_byte_at(seed: int, slot: int, positions: np.ndarray) -> np.ndarray:
    """Fill byte at each position (vectorised, one hash per position)."""
    pos = np.asarray(positions, dtype=np.uint64)
    keys = np.uint64(fill_key_base(seed, slot)) + (pos >> np.uint64(3))
    w = H(keys)
    return ((w >> ((pos & np.uint64(7)) * np.uint64(8))) & np.uint64(0xFF)).astype(np.uint8)


# ---------------------------------------------------------------------------
# Channel payloads.
# ---------------------------------------------------------------------------

def spsc_token_words(channel: int, first_token: int, n_tokens: int, words_per_token: int = 8) -> np.ndarray:
    """Word w of token s on channel c is H(c * 2**40 + s * words_per_token + w)."""
    base = np.uint64((channel & 0xFFFFFF) << 40)
    idx = np.arange(first_token * words_per_token, (first_token + n_tokens) * words_per_token, dtype=np.uint64)
    return H(base + idx)


def mpsc_payload_key_base(producer: int, seq: int) -> int:
    return (1 << 63) | ((producer & 0x7FFFFF) << 40) | ((seq & 0xFFFFFF) << 16)


def mpsc_payload_bytes(producer: int, seq: int, n: int) -> np.ndarray:
    """Byte i of message (p, s) is byte (i mod 8) of H(2**63 + p*2**40 + s*2**16 + floor(i/8))."""
    if n <= 0:
        return np.zeros(0, dtype=np.uint8)
    nw = (n + 7) // 8
    keys = np.uint64(mpsc_payload_key_base(producer, seq)) + np.arange(nw, dtype=np.uint64)
    return H(keys).astype("<u8").view(np.uint8)[:n].copy()
