"""Full-size oracle expectations, computed on the host's cores.

The configurations at full size hold 16 GiB of slots (the batched memcpy) or
26 GB of channel payloads (the MPSC streams); the oracle's plain numpy
definitions are applied slot by slot or producer by producer in a pool of
worker processes started with ``spawn`` (no CUDA state is inherited). Every
function here only calls ``oracle`` and the seeded input generators of
``workloads``; nothing reads a GPU result.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import digest as od
from oracle import memcpy as om
from workloads import configs, splitmix

BLOCK = 1 << 20

_W = None  # the worker's copy of the workload


def _init_batched(maker: str, seed: int):
    global _W
    _W = (getattr(configs, maker)(seed), seed)


def _slot_expectation(args):
    """(block digests, {block index: bytes}) of slot s after the whole table."""
    s, full_blocks = args
    w, seed = _W
    size = int(w.slot_sizes[s])
    data = splitmix.fill_bytes(seed, s, 0, size)
    if s in set(np.asarray(w.dst_slots).tolist()):
        data = om.final_slot_bytes(w.ops, s, data, lambda src, off, n: splitmix.fill_bytes(seed, src, off, n))
    dig = od.block_digests(data, BLOCK)
    return dig, {b: data[b * BLOCK:(b + 1) * BLOCK].copy() for b in full_blocks}


def pool_size() -> int:
    return max(1, min(16, (os.cpu_count() or 2) - 1))


def batched_expectations(maker: str, seed: int, full_blocks: dict):
    """For every slot of configs.<maker>(seed): the digest of each 1 MiB
    block of its final content, and the full bytes of the blocks listed in
    full_blocks[slot]."""
    w = getattr(configs, maker)(seed)
    jobs = [(s, sorted(full_blocks.get(s, ()))) for s in range(len(w.slot_sizes))]
    ctx = mp.get_context("spawn")
    with ctx.Pool(pool_size(), initializer=_init_batched, initargs=(maker, seed)) as pool:
        return pool.map(_slot_expectation, jobs, chunksize=1)


def producer_message_digests(p: int, sizes: np.ndarray) -> np.ndarray:
    """Byte digest of every message (p, s) of the MPSC payload rule, for the
    sizes of producer p's messages (index s), computed for all of them at
    once: the words of message s are H(2^63 + p 2^40 + s 2^16 + j), the bytes
    past its size zeroed in its last word."""
    sizes = np.asarray(sizes, dtype=np.int64)
    nw = (sizes + 7) // 8
    starts = np.concatenate([[0], np.cumsum(nw)[:-1]]).astype(np.int64)
    s_idx = np.repeat(np.arange(len(sizes), dtype=np.uint64), nw)
    j = (np.arange(int(nw.sum()), dtype=np.int64) - np.repeat(starts, nw)).astype(np.uint64)
    base = np.uint64(splitmix.mpsc_payload_key_base(p, 0))
    w = splitmix.H(base + (s_idx << np.uint64(16)) + j)
    rem = sizes % 8
    last = starts + nw - 1
    cut = rem > 0
    w[last[cut]] &= (np.uint64(1) << (np.uint64(8) * rem[cut].astype(np.uint64))) - np.uint64(1)
    return od.segment_digests(w, nw)


def _producer_job(args):
    p, sizes = args
    return producer_message_digests(p, sizes)


def mpsc_expectations(sizes: np.ndarray) -> np.ndarray:
    """[P, M] oracle digests of every message of an MPSC workload."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(pool_size()) as pool:
        rows = pool.map(_producer_job, [(p, sizes[p]) for p in range(sizes.shape[0])], chunksize=8)
    return np.stack(rows)


def spsc_channel_digest(args) -> int:
    """Word digest of the whole token stream of one SPSC channel: word w of
    token s on channel c is H(c 2^40 + s wpt + w), in token order."""
    c, tokens, wpt = args
    d = 0
    step = 1 << 20
    for t0 in range(0, tokens, step):
        n = min(step, tokens - t0)
        d = (d + od.word_digest(splitmix.spsc_token_words(c, t0, n, wpt), t0 * wpt)) % (1 << 64)
    return d


def spsc_expectations(n_channels: int, tokens: int, wpt: int = 8):
    ctx = mp.get_context("spawn")
    with ctx.Pool(pool_size()) as pool:
        return pool.map(spsc_channel_digest, [(c, tokens, wpt) for c in range(n_channels)], chunksize=1)


def burst_template_digest(args) -> int:
    """Result digest of a burst request of template t (the serving engine's
    definition): sum over messages m of (2m + 1) * byte digest of message m,
    whose bytes are the MPSC payload of (producer t, seq m)."""
    t, sizes = args
    return od.combine(producer_message_digests(t, sizes))


def burst_expectations(tmpl) -> list:
    """Oracle result digests of every burst template of `tmpl`."""
    jobs = [(t, tmpl.msg_sizes[tmpl.msg_start[t]:tmpl.msg_start[t + 1]]) for t in range(len(tmpl.msg_start) - 1)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(pool_size()) as pool:
        return pool.map(burst_template_digest, jobs, chunksize=8)


def memcpy_template_digest(seed: int, tmpl, t: int) -> int:
    """Result digest of a memcpy request of template t: sum over its ops k of
    (2k + 1) * byte digest of op k's destination bytes, which the memcpy
    oracle makes equal to the seeded source bytes the op reads (the template's
    destinations are disjoint offsets of the request's own region)."""
    a, b = int(tmpl.op_start[t]), int(tmpl.op_start[t + 1])
    return od.combine([od.byte_digest(splitmix.fill_bytes(seed, int(o["src"]), int(o["src_off"]), int(o["n"])))
                       for o in tmpl.ops[a:b]])
