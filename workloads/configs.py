"""Seeded synthetic workloads for the five measured configurations.

Each builder returns plain numpy arrays describing INPUTS only: slot sizes and
tags, operation tables (destination slot, source slot, destination offset,
source offset, size), epoch boundaries, channel parameters and request traces.
Slot contents are the SplitMix64 fill of ``workloads.splitmix``.

Operation-table record layout (32 bytes, little endian) -- the same layout
the C ABI's ``hicr_op_t`` uses:
    u32 dst, u32 src, u64 dst_off, u64 src_off, u64 n
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .splitmix import Stream

KiB = 1024
MiB = 1024 * KiB
GiB = 1024 * MiB

OP_DTYPE = np.dtype([("dst", "<u4"), ("src", "<u4"), ("dst_off", "<u8"),
                     ("src_off", "<u8"), ("n", "<u8")])
assert OP_DTYPE.itemsize == 32


def make_ops(dst, src, dst_off, src_off, n) -> np.ndarray:
    ops = np.zeros(len(n), dtype=OP_DTYPE)
    ops["dst"] = dst
    ops["src"] = src
    ops["dst_off"] = dst_off
    ops["src_off"] = src_off
    ops["n"] = n
    return ops


@dataclass
class MemcpyWorkload:
    """Slots plus an operation table cut into fence epochs.

    ``epochs`` holds (first_op, end_op) pairs; ops inside one epoch have
    pairwise disjoint destination ranges and never write a source range.
    """
    name: str
    seed: int
    slot_sizes: np.ndarray          # uint64 per slot
    slot_tags: np.ndarray           # uint32 per slot
    ops: np.ndarray                 # OP_DTYPE
    epochs: list = field(default_factory=list)
    src_slots: np.ndarray = None    # slots only ever read
    dst_slots: np.ndarray = None    # slots written

    @property
    def total_bytes(self) -> int:
        return int(self.ops["n"].sum())


# ---------------------------------------------------------------------------
# Config 1 -- two 64 MiB slots, 1,024 ops of U[1, 65536] bytes, one fence.
# ---------------------------------------------------------------------------

def tiny(seed: int = 0, slot_bytes: int = 64 * MiB, n_ops: int = 1024,
         max_n: int = 64 * KiB) -> MemcpyWorkload:
    """Slot 0 is the source, slot 1 the destination, both tag 0.

    Source offsets are uniform over the valid range. Destinations are laid
    out without overlap by a random composition: with S the summed op size
    and F = slot_bytes - S the free space, k sorted uniform cut points in
    [0, F] give the gaps and the ops are placed in a random order.
    """
    s_n = Stream(seed, 101)
    s_soff = Stream(seed, 102)
    s_cut = Stream(seed, 103)
    s_perm = Stream(seed, 104)
    n = s_n.integers(1, max_n, n_ops)
    S = int(n.sum())
    if S > slot_bytes:
        raise ValueError("ops do not fit the destination slot")
    soff = np.floor(s_soff.uniform(n_ops) * (slot_bytes - n + 1).astype(np.float64)).astype(np.int64)
    soff = np.minimum(soff, slot_bytes - n)
    F = slot_bytes - S
    cuts = np.sort(s_cut.integers(0, F, n_ops))
    order = np.argsort(s_perm.uniform(n_ops), kind="stable")
    placed = n[order]
    prefix = np.concatenate([[0], np.cumsum(placed)[:-1]])
    doff = np.empty(n_ops, dtype=np.int64)
    doff[order] = cuts + prefix
    ops = make_ops(1, 0, doff, soff, n)
    return MemcpyWorkload("tiny", seed, np.array([slot_bytes, slot_bytes], dtype=np.uint64),
                          np.zeros(2, dtype=np.uint32), ops, [(0, n_ops)],
                          np.array([0]), np.array([1]))


# ---------------------------------------------------------------------------
# Config 2 -- 256 slots totalling 16 GiB, 100,000 ops log-uniform 16 B - 4 MiB.
# ---------------------------------------------------------------------------

def slot_sizes_log_uniform(seed: int, n_slots: int, total: int, lo: int, hi: int,
                           granule: int = 4 * KiB) -> np.ndarray:
    """Draw log-uniform sizes in [lo, hi], scale to ``total``, clamp, round down
    to ``granule`` and hand the remainder to the smallest slots (each kept <= hi)."""
    st = Stream(seed, 201)
    u = st.uniform(n_slots)
    raw = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    sizes = raw * (total / raw.sum())
    sizes = np.clip(sizes, lo, hi)
    sizes = (np.floor(sizes / granule) * granule).astype(np.int64)
    rem = total - int(sizes.sum())
    for j in np.argsort(sizes, kind="stable"):
        if rem <= 0:
            break
        room = hi - int(sizes[j])
        add = min(rem, room)
        add -= add % granule
        sizes[j] += add
        rem -= add
    if rem < 0:  # clamping can push above the total; trim from the largest
        for j in np.argsort(-sizes, kind="stable"):
            if rem >= 0:
                break
            cut = min(-rem, int(sizes[j]) - lo)
            cut -= cut % granule
            sizes[j] -= cut
            rem += cut
    return sizes.astype(np.uint64)


def batched(seed: int = 0, n_slots: int = 256, total_bytes: int = 16 * GiB,
            slot_lo: int = 1 * MiB, slot_hi: int = 256 * MiB, n_ops: int = 100_000,
            n_lo: int = 16, n_hi: int = 4 * MiB, unaligned_frac: float = 0.10,
            max_gap: int = 1024, name: str = "batched") -> MemcpyWorkload:
    """Config 2 and its scaled-down variants.

    Even slots are sources (never written), odd slots destinations. For each
    op in generation order: size log-uniform in [n_lo, n_hi]; with probability
    ``unaligned_frac`` both offsets get independent residues 1..15 mod 16,
    otherwise both are multiples of 16; the source slot is uniform among
    source slots that can hold the op and the source offset uniform over the
    valid range. Destinations fill each epoch without overlap: every
    destination slot keeps a cursor, the op goes to a uniformly chosen
    destination slot with room, after a random 16-byte-granular gap. When no
    slot has room the epoch ends and all cursors reset (a fence separates
    epochs, so later epochs may overwrite earlier ones).
    """
    sizes = slot_sizes_log_uniform(seed, n_slots, total_bytes, slot_lo, slot_hi)
    tags = np.zeros(n_slots, dtype=np.uint32)
    src_slots = np.arange(0, n_slots, 2)
    dst_slots = np.arange(1, n_slots, 2)
    isz = sizes.astype(np.int64)

    n = Stream(seed, 202).log_uniform(n_lo, n_hi, n_ops)
    u_mis = Stream(seed, 203).uniform(n_ops)
    u_src = Stream(seed, 204).uniform(n_ops)
    u_soff = Stream(seed, 205).uniform(n_ops)
    r_s = Stream(seed, 206).integers(1, 15, n_ops)
    r_d = Stream(seed, 207).integers(1, 15, n_ops)
    u_dst = Stream(seed, 208).uniform(n_ops)
    gaps = Stream(seed, 209).integers(0, max_gap // 16, n_ops) * 16

    src_sizes = isz[src_slots]
    order_src = np.argsort(src_sizes, kind="stable")
    sorted_src_sizes = src_sizes[order_src]
    dst_sizes = isz[dst_slots]

    out_dst = np.empty(n_ops, dtype=np.int64)
    out_src = np.empty(n_ops, dtype=np.int64)
    out_doff = np.empty(n_ops, dtype=np.int64)
    out_soff = np.empty(n_ops, dtype=np.int64)
    epochs = []
    epoch_start = 0
    cursor = np.zeros(len(dst_slots), dtype=np.int64)
    for i in range(n_ops):
        ni = int(n[i])
        mis = u_mis[i] < unaligned_frac
        rs = int(r_s[i]) if mis else 0
        rd = int(r_d[i]) if mis else 0
        need = ni + 16
        # source slot: uniform among those that can hold the op
        first_ok = int(np.searchsorted(sorted_src_sizes, need, side="left"))
        if first_ok >= len(sorted_src_sizes):
            raise ValueError("an op is larger than every source slot")
        cand = order_src[first_ok:]
        j = int(cand[min(int(u_src[i] * len(cand)), len(cand) - 1)])
        s_slot = int(src_slots[j])
        span = (int(isz[s_slot]) - ni - rs) // 16
        soff = 16 * min(int(u_soff[i] * (span + 1)), span) + rs
        # destination slot with room in this epoch
        start = ((cursor + 15) // 16) * 16 + int(gaps[i])
        room = np.nonzero(start + rd + ni <= dst_sizes)[0]
        if len(room) == 0:
            epochs.append((epoch_start, i))
            epoch_start = i
            cursor[:] = 0
            start = np.full_like(cursor, int(gaps[i]))
            room = np.nonzero(start + rd + ni <= dst_sizes)[0]
            if len(room) == 0:
                raise ValueError("an op is larger than every destination slot")
        k = int(room[min(int(u_dst[i] * len(room)), len(room) - 1)])
        doff = int(start[k]) + rd
        cursor[k] = doff + ni
        out_dst[i] = dst_slots[k]
        out_src[i] = s_slot
        out_doff[i] = doff
        out_soff[i] = soff
    epochs.append((epoch_start, n_ops))
    ops = make_ops(out_dst, out_src, out_doff, out_soff, n)
    return MemcpyWorkload(name, seed, sizes, tags, ops, epochs, src_slots, dst_slots)


def batched_large(seed: int = 0, **kw) -> MemcpyWorkload:
    """The large-segment sub-case of config 2: sizes log-uniform 1-4 MiB, all aligned."""
    kw.setdefault("n_lo", 1 * MiB)
    kw.setdefault("n_hi", 4 * MiB)
    kw.setdefault("unaligned_frac", 0.0)
    kw.setdefault("name", "batched_large")
    return batched(seed, **kw)


def batched_small(seed: int = 0) -> MemcpyWorkload:
    """Scaled-down config 2 for parity tests (32 slots, 256 MiB, 3,000 ops up to 1 MiB)."""
    return batched(seed, n_slots=32, total_bytes=256 * MiB, slot_lo=256 * KiB,
                   slot_hi=32 * MiB, n_ops=3000, n_lo=16, n_hi=1 * MiB, name="batched_small")


# ---------------------------------------------------------------------------
# Config 3 -- SPSC channels (parameters only; payload words from splitmix).
# ---------------------------------------------------------------------------

@dataclass
class SpscWorkload:
    n_channels: int = 64
    capacity: int = 4096
    token_bytes: int = 64
    tokens_per_channel: int = 10_000_000


# ---------------------------------------------------------------------------
# Config 4 -- MPSC channels.
# ---------------------------------------------------------------------------

@dataclass
class MpscWorkload:
    n_producers: int
    n_consumers: int
    msgs_per_producer: int
    ring_bytes: int
    max_msgs: int
    sizes: np.ndarray  # int64 [n_producers, msgs_per_producer]

    def consumer_of(self, p: int) -> int:
        return p % self.n_consumers

    @property
    def total_bytes(self) -> int:
        return int(self.sizes.sum())


def mpsc(seed: int = 0, n_producers: int = 1024, n_consumers: int = 16,
         msgs_per_producer: int = 1024, ring_bytes: int = 1 * GiB,
         max_msgs: int = 65536, lo: int = 8, hi: int = 256 * KiB) -> MpscWorkload:
    """Producer p feeds consumer p mod n_consumers; message (p, s) has a
    log-uniform size drawn from stream 401 at index p*msgs_per_producer + s."""
    sizes = Stream(seed, 401).log_uniform(lo, hi, n_producers * msgs_per_producer)
    return MpscWorkload(n_producers, n_consumers, msgs_per_producer, ring_bytes, max_msgs,
                        sizes.reshape(n_producers, msgs_per_producer))


# ---------------------------------------------------------------------------
# Config 5 -- serving trace.
# ---------------------------------------------------------------------------

@dataclass
class ServeTrace:
    arrival_ns: np.ndarray   # int64, sorted
    kind: np.ndarray         # 0 = memcpy batch, 1 = MPSC burst
    template: np.ndarray     # template index within its kind
    rate: float
    duration_s: float


def serve_trace(seed: int = 0, rate: float = 20000.0, duration_s: float = 60.0,
                memcpy_frac: float = 0.7, n_templates: int = 1024) -> ServeTrace:
    """Poisson arrivals (exponential gaps of mean 1/rate, from stream 501);
    each request is a memcpy batch with probability memcpy_frac, else an MPSC
    burst (stream 502), and names a template of its kind uniformly (503)."""
    expected = int(rate * duration_s * 1.1) + 64
    gaps = -np.log1p(-Stream(seed, 501).uniform(expected)) / rate
    t = np.cumsum(gaps)
    m = int(np.searchsorted(t, duration_s, side="left"))
    t = t[:m]
    kind = (Stream(seed, 502).uniform(m) >= memcpy_frac).astype(np.int32)
    template = Stream(seed, 503).integers(0, n_templates - 1, m)
    return ServeTrace((t * 1e9).astype(np.int64), kind, template.astype(np.int64), rate, duration_s)


@dataclass
class ServeTemplates:
    """memcpy templates: ops whose dst_off is relative to the request's own
    region (packed, 16-byte aligned starts), src = source slot index of the
    source workload; MPSC burst templates: message sizes. Message m of burst
    template t carries the MPSC payload of (producer t, seq m)."""
    op_start: np.ndarray      # int64 [n_templates + 1] into ops
    ops: np.ndarray           # OP_DTYPE; dst = 0
    region_bytes: np.ndarray  # int64 per memcpy template
    msg_start: np.ndarray     # int64 [n_templates + 1] into msg_sizes
    msg_sizes: np.ndarray     # int64


def serve_templates(seed: int, src: MemcpyWorkload, n_templates: int = 1024, max_ops: int = 4096,
                    max_msgs: int = 512, n_lo: int = 16, n_hi: int = 4 * MiB, msg_lo: int = 8,
                    msg_hi: int = 256 * KiB) -> ServeTemplates:
    """Op counts log-uniform [1, max_ops] (stream 510), sizes log-uniform
    [n_lo, n_hi] (511), source slot uniform among the source slots that hold
    the op (512), 16-byte aligned source offset uniform (513); message counts
    log-uniform [1, max_msgs] (514), sizes log-uniform [msg_lo, msg_hi] (515)."""
    counts = Stream(seed, 510).log_uniform(1, max_ops, n_templates)
    total = int(counts.sum())
    n = Stream(seed, 511).log_uniform(n_lo, n_hi, total)
    u_src = Stream(seed, 512).uniform(total)
    u_soff = Stream(seed, 513).uniform(total)
    isz = src.slot_sizes.astype(np.int64)
    srcs = np.asarray(src.src_slots)
    order = np.argsort(isz[srcs], kind="stable")
    sorted_sizes = isz[srcs][order]
    first = np.searchsorted(sorted_sizes, n + 16, side="left")
    if (first >= len(srcs)).any():
        raise ValueError("an op is larger than every source slot")
    pick_idx = first + np.minimum((u_src * (len(srcs) - first)).astype(np.int64), len(srcs) - first - 1)
    pick = srcs[order[pick_idx]]
    span = (isz[pick] - n) // 16
    soff = 16 * np.minimum((u_soff * (span + 1)).astype(np.int64), span)
    op_start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    sz16 = ((n + 15) // 16) * 16
    csum = np.concatenate([[0], np.cumsum(sz16)])
    doff = csum[:-1] - np.repeat(csum[op_start[:-1]], counts)
    region = csum[op_start[1:]] - csum[op_start[:-1]]
    ops = make_ops(0, pick, doff, soff, n)
    mcounts = Stream(seed, 514).log_uniform(1, max_msgs, n_templates)
    msg_start = np.concatenate([[0], np.cumsum(mcounts)]).astype(np.int64)
    msizes = Stream(seed, 515).log_uniform(msg_lo, msg_hi, int(mcounts.sum()))
    return ServeTemplates(op_start, ops, region.astype(np.int64), msg_start, msizes)
