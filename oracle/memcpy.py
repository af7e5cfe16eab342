"""Oracle for memory slots, memcpy, fence and message counters.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What it restates (HiCR paper):
  * Sec. 3.1.3 (Memory Management): a local memory slot is a segment
    (address, size) in a memory space; it is either allocated in a chosen
    space (malloc-like, fails when the space is unsupported or exhausted) or
    registered around an existing allocation.
  * Sec. 3.1.4 (Communication Management): memcpy(dst, dOff, src, sOff, n)
    copies n bytes between two slots; it is initiated when the manager
    supports the pair of memory spaces and rejected otherwise. Completion is
    not guaranteed at return; fence suspends until the expected number of
    incoming and outgoing transfers has completed.
  * Fig. 5 (broadcast example): allocate, memcpy, then fence() before use.

Readings where the paper is silent (each also listed in the design notes):
  * an op whose source and destination are the same slot with intersecting
    ranges is rejected (OVERLAP) -- C memcpy leaves it undefined;
  * ops between two fences are unordered; a destination range that touches
    another op's source or destination range in the same epoch is a caller
    hazard (HAZARD in checked mode);
  * a zero-size op is accepted, moves nothing and counts as one message;
  * counters count ops (messages), not bytes, are 64-bit and never reset;
  * every slot carries a tag; an op belongs to the tags of both its slots and
    fence(tag) waits for every earlier op of that tag;
  * only the pair (device HBM, device HBM) is supported by default.

The executable definition is deliberately plain: validate, then for every
accepted op, in issue order, ``dst[dOff:dOff+n] = src[sOff:sOff+n]`` (a numpy
slice copy, i.e. byte i of the destination takes byte i of the source), then
bump sent[src], recv[dst] and the per-tag counts.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Status codes of the C ABI, restated independently here.
OK = 0
ERR_INVALID = -1
ERR_UNSUPPORTED = -2
ERR_BOUNDS = -3
ERR_OVERLAP = -4
ERR_HAZARD = -5
ERR_NOMEM = -6
ERR_FULL = -7
ERR_EMPTY = -8
ERR_TOO_LARGE = -9
ERR_TIMEOUT = -10
ERR_BUSY = -11
ERR_DEVICE = -12

SPACE_HBM = 0
SPACE_HOST = 1

U64_MAX = (1 << 64) - 1


@dataclass
class Slot:
    space: int
    data: np.ndarray  # uint8, the slot's bytes
    tag: int = 0
    live: bool = True


def _range_ok(off: int, n: int, size: int) -> bool:
    """off + n <= size without overflowing 64 bits."""
    if off < 0 or n < 0 or off > U64_MAX or n > U64_MAX:
        return False
    return off <= size and n <= size - off


def _intersects(a: int, b: int, n: int, m: int) -> bool:
    """Do [a, a+n) and [b, b+m) share a byte?"""
    return n > 0 and m > 0 and a < b + m and b < a + n


class CommManager:
    """Single instance: slot table, memcpy, fence and counters."""

    def __init__(self, supported_pairs=((SPACE_HBM, SPACE_HBM),)):
        self.slots: dict[int, Slot] = {}
        self.sent: dict[int, int] = {}
        self.recv: dict[int, int] = {}
        self.tag_ops: dict[int, int] = {}
        self.supported = set(supported_pairs)
        self._next = 0

    # -- Memory manager (Sec. 3.1.3) -------------------------------------
    def register(self, space: int, data: np.ndarray, tag: int = 0) -> int:
        sid = self._next
        self._next += 1
        self.slots[sid] = Slot(space, data, tag)
        self.sent[sid] = 0
        self.recv[sid] = 0
        return sid

    def deregister(self, sid: int) -> int:
        s = self.slots.get(sid)
        if s is None or not s.live:
            return ERR_INVALID
        s.live = False
        return OK

    # -- Communication manager (Sec. 3.1.4) ------------------------------
    def validate(self, dst: int, doff: int, src: int, soff: int, n: int) -> int:
        d = self.slots.get(dst)
        s = self.slots.get(src)
        if d is None or s is None or not d.live or not s.live:
            return ERR_INVALID
        if (d.space, s.space) not in self.supported:
            return ERR_UNSUPPORTED
        if not _range_ok(soff, n, len(s.data)) or not _range_ok(doff, n, len(d.data)):
            return ERR_BOUNDS
        if dst == src and _intersects(doff, soff, n, n):
            return ERR_OVERLAP
        return OK

    def _apply(self, dst: int, doff: int, src: int, soff: int, n: int) -> None:
        d = self.slots[dst]
        s = self.slots[src]
        if n:
            d.data[doff:doff + n] = s.data[soff:soff + n]
        self.sent[src] += 1
        self.recv[dst] += 1
        self.tag_ops[s.tag] = self.tag_ops.get(s.tag, 0) + 1
        if d.tag != s.tag:
            self.tag_ops[d.tag] = self.tag_ops.get(d.tag, 0) + 1

    def memcpy(self, dst: int, doff: int, src: int, soff: int, n: int) -> int:
        st = self.validate(dst, doff, src, soff, n)
        if st == OK:
            self._apply(dst, doff, src, soff, n)
        return st

    def memcpy_batch(self, ops: np.ndarray, checked: bool = False):
        """All-or-nothing: returns (status, first_bad_index or None)."""
        for i in range(len(ops)):
            o = ops[i]
            st = self.validate(int(o["dst"]), int(o["dst_off"]), int(o["src"]), int(o["src_off"]), int(o["n"]))
            if st != OK:
                return st, i
        if checked:
            bad = first_hazard(ops)
            if bad is not None:
                return ERR_HAZARD, bad
        for i in range(len(ops)):
            o = ops[i]
            self._apply(int(o["dst"]), int(o["dst_off"]), int(o["src"]), int(o["src_off"]), int(o["n"]))
        return OK, None

    def fence(self, tag: int = 0) -> int:
        # Every accepted op already completed (the oracle is synchronous).
        return OK

    def fence_slot(self, sid: int, expect_sent: int, expect_recv: int) -> int:
        """Wait for the expected number of outgoing / incoming transfers: in a
        synchronous model the wait either is already satisfied or never ends."""
        if sid not in self.slots:
            return ERR_INVALID
        if self.sent[sid] >= expect_sent and self.recv[sid] >= expect_recv:
            return OK
        return ERR_TIMEOUT

    def counters(self, sid: int):
        return self.sent[sid], self.recv[sid]


def first_hazard(ops: np.ndarray):
    """Index of the first op whose destination touches an earlier op's source
    or destination range on the same slot (or whose source range is touched
    by an earlier destination), brute force over all pairs; None if none."""
    for j in range(len(ops)):
        b = ops[j]
        for i in range(j):
            a = ops[i]
            an, bn = int(a["n"]), int(b["n"])
            if int(a["dst"]) == int(b["dst"]) and _intersects(int(a["dst_off"]), int(b["dst_off"]), an, bn):
                return j
            if int(a["dst"]) == int(b["src"]) and _intersects(int(a["dst_off"]), int(b["src_off"]), an, bn):
                return j
            if int(b["dst"]) == int(a["src"]) and _intersects(int(b["dst_off"]), int(a["src_off"]), bn, an):
                return j
    return None


# ---------------------------------------------------------------------------
# Full-size helpers: expected bytes one position at a time.
# ---------------------------------------------------------------------------

def expected_bytes_at(ops: np.ndarray, epochs, slot: int, positions: np.ndarray,
                      initial_byte, upto_epoch: int | None = None) -> np.ndarray:
    """Expected content of ``slot`` at ``positions`` after the epochs
    ``[0, upto_epoch)`` have been applied in order.

    Within one epoch destinations are disjoint, so at most one op of that
    epoch covers a position; across epochs the later one wins. The value of
    a covered position is the value of the source position *before* that
    epoch (computed recursively), an uncovered one keeps ``initial_byte``
    (a callable (slot, positions) -> uint8 array).
    """
    positions = np.asarray(positions, dtype=np.int64)
    if upto_epoch is None:
        upto_epoch = len(epochs)
    out = initial_byte(slot, positions) if upto_epoch == 0 else None
    if upto_epoch == 0:
        return out
    # Which op of the last epoch (if any) covers each position?
    a, b = epochs[upto_epoch - 1]
    ep = ops[a:b]
    sel = np.nonzero(ep["dst"] == slot)[0]
    earlier = expected_bytes_at(ops, epochs, slot, positions, initial_byte, upto_epoch - 1)
    if len(sel) == 0:
        return earlier
    starts = ep["dst_off"][sel].astype(np.int64)
    order = np.argsort(starts, kind="stable")
    sel = sel[order]
    starts = starts[order]
    ends = starts + ep["n"][sel].astype(np.int64)
    k = np.searchsorted(starts, positions, side="right") - 1
    valid = k >= 0
    kk = np.where(valid, k, 0)
    covered = valid & (positions < ends[kk])
    result = earlier.copy()
    if covered.any():
        idx = sel[kk[covered]]
        src_slots = ep["src"][idx].astype(np.int64)
        src_pos = ep["src_off"][idx].astype(np.int64) + (positions[covered] - starts[kk[covered]])
        vals = np.empty(len(idx), dtype=np.uint8)
        for s in np.unique(src_slots):
            m = src_slots == s
            vals[m] = expected_bytes_at(ops, epochs, int(s), src_pos[m], initial_byte, upto_epoch - 1)
        result[covered] = vals
    return result


def final_slot_bytes(ops: np.ndarray, slot: int, initial: np.ndarray, source_bytes) -> np.ndarray:
    """Content of ``slot`` after every op of ``ops`` in issue order, for a
    table in which no slot is both read and written (the batched workload's
    read-only source half): start from ``initial`` (the slot's bytes before
    the table) and, for each op whose destination is ``slot``, in issue
    order, set bytes [dst_off, dst_off + n) to ``source_bytes(src, src_off,
    n)``. This is CommManager.memcpy_batch seen from one destination slot;
    it is exact here because no op reads a byte that another op writes, so
    every source byte keeps its initial value."""
    if np.intersect1d(ops["dst"], ops["src"]).size:
        raise ValueError("a slot is both read and written")
    out = np.array(initial, dtype=np.uint8, copy=True)
    for o in ops[ops["dst"] == slot]:  # a boolean selection keeps issue order
        n = int(o["n"])
        if n:
            d = int(o["dst_off"])
            out[d:d + n] = source_bytes(int(o["src"]), int(o["src_off"]), n)
    return out


def counters_from_ops(ops: np.ndarray, n_slots: int):
    """sent[s] = #ops reading slot s, recv[s] = #ops writing slot s."""
    sent = np.bincount(ops["src"].astype(np.int64), minlength=n_slots).astype(np.uint64)
    recv = np.bincount(ops["dst"].astype(np.int64), minlength=n_slots).astype(np.uint64)
    return sent, recv
