"""Oracle for the Channels frontend -- TEST INFRASTRUCTURE ONLY.

HiCR paper Sec. 4.3 (Built-in Frontends, Channels): a channel is a
pre-allocated circular buffer at the consumer. The producer knows where the
next message goes and may push while the buffer is not full; once full it may
not push until the consumer reports a message consumed. SPSC channels have one
producer; MPSC channels have several, and in "locking" mode a collective
exclusive access keeps the shared buffer from overflowing.

Readings where the paper is silent:
  * host push/pop are non-blocking: a push that does not fit returns FULL, a
    pop of more than is buffered returns EMPTY; a multi-token SPSC push is
    all-or-nothing;
  * peek(k) reports the k-th oldest unpopped message (ring offset, size,
    producer, sequence number) without changing state; k >= depth is EMPTY;
  * head/tail are 64-bit monotonic counters; the slot of token t is t mod C;
  * MPSC (locking mode): the exclusive access is modelled as one atomic
    reservation of a ticket (message index) plus a contiguous byte range.
    Each reservation is rounded up to 16 bytes; a message that would cross
    the end of the ring skips to its start and the skipped bytes count as
    reserved (no split messages). A reservation succeeds only if bytes
    reserved and not yet freed stay <= ring_bytes and messages in flight stay
    <= max_msgs. A message larger than the ring is TOO_LARGE. The consumer
    frees messages in ticket (commit) order; freeing a message frees every
    byte up to its end.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .memcpy import OK, ERR_FULL, ERR_EMPTY, ERR_TOO_LARGE, ERR_INVALID

ALIGN = 16


def round_up(n: int, a: int = ALIGN) -> int:
    return (n + a - 1) // a * a


class SpscOracle:
    def __init__(self, token_bytes: int, capacity: int):
        self.token_bytes = token_bytes
        self.capacity = capacity
        self.ring = np.zeros(token_bytes * capacity, dtype=np.uint8)
        self.head = 0   # tokens pushed
        self.tail = 0   # tokens popped

    def depth(self):
        d = self.head - self.tail
        return d, d * self.token_bytes

    def push(self, data: np.ndarray) -> int:
        data = np.asarray(data, dtype=np.uint8)
        if len(data) % self.token_bytes:
            return ERR_INVALID
        k = len(data) // self.token_bytes
        if self.head - self.tail + k > self.capacity:
            return ERR_FULL
        for j in range(k):
            pos = (self.head + j) % self.capacity
            self.ring[pos * self.token_bytes:(pos + 1) * self.token_bytes] = \
                data[j * self.token_bytes:(j + 1) * self.token_bytes]
        self.head += k
        return OK

    def peek(self, k: int):
        if k >= self.head - self.tail:
            return ERR_EMPTY, None
        t = self.tail + k
        return OK, ((t % self.capacity) * self.token_bytes, self.token_bytes, 0, t)

    def token(self, k: int) -> np.ndarray:
        st, info = self.peek(k)
        assert st == OK
        return self.ring[info[0]:info[0] + self.token_bytes].copy()

    def pop(self, count: int) -> int:
        if count > self.head - self.tail:
            return ERR_EMPTY
        self.tail += count
        return OK


class MpscOracle:
    """Locking-mode MPSC channel over one shared ring."""

    def __init__(self, n_producers: int, ring_bytes: int, max_msgs: int):
        self.n_producers = n_producers
        self.R = ring_bytes
        self.max_msgs = max_msgs
        self.ring = np.zeros(ring_bytes, dtype=np.uint8)
        self.reserved = 0          # absolute bytes reserved (incl. skipped)
        self.freed = 0             # absolute bytes freed
        self.msg_head = 0          # tickets handed out
        self.msg_tail = 0          # messages freed
        self.meta = deque()        # (start_abs, size, producer, seq, end_abs)
        self.seq = [0] * n_producers
        self.max_inflight = 0

    def depth(self):
        return self.msg_head - self.msg_tail, self.reserved - self.freed

    def placement(self, n: int):
        """(start_abs, end_abs) a reservation of n bytes would take now."""
        r = round_up(n)
        pos = self.reserved % self.R
        pad = self.R - pos if pos + r > self.R else 0
        start = self.reserved + pad
        return start, start + r

    def push(self, producer: int, payload: np.ndarray) -> int:
        payload = np.asarray(payload, dtype=np.uint8)
        n = len(payload)
        if producer < 0 or producer >= self.n_producers:
            return ERR_INVALID
        if round_up(n) > self.R:
            return ERR_TOO_LARGE
        start, end = self.placement(n)
        if end - self.freed > self.R or self.msg_head - self.msg_tail + 1 > self.max_msgs:
            return ERR_FULL
        off = start % self.R
        self.ring[off:off + n] = payload
        self.meta.append((start, n, producer, self.seq[producer], end))
        self.seq[producer] += 1
        self.reserved = end
        self.msg_head += 1
        self.max_inflight = max(self.max_inflight, end - self.freed)
        return OK

    def peek(self, k: int):
        if k >= self.msg_head - self.msg_tail:
            return ERR_EMPTY, None
        start, n, p, s, _ = self.meta[k]
        return OK, (start % self.R, n, p, s)

    def payload(self, k: int) -> np.ndarray:
        st, info = self.peek(k)
        assert st == OK
        return self.ring[info[0]:info[0] + info[1]].copy()

    def pop(self, count: int) -> int:
        if count > self.msg_head - self.msg_tail:
            return ERR_EMPTY
        for _ in range(count):
            _, _, _, _, end = self.meta.popleft()
            self.freed = end
            self.msg_tail += 1
        return OK


def replay_offsets(sizes, ring_bytes: int):
    """Ring offsets the reservation rule gives to messages reserved in the
    order given (ticket order), independent of when they are freed."""
    reserved = 0
    out = []
    for n in sizes:
        r = round_up(int(n))
        pos = reserved % ring_bytes
        pad = ring_bytes - pos if pos + r > ring_bytes else 0
        start = reserved + pad
        out.append(start % ring_bytes)
        reserved = start + r
    return out


def check_mpsc_log(workload_sizes, n_consumers: int, consumer: int, log, ring_bytes: int):
    """Interleaving-agnostic check of one consumer's delivery log.

    ``log`` is a sequence of (producer, seq, size, ring_offset) in the order
    the consumer drained them (ticket order). Valid iff: the multiset of
    (producer, seq) equals every message of the producers that feed this
    consumer, exactly once; each producer's messages arrive in push order;
    sizes match; offsets equal the reservation rule replayed in this order.
    Returns a list of problems (empty when valid)."""
    problems = []
    P, M = workload_sizes.shape
    expect = {(p, s) for p in range(consumer, P, n_consumers) for s in range(M)}
    seen = set()
    last = {}
    for t, (p, s, n, off) in enumerate(log):
        p, s, n = int(p), int(s), int(n)
        if (p, s) in seen:
            problems.append(f"ticket {t}: duplicate ({p},{s})")
        seen.add((p, s))
        if (p, s) not in expect:
            problems.append(f"ticket {t}: unexpected ({p},{s})")
            continue
        if s <= last.get(p, -1):
            problems.append(f"ticket {t}: producer {p} out of order ({s} after {last[p]})")
        last[p] = s
        if n != int(workload_sizes[p, s]):
            problems.append(f"ticket {t}: size {n} != {int(workload_sizes[p, s])}")
    missing = expect - seen
    if missing:
        problems.append(f"{len(missing)} messages missing")
    offs = replay_offsets([int(x[2]) for x in log], ring_bytes)
    bad = [t for t, (x, o) in enumerate(zip(log, offs)) if int(x[3]) != o]
    if bad:
        problems.append(f"{len(bad)} ring offsets differ from the reservation rule (first ticket {bad[0]})")
    return problems


class MpscNonLockingOracle:
    """Non-locking MPSC (Sec. 4.3): one ring per producer, no shared exclusive
    access. Each producer ring follows the placement rule of MpscOracle
    (16-byte rounding, skip to the start, capacity per ring). Reading for the
    host calls: the consumer drains producers in index order, each producer's
    messages oldest first, so peek(k) is the k-th message of that order."""

    def __init__(self, n_producers: int, ring_bytes: int, max_msgs: int):
        self.rings = [MpscOracle(1, ring_bytes, max_msgs) for _ in range(n_producers)]

    def push(self, producer: int, payload: np.ndarray) -> int:
        if producer < 0 or producer >= len(self.rings):
            return ERR_INVALID
        return self.rings[producer].push(0, payload)

    def _locate(self, k: int):
        for p, r in enumerate(self.rings):
            d = r.depth()[0]
            if k < d:
                return p, k
            k -= d
        return None

    def peek(self, k: int):
        loc = self._locate(k)
        if loc is None:
            return ERR_EMPTY, None
        p, j = loc
        st, (off, n, _, s) = self.rings[p].peek(j)
        return OK, (off, n, p, s)

    def payload(self, k: int) -> np.ndarray:
        p, j = self._locate(k)
        return self.rings[p].payload(j)

    def pop(self, count: int) -> int:
        if count > self.depth()[0]:
            return ERR_EMPTY
        for r in self.rings:
            take = min(count, r.depth()[0])
            r.pop(take)
            count -= take
        return OK

    def depth(self):
        m = sum(r.depth()[0] for r in self.rings)
        b = sum(r.depth()[1] for r in self.rings)
        return m, b


def check_mpsc_nl_log(workload_sizes, n_consumers: int, consumer: int, log, ring_bytes: int):
    """Interleaving-agnostic check of one non-locking consumer's log
    (producer, seq, size, ring offset) in consumption order: every message of
    the consumer's producers exactly once, each producer in push order, sizes
    equal, and each producer's offsets equal the placement rule replayed over
    that producer's own ring."""
    problems = []
    P, M = workload_sizes.shape
    per = {}
    for t, (p, s, n, off) in enumerate(log):
        per.setdefault(int(p), []).append((int(s), int(n), int(off), t))
    mine = list(range(consumer, P, n_consumers))
    if sorted(per) != mine:
        problems.append(f"producers seen {sorted(per)[:5]}... expected {mine[:5]}...")
    for p in mine:
        lst = per.get(p, [])
        if [x[0] for x in lst] != list(range(M)):
            problems.append(f"producer {p}: sequence numbers {[x[0] for x in lst][:8]}... not 0..{M - 1} in order")
            continue
        if [x[1] for x in lst] != [int(v) for v in workload_sizes[p]]:
            problems.append(f"producer {p}: sizes differ")
        if [x[2] for x in lst] != replay_offsets([x[1] for x in lst], ring_bytes):
            problems.append(f"producer {p}: ring offsets differ from the placement rule")
    return problems
