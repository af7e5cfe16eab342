"""Pins of the channel oracle.

* SPSC: random push/pop/peek programs against a bounded FIFO built from
  ``collections.deque`` (a library queue), including all-or-nothing pushes;
* MPSC: a hand-worked wrap-around example (tests/golden/mpsc_wrap.txt), one
  producer reduces to the FIFO, capacity invariant under random programs,
  per-producer order, replay of offsets;
* digests: the numpy reduction equals the plain integer loop, and the digest
  reacts to a changed, moved or dropped word;
* planted mistakes in the oracle are caught.
"""
import os
from collections import deque

import numpy as np
import pytest

from oracle import channels as oc
from oracle import digest as od
from oracle import memcpy as om
from workloads import splitmix

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ST = {"OK": om.OK, "FULL": om.ERR_FULL, "EMPTY": om.ERR_EMPTY, "TOO_LARGE": om.ERR_TOO_LARGE}


@pytest.mark.parametrize("seed", range(6))
def test_spsc_matches_bounded_deque(seed):
    rng = np.random.default_rng(seed)
    tb, cap = 8, int(rng.integers(1, 9))
    ch = oc.SpscOracle(tb, cap)
    ref = deque()
    counter = 0
    for _ in range(400):
        r = rng.random()
        if r < 0.45:
            k = int(rng.integers(0, cap + 2))
            toks = [bytes([(counter + j) % 256] * tb) for j in range(k)]
            st = ch.push(np.frombuffer(b"".join(toks), dtype=np.uint8) if k else np.zeros(0, np.uint8))
            if len(ref) + k <= cap:
                assert st == om.OK
                ref.extend(toks)
                counter += k
            else:
                assert st == om.ERR_FULL
        elif r < 0.8:
            k = int(rng.integers(0, cap + 2))
            st = ch.pop(k)
            if k <= len(ref):
                assert st == om.OK
                for _ in range(k):
                    ref.popleft()
            else:
                assert st == om.ERR_EMPTY
        else:
            k = int(rng.integers(0, cap + 1))
            st, info = ch.peek(k)
            if k < len(ref):
                assert st == om.OK and bytes(ch.token(k)) == ref[k]
            else:
                assert st == om.ERR_EMPTY
        assert ch.depth() == (len(ref), len(ref) * tb)
        assert 0 <= ch.head - ch.tail <= cap


def load_mpsc_golden():
    prog = []
    for line in open(os.path.join(GOLD, "mpsc_wrap.txt")):
        line = line.split("#")[0].strip()
        if line:
            prog.append(line.split())
    return prog


def run_mpsc_golden(cls=oc.MpscOracle):
    prog = load_mpsc_golden()
    R, M, P = map(int, prog[0][1:])
    ch = cls(P, R, M)
    mism = []
    for f in prog[1:]:
        if f[0] == "push":
            p, n = int(f[1]), int(f[2])
            before = ch.placement(n)[0] % R
            st = ch.push(p, splitmix.mpsc_payload_bytes(p, ch.seq[p], n))
            if st != ST[f[3]] or (st == om.OK and before != int(f[4])):
                mism.append(f)
        elif f[0] == "pop":
            if ch.pop(int(f[1])) != ST[f[2]]:
                mism.append(f)
        elif f[0] == "peek":
            st, info = ch.peek(int(f[1]))
            if st != ST[f[2]] or (st == om.OK and list(info) != [int(x) for x in f[3:7]]):
                mism.append(f)
        elif f[0] == "depth":
            if ch.depth() != (int(f[1]), int(f[2])):
                mism.append(f)
    return mism


def test_mpsc_golden_wraparound():
    assert run_mpsc_golden() == []


def test_mpsc_single_producer_is_fifo():
    rng = np.random.default_rng(7)
    ch = oc.MpscOracle(1, 4096, 64)
    ref = deque()
    for step in range(2000):
        if rng.random() < 0.55:
            n = int(rng.integers(0, 700))
            payload = rng.integers(0, 256, n, dtype=np.uint8)
            st = ch.push(0, payload)
            if st == om.OK:
                ref.append(bytes(payload))
            else:
                assert st == om.ERR_FULL
                # FULL only when the rule says so
                start, end = ch.placement(n)
                assert end - ch.freed > 4096 or len(ref) + 1 > 64
        elif ref:
            assert bytes(ch.payload(0)) == ref[0]
            assert ch.pop(1) == om.OK
            ref.popleft()
        assert ch.depth()[0] == len(ref)
        assert ch.reserved - ch.freed <= 4096
    assert ch.max_inflight <= 4096


def test_mpsc_many_producers_order_capacity_and_replay():
    rng = np.random.default_rng(11)
    P, R, M = 5, 1 << 14, 32
    ch = oc.MpscOracle(P, R, M)
    log = []
    sizes = {}
    for step in range(5000):
        p = int(rng.integers(0, P))
        if rng.random() < 0.6:
            n = int(np.exp(rng.uniform(np.log(8), np.log(4000))))
            s = ch.seq[p]
            st = ch.push(p, splitmix.mpsc_payload_bytes(p, s, n))
            if st == om.OK:
                sizes[(p, s)] = n
            assert ch.reserved - ch.freed <= R
        elif ch.depth()[0]:
            st, (off, n, pp, s) = ch.peek(0)
            assert (ch.payload(0) == splitmix.mpsc_payload_bytes(pp, s, n)).all()
            log.append((pp, s, n, off))
            assert ch.pop(1) == om.OK
    # per-producer order in delivery and the reservation rule replays offsets
    last = {}
    for p, s, n, off in log:
        assert s > last.get(p, -1)
        last[p] = s
    assert [x[3] for x in log] == oc.replay_offsets([x[2] for x in log], R)


def test_check_mpsc_log_detects_faults():
    P, M, C, R = 4, 3, 2, 4096
    sizes = np.array([[10, 20, 30], [40, 50, 60], [70, 80, 90], [15, 25, 35]])
    order = [(0, 0), (2, 0), (0, 1), (2, 1), (2, 2), (0, 2)]
    ns = [int(sizes[p, s]) for p, s in order]
    offs = oc.replay_offsets(ns, R)
    log = [(p, s, n, o) for (p, s), n, o in zip(order, ns, offs)]
    assert oc.check_mpsc_log(sizes, C, 0, log, R) == []
    swapped = log[:]
    swapped[0], swapped[2] = swapped[2], swapped[0]
    assert oc.check_mpsc_log(sizes, C, 0, swapped, R)          # producer order broken
    assert oc.check_mpsc_log(sizes, C, 0, log[:-1], R)         # a message missing
    assert oc.check_mpsc_log(sizes, C, 0, log + [log[0]], R)   # a duplicate
    moved = [tuple(x) for x in log]
    moved[3] = (moved[3][0], moved[3][1], moved[3][2], moved[3][3] + 16)
    assert oc.check_mpsc_log(sizes, C, 0, moved, R)            # wrong offset


def test_replay_offsets_skip_to_start():
    assert oc.replay_offsets([20, 10, 30, 1], 64) == [0, 32, 0, 32]
    assert oc.replay_offsets([48, 16, 16], 64) == [0, 48, 0]
    assert oc.replay_offsets([0, 0, 5], 64) == [0, 0, 0]


def test_digest_numpy_equals_loop_and_reacts():
    rng = np.random.default_rng(3)
    w = rng.integers(0, 1 << 63, 257, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    d = od.word_digest(w)
    assert d == od.word_digest_loop(w)
    assert od.word_digest(w[5:], 5) == od.word_digest_loop(w[5:], 5)
    changed = w.copy()
    changed[17] ^= np.uint64(1 << 40)
    assert od.word_digest(changed) != d
    moved = w.copy()
    moved[[3, 9]] = moved[[9, 3]]
    assert od.word_digest(moved) != d
    assert od.word_digest(w[:-1]) != d
    # byte digest: zero padding of the last word, little endian
    b = np.arange(1, 12, dtype=np.uint8)
    assert od.byte_digest(b) == (0x0807060504030201 + 3 * 0x0B0A09) % (1 << 64)


class _NoSkip(oc.MpscOracle):
    def placement(self, n):
        r = oc.round_up(n)
        return self.reserved, self.reserved + r


class _NoRound(oc.MpscOracle):
    def placement(self, n):
        pos = self.reserved % self.R
        pad = self.R - pos if pos + n > self.R else 0
        return self.reserved + pad, self.reserved + pad + n


class _LooseCapacity(oc.MpscOracle):
    def push(self, producer, payload):
        saved = self.freed
        self.freed += 16
        try:
            return super().push(producer, payload)
        finally:
            self.freed = saved


@pytest.mark.parametrize("mutant", [_NoSkip, _NoRound, _LooseCapacity])
def test_mpsc_planted_mistakes_are_caught(mutant):
    try:
        mism = run_mpsc_golden(mutant)
    except (AssertionError, ValueError, IndexError):
        mism = ["raised"]
    assert mism


def test_nonlocking_reduces_to_per_producer_fifos():
    rng = np.random.default_rng(21)
    P, R, M = 3, 1024, 8
    ch = oc.MpscNonLockingOracle(P, R, M)
    refs = [deque() for _ in range(P)]
    for step in range(3000):
        if rng.random() < 0.55:
            p = int(rng.integers(0, P))
            n = int(rng.integers(0, 300))
            payload = rng.integers(0, 256, n, dtype=np.uint8)
            st = ch.push(p, payload)
            if st == om.OK:
                refs[p].append(bytes(payload))
            else:
                assert st in (om.ERR_FULL, om.ERR_TOO_LARGE)
        else:
            flat = [m for r in refs for m in r]
            k = int(rng.integers(0, 4))
            if k < len(flat):
                assert bytes(ch.payload(k)) == flat[k]
            c = int(rng.integers(0, 3))
            st = ch.pop(c)
            if c <= len(flat):
                assert st == om.OK
                for _ in range(c):  # remove in index order
                    for r in refs:
                        if r:
                            r.popleft()
                            break
            else:
                assert st == om.ERR_EMPTY
        assert ch.depth()[0] == sum(len(r) for r in refs)


def test_check_mpsc_nl_log():
    sizes = np.array([[10, 20], [30, 40], [50, 60], [70, 80]])
    log = [(0, 0, 10, 0), (2, 0, 50, 0), (0, 1, 20, 16), (2, 1, 60, 64)]
    assert oc.check_mpsc_nl_log(sizes, 2, 0, log, 128) == []
    bad = [log[2], log[1], log[0], log[3]]
    assert oc.check_mpsc_nl_log(sizes, 2, 0, bad, 128)
    assert oc.check_mpsc_nl_log(sizes, 2, 0, log[:3], 128)


def _nl_program(cls, seed=5):
    """A random push/peek/pop program on a non-locking channel checked against
    per-producer FIFOs (deques) and the placement rule replayed per ring;
    returns the number of mismatches."""
    rng = np.random.default_rng(seed)
    P, R, M = 3, 512, 4
    ch = cls(P, R, M)
    refs = [deque() for _ in range(P)]
    placed = [[] for _ in range(P)]
    bad = 0
    for step in range(1500):
        if rng.random() < 0.55:
            p = int(rng.integers(0, P))
            n = int(rng.integers(1, 200))
            payload = rng.integers(0, 256, n, dtype=np.uint8)
            depth_ok = len(refs[p]) < M
            if ch.push(p, payload) == om.OK:
                refs[p].append(bytes(payload))
                placed[p].append(n)
                bad += not depth_ok
        else:
            flat = [(p, m) for p, r in enumerate(refs) for m in r]
            if flat:
                st, info = ch.peek(0)
                if st != om.OK or bytes(ch.payload(0)) != flat[0][1] or info[2] != flat[0][0]:
                    bad += 1
                ch.pop(1)
                for r in refs:
                    if r:
                        r.popleft()
                        break
    for p in range(P):  # offsets of every message a ring ever held follow the rule
        offs = [e[0] % R for e in ch.rings[p].meta]
        exp = oc.replay_offsets(placed[p], R)[len(placed[p]) - len(offs):] if offs else []
        bad += offs != exp
    return bad


class _NLReverseDrain(oc.MpscNonLockingOracle):
    def _locate(self, k):
        for p in reversed(range(len(self.rings))):
            d = self.rings[p].depth()[0]
            if k < d:
                return p, k
            k -= d
        return None


class _NLNoSkip(oc.MpscNonLockingOracle):
    def __init__(self, n_producers, ring_bytes, max_msgs):
        self.rings = [_NoSkip(1, ring_bytes, max_msgs) for _ in range(n_producers)]


class _NLLooseCapacity(oc.MpscNonLockingOracle):
    def __init__(self, n_producers, ring_bytes, max_msgs):
        self.rings = [oc.MpscOracle(1, ring_bytes, max_msgs + 1) for _ in range(n_producers)]


def test_nonlocking_program_is_clean():
    assert _nl_program(oc.MpscNonLockingOracle) == 0


@pytest.mark.parametrize("mutant", [_NLReverseDrain, _NLNoSkip, _NLLooseCapacity])
def test_nonlocking_planted_mistakes_are_caught(mutant):
    try:
        bad = _nl_program(mutant)
    except (AssertionError, ValueError, IndexError):
        bad = 1
    assert bad > 0
