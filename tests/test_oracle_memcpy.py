"""Pins of the memcpy / fence / counter oracle against things other than itself.

* a hand-worked example of the definition (tests/golden/memcpy_worked.txt);
* a single op equals Python ``bytes`` slicing and C's memcpy (ctypes.memmove
  on non-overlapping buffers);
* brute force on two 64-byte slots: every order of a hazard-free op set gives
  the same bytes, equal to a per-byte construction from the original slots;
* counters: closed forms for config 1 and from the op table;
* full-size helper (expected bytes one position at a time) equals applying
  the whole table;
* planted mistakes in the oracle are caught by these pins.
"""
import ctypes
import itertools
import os

import numpy as np
import pytest

from oracle import memcpy as om
from workloads import configs, splitmix

GOLD = os.path.join(os.path.dirname(__file__), "golden")
STATUS = {"OK": om.OK, "INVALID": om.ERR_INVALID, "BOUNDS": om.ERR_BOUNDS,
          "OVERLAP": om.ERR_OVERLAP, "UNSUPPORTED": om.ERR_UNSUPPORTED}


def load_worked():
    slots, ops, final, counts = {}, [], {}, {}
    for line in open(os.path.join(GOLD, "memcpy_worked.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        if f[0] == "slot":
            slots[f[1]] = bytes.fromhex(f[2])
        elif f[0] == "op":
            ops.append((f[1], int(f[2]), f[3], int(f[4]), int(f[5]), f[6]))
        elif f[0] == "final":
            final[f[1]] = bytes.fromhex(f[2])
        elif f[0] == "count":
            counts[f[1]] = (int(f[2]), int(f[3]))
    return slots, ops, final, counts


def run_worked(cm_cls=om.CommManager):
    slots, ops, final, counts = load_worked()
    cm = cm_cls()
    ids = {name: cm.register(om.SPACE_HBM, np.frombuffer(b, dtype=np.uint8).copy()) for name, b in slots.items()}
    statuses = []
    for d, doff, s, soff, n, _ in ops:
        statuses.append(cm.memcpy(ids.get(d, 99), doff, ids.get(s, 99), soff, n))
    return cm, ids, statuses, ops, final, counts


def test_worked_example():
    cm, ids, statuses, ops, final, counts = run_worked()
    assert statuses == [STATUS[o[5]] for o in ops]
    for name, b in final.items():
        assert bytes(cm.slots[ids[name]].data) == b
    for name, (s, r) in counts.items():
        assert cm.counters(ids[name]) == (s, r)
    assert cm.fence(0) == om.OK
    assert cm.tag_ops[0] == 4  # the four accepted ops, all on tag 0


def test_single_op_equals_bytes_slicing_and_c_memcpy():
    rng = np.random.default_rng(1)
    for _ in range(200):
        ns, nd = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        src = rng.integers(0, 256, ns, dtype=np.uint8)
        dst = rng.integers(0, 256, nd, dtype=np.uint8)
        n = int(rng.integers(0, min(ns, nd) + 1))
        soff = int(rng.integers(0, ns - n + 1))
        doff = int(rng.integers(0, nd - n + 1))
        cm = om.CommManager()
        a = cm.register(om.SPACE_HBM, src.copy())
        b = cm.register(om.SPACE_HBM, dst.copy())
        assert cm.memcpy(b, doff, a, soff, n) == om.OK
        sb, db = bytes(src), bytes(dst)
        assert bytes(cm.slots[b].data) == db[:doff] + sb[soff:soff + n] + db[doff + n:]
        buf = ctypes.create_string_buffer(db, nd)
        sbuf = ctypes.create_string_buffer(sb, ns)
        ctypes.memmove(ctypes.addressof(buf) + doff, ctypes.addressof(sbuf) + soff, n)
        assert bytes(cm.slots[b].data) == buf.raw[:nd]
        assert bytes(cm.slots[a].data) == sb  # source untouched
        assert cm.counters(a) == (1, 0) and cm.counters(b) == (0, 1)


def test_rejections_have_no_effect():
    cm = om.CommManager()
    a = cm.register(om.SPACE_HBM, np.arange(32, dtype=np.uint8))
    h = cm.register(om.SPACE_HOST, np.zeros(32, dtype=np.uint8))
    before = cm.slots[a].data.copy()
    assert cm.memcpy(a, 0, h, 0, 4) == om.ERR_UNSUPPORTED
    assert cm.memcpy(h, 0, a, 0, 4) == om.ERR_UNSUPPORTED
    assert cm.memcpy(a, 32, a, 0, 1) == om.ERR_BOUNDS
    assert cm.memcpy(a, 31, a, 0, 1) == om.OK          # last byte; [0,1) vs [31,32)
    assert cm.memcpy(a, 0, a, 31, 2) == om.ERR_BOUNDS
    assert cm.memcpy(a, 1, a, 0, 2) == om.ERR_OVERLAP
    assert cm.memcpy(a, 0, a, 1, 2) == om.ERR_OVERLAP
    assert cm.memcpy(a, 2, a, 0, 2) == om.OK           # touching, not intersecting
    assert cm.memcpy(a, 5, a, 5, 0) == om.OK           # zero-size same range
    assert cm.memcpy(a, 1, a, (1 << 64) - 1, 1) == om.ERR_BOUNDS
    assert cm.deregister(a) == om.OK
    assert cm.memcpy(a, 0, a, 8, 1) == om.ERR_INVALID
    assert cm.counters(a) == (3, 3)
    exp = before.copy()
    exp[31] = exp[0]
    exp[2:4] = exp[0:2]
    assert (cm.slots[a].data == exp).all()


def test_batch_all_or_nothing():
    cm = om.CommManager()
    a = cm.register(om.SPACE_HBM, np.arange(64, dtype=np.uint8))
    b = cm.register(om.SPACE_HBM, np.zeros(64, dtype=np.uint8))
    ops = configs.make_ops([b, b, b], [a, a, a], [0, 10, 60], [0, 0, 0], [4, 4, 5])
    st, bad = cm.memcpy_batch(ops)
    assert (st, bad) == (om.ERR_BOUNDS, 2)
    assert (cm.slots[b].data == 0).all() and cm.counters(b) == (0, 0)
    ops = configs.make_ops([b, b], [a, a], [0, 2], [0, 10], [4, 4])
    assert cm.memcpy_batch(ops, checked=True) == (om.ERR_HAZARD, 1)
    assert cm.memcpy_batch(ops[:1], checked=True) == (om.OK, None)


def _touch_sets(op):
    """The (slot, byte) pairs an op writes and reads, spelled out byte by byte."""
    dst, doff, src, soff, n = op
    return {(dst, doff + i) for i in range(n)}, {(src, soff + i) for i in range(n)}


def _first_hazard_plain(ops):
    """Two ops conflict iff some byte written by one is read or written by the
    other; the answer is the first op (issue order) that conflicts with an
    earlier one."""
    sets = [_touch_sets(o) for o in ops]
    for j in range(len(ops)):
        wj, rj = sets[j]
        for i in range(j):
            wi, ri = sets[i]
            if wi & (wj | rj) or wj & ri:
                return j
    return None


def _as_table(ops):
    return configs.make_ops([o[0] for o in ops], [o[2] for o in ops], [o[1] for o in ops],
                            [o[3] for o in ops], [o[4] for o in ops])


def test_first_hazard_equals_the_byte_set_construction():
    """first_hazard pinned in both directions: every hazard the byte sets show
    is reported (none missed) and nothing else is (no src/src overlap, no
    adjacent-but-disjoint ranges, no zero-size op counts). All ordered pairs
    of ops on two 32-byte slots with offsets and sizes at the interesting
    corners, then random triples over every offset and size."""
    size = 32
    offs = [0, 1, 7, 15, 16, 17, 24, 31]
    ns = [0, 1, 2, 8, 15, 16, 17]
    singles = [(d, do, s, so, n) for d in (0, 1) for s in (0, 1) for n in ns for do in offs for so in offs
               if do + n <= size and so + n <= size]
    rng = np.random.default_rng(11)
    pairs = [(singles[a], singles[b]) for a, b in rng.integers(0, len(singles), size=(12000, 2))]
    hits = 0
    for ops in pairs:
        exp = _first_hazard_plain(ops)
        hits += exp is not None
        assert om.first_hazard(_as_table(ops)) == exp, ops
    assert 0.1 * len(pairs) < hits < 0.9 * len(pairs)
    for _ in range(3000):
        ops = []
        for _ in range(3):
            n = int(rng.integers(0, 12))
            ops.append((int(rng.integers(0, 2)), int(rng.integers(0, size - n + 1)), int(rng.integers(0, 2)),
                        int(rng.integers(0, size - n + 1)), n))
        assert om.first_hazard(_as_table(ops)) == _first_hazard_plain(ops), ops
    # the corners an over-strict checker would flag
    assert om.first_hazard(_as_table([(1, 0, 0, 0, 8), (1, 8, 0, 0, 8)])) is None     # adjacent dsts, shared src
    assert om.first_hazard(_as_table([(1, 0, 0, 4, 8), (1, 8, 0, 8, 8)])) is None     # overlapping srcs only
    assert om.first_hazard(_as_table([(1, 0, 0, 0, 8), (0, 8, 1, 8, 4)])) is None     # dst next to a src
    assert om.first_hazard(_as_table([(1, 4, 0, 0, 0), (1, 0, 0, 0, 8)])) is None     # zero-size op inside
    assert om.first_hazard(_as_table([(1, 0, 0, 0, 8), (0, 0, 1, 7, 1)])) == 1        # one-byte read of a dst


def _hazard_free_sets(rng, k, size=64):
    while True:
        ops = []
        for _ in range(k):
            n = int(rng.integers(0, 12))
            src, dst = (0, 1) if rng.random() < 0.8 else (1, 0)
            ops.append((dst, int(rng.integers(0, size - n + 1)), src, int(rng.integers(0, size - n + 1)), n))
        arr = configs.make_ops([o[0] for o in ops], [o[2] for o in ops], [o[1] for o in ops],
                               [o[3] for o in ops], [o[4] for o in ops])
        if om.first_hazard(arr) is None:
            return ops


def per_byte_construction(orig, ops):
    """Hazard-free set: no op's source is written by another, so each written
    byte takes the ORIGINAL source byte; built with bytes concatenation."""
    out = [bytearray(o) for o in orig]
    for d, doff, s, soff, n in ops:
        seg = bytes(orig[s])[soff:soff + n]
        out[d] = out[d][:doff] + bytearray(seg) + out[d][doff + n:]
    return [bytes(x) for x in out]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_brute_force_orders(k):
    rng = np.random.default_rng(100 + k)
    for trial in range(4 if k >= 5 else 12):
        ops = _hazard_free_sets(rng, k)
        orig = [bytes(rng.integers(0, 256, 64, dtype=np.uint8)), bytes(rng.integers(0, 256, 64, dtype=np.uint8))]
        expect = per_byte_construction(orig, ops)
        perms = list(itertools.permutations(range(k)))
        if len(perms) > 120:
            perms = [perms[int(i)] for i in rng.choice(len(perms), 120, replace=False)]
        for perm in perms:
            cm = om.CommManager()
            ids = [cm.register(om.SPACE_HBM, np.frombuffer(o, dtype=np.uint8).copy()) for o in orig]
            for j in perm:
                d, doff, s, soff, n = ops[j]
                assert cm.memcpy(ids[d], doff, ids[s], soff, n) == om.OK
            assert [bytes(cm.slots[i].data) for i in ids] == expect
            sent = sum(1 for o in ops if o[2] == 0)
            assert cm.counters(ids[0]) == (sent, k - sent)


def test_tiny_config_counters_closed_form():
    w = configs.tiny(0)
    sent, recv = om.counters_from_ops(w.ops, 2)
    assert (int(sent[0]), int(recv[1])) == (1024, 1024)
    assert (int(sent[1]), int(recv[0])) == (0, 0)
    # the oracle reaches the same counts by executing the table
    cm = om.CommManager()
    s = cm.register(om.SPACE_HBM, splitmix.fill_bytes(0, 0, 0, 1 << 16).repeat(1024)[: 64 << 20])
    d = cm.register(om.SPACE_HBM, np.zeros(64 << 20, dtype=np.uint8))
    assert cm.memcpy_batch(w.ops, checked=False) == (om.OK, None)
    assert cm.counters(s) == (1024, 0) and cm.counters(d) == (0, 1024)
    assert cm.fence_slot(d, 0, 1024) == om.OK
    assert cm.fence_slot(d, 0, 1025) == om.ERR_TIMEOUT


def _apply_full(w, seed):
    cm = om.CommManager()
    ids = []
    for s, sz in enumerate(w.slot_sizes):
        ids.append(cm.register(om.SPACE_HBM, splitmix.fill_bytes(seed, s, 0, int(sz))))
    for a, b in w.epochs:
        assert cm.memcpy_batch(w.ops[a:b]) == (om.OK, None)
    return cm, ids


def test_sampled_expected_bytes_equal_full_apply():
    w = configs.batched(3, n_slots=8, total_bytes=8 << 20, slot_lo=256 << 10, slot_hi=4 << 20,
                        n_ops=300, n_lo=16, n_hi=256 << 10)
    assert len(w.epochs) >= 2
    cm, ids = _apply_full(w, 3)
    init = lambda slot, pos: splitmix.fill_byte_at(3, slot, pos)  # noqa: E731
    for s in range(len(ids)):
        pos = np.arange(int(w.slot_sizes[s]))
        got = om.expected_bytes_at(w.ops, w.epochs, s, pos, init)
        assert (got == cm.slots[ids[s]].data).all(), s


def test_chained_epochs_follow_sources():
    # epoch 2 copies from a range written in epoch 1: the value must chain
    ops = configs.make_ops([1, 0], [0, 1], [0, 32], [0, 0], [8, 8])
    epochs = [(0, 1), (1, 2)]
    init = lambda slot, pos: (np.asarray(pos) + 100 * slot).astype(np.uint8)  # noqa: E731
    got = om.expected_bytes_at(ops, epochs, 0, np.arange(32, 40), init)
    assert list(got) == list(range(0, 8))


# -- planted mistakes: the pins above must catch each of them ---------------

class _OffByOne(om.CommManager):
    def _apply(self, dst, doff, src, soff, n):
        d, s = self.slots[dst], self.slots[src]
        if n:
            d.data[doff:doff + n - 1] = s.data[soff:soff + n - 1]
        self.sent[src] += 1
        self.recv[dst] += 1


class _SwappedCounters(om.CommManager):
    def _apply(self, dst, doff, src, soff, n):
        super()._apply(dst, doff, src, soff, n)
        self.sent[src] -= 1
        self.recv[dst] -= 1
        self.sent[dst] += 1
        self.recv[src] += 1


class _NoOverlapCheck(om.CommManager):
    def validate(self, dst, doff, src, soff, n):
        st = super().validate(dst, doff, src, soff, n)
        return om.OK if st == om.ERR_OVERLAP else st


class _InclusiveBound(om.CommManager):
    def validate(self, dst, doff, src, soff, n):
        d = self.slots.get(dst)
        if d is not None and n > 0 and doff + n == len(d.data):
            return om.ERR_BOUNDS
        return super().validate(dst, doff, src, soff, n)


@pytest.mark.parametrize("mutant", [_OffByOne, _SwappedCounters, _NoOverlapCheck, _InclusiveBound])
def test_planted_mistakes_are_caught(mutant):
    caught = False
    try:
        cm, ids, statuses, ops, final, counts = run_worked(mutant)
        ok = statuses == [STATUS[o[5]] for o in ops]
        ok = ok and all(bytes(cm.slots[ids[n]].data) == b for n, b in final.items())
        ok = ok and all(cm.counters(ids[n]) == c for n, c in counts.items())
        caught = not ok
    except (AssertionError, ValueError, IndexError):
        caught = True
    assert caught
