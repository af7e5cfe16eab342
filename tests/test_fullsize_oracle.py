"""Pins of the full-size oracle helpers (CPU): each equals the plain oracle
definition it restates on inputs small enough for the plain form."""
import numpy as np

from oracle import digest as od
from oracle import memcpy as om
from tests import fullsize_oracle as fo
from workloads import configs, splitmix


def test_final_slot_bytes_equals_the_comm_manager():
    w = configs.batched(4, n_slots=8, total_bytes=16 << 20, slot_lo=1 << 20, slot_hi=4 << 20, n_ops=400,
                        n_lo=1, n_hi=64 << 10)
    cm = om.CommManager()
    init = [splitmix.fill_bytes(4, s, 0, int(sz)) for s, sz in enumerate(w.slot_sizes)]
    for s in range(len(init)):
        cm.register(om.SPACE_HBM, init[s].copy())
    assert cm.memcpy_batch(w.ops) == (om.OK, None)
    for s in range(len(init)):
        got = om.final_slot_bytes(w.ops, s, init[s], lambda src, off, n: init[src][off:off + n])
        assert (got == cm.slots[s].data).all(), s
    # a table that writes a slot it also reads is refused, not mis-applied
    bad = configs.make_ops([0, 1], [1, 2], [0, 0], [0, 0], [4, 4])
    try:
        om.final_slot_bytes(bad, 0, init[0], lambda *a: None)
        raise AssertionError("accepted a table whose sources are written")
    except ValueError:
        pass


def test_block_and_segment_digests_equal_the_plain_digest():
    rng = np.random.default_rng(1)
    for n in (0, 8, 100, 4096, 4096 * 3 + 13):
        b = rng.integers(0, 256, n, dtype=np.uint8)
        d = od.block_digests(b, 4096)
        exp = [od.byte_digest(b[i:i + 4096]) for i in range(0, n, 4096)]
        assert [int(x) for x in d] == exp
    counts = np.array([0, 1, 5, 0, 17, 2])
    words = rng.integers(0, 1 << 63, int(counts.sum()), dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    got = od.segment_digests(words, counts)
    k = 0
    for i, c in enumerate(counts):
        assert int(got[i]) == od.word_digest_loop(words[k:k + c])
        k += c


def test_producer_message_digests_equal_the_payload_rule():
    rng = np.random.default_rng(2)
    for p in (0, 5, 1023):
        sizes = np.concatenate([[0, 1, 7, 8, 9, 15, 16, 17], rng.integers(0, 70000, 40)])
        got = fo.producer_message_digests(p, sizes)
        for s, n in enumerate(sizes):
            assert int(got[s]) == od.byte_digest(splitmix.mpsc_payload_bytes(p, s, int(n))), (p, s, n)
