"""The all-cores CPU memcpy baseline (oracle/memcpy_threads.c) gives the same
slots as the single-threaded oracle for every thread count, including byte
ranges that split ops between threads, and a single op equals numpy slicing."""
import shutil

import numpy as np
import pytest

from oracle import memcpy as om
from workloads import configs, splitmix

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")


def _slots(w, seed):
    return [splitmix.fill_bytes(seed, s, 0, int(sz)) for s, sz in enumerate(w.slot_sizes)]


@pytest.mark.parametrize("threads", [1, 3, 8, 61])
def test_threaded_equals_oracle(threads):
    from oracle.native import ThreadedMemcpy
    w = configs.batched(4, n_slots=8, total_bytes=24 << 20, slot_lo=1 << 20, slot_hi=8 << 20, n_ops=1500,
                        n_lo=1, n_hi=256 << 10, max_gap=64)
    assert len(w.epochs) >= 2
    cm = om.CommManager()
    ids = [cm.register(om.SPACE_HBM, a) for a in _slots(w, 4)]
    for a, b in w.epochs:
        assert cm.memcpy_batch(w.ops[a:b]) == (om.OK, None)
        cm.fence(0)
    mine = _slots(w, 4)
    assert ThreadedMemcpy(mine, w.ops, w.epochs).run(threads) == 0
    for k, i in enumerate(ids):
        assert (mine[k] == cm.slots[i].data).all(), k


def test_single_op_is_slicing():
    from oracle.native import ThreadedMemcpy
    a = np.arange(1000, dtype=np.uint8)
    b = np.zeros(1000, dtype=np.uint8)
    ops = configs.make_ops([1], [0], [17], [3], [901])
    ThreadedMemcpy([a, b], ops, [(0, 1)]).run(4)
    exp = np.zeros(1000, dtype=np.uint8)
    exp[17:918] = a[3:904]
    assert (b == exp).all()
