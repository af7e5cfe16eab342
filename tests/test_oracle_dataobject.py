"""Pins of the Data Object oracle: a hand-worked program (values computed by
hand from the definition) and the reduction of get to bytes slicing."""
import numpy as np

from oracle import memcpy as om
from oracle.dataobject import DataObjects


def test_worked_program():
    cm = om.CommManager()
    a = cm.register(om.SPACE_HBM, np.arange(16, dtype=np.uint8))
    b = cm.register(om.SPACE_HBM, np.zeros(8, dtype=np.uint8))
    do = DataObjects(cm)
    assert do.publish(a, 4, 4) == (om.OK, 1)          # bytes 4..7
    assert do.publish(a, 14, 3) == (om.ERR_BOUNDS, None)
    assert do.publish(a, 0, 2) == (om.OK, 2)          # ids count on
    assert do.get_handle(1) == (om.OK, (1, 4, om.SPACE_HBM))
    assert do.get(1, b, 2) == om.OK                   # b = 0 0 4 5 6 7 0 0
    assert do.get(2, b, 7) == om.ERR_BOUNDS
    assert do.get(2, a, 1) == om.ERR_OVERLAP          # [0,2) vs [1,3) in one slot
    assert do.release(1) == om.OK
    assert do.get(1, b, 0) == om.ERR_INVALID
    assert do.release(1) == om.ERR_INVALID
    assert do.get_handle(1) == (om.ERR_INVALID, None)
    assert list(cm.slots[b].data) == [0, 0, 4, 5, 6, 7, 0, 0]
    assert cm.counters(a) == (1, 0) and cm.counters(b) == (0, 1)


def test_get_is_bytes_slicing():
    rng = np.random.default_rng(0)
    for _ in range(100):
        src = rng.integers(0, 256, 200, dtype=np.uint8)
        dst = rng.integers(0, 256, 150, dtype=np.uint8)
        cm = om.CommManager()
        s = cm.register(om.SPACE_HBM, src.copy())
        d = cm.register(om.SPACE_HBM, dst.copy())
        do = DataObjects(cm)
        n = int(rng.integers(0, 100))
        off = int(rng.integers(0, 200 - n + 1))
        doff = int(rng.integers(0, 150 - n + 1))
        st, k = do.publish(s, off, n)
        assert do.get(k, d, doff) == om.OK
        assert bytes(cm.slots[d].data) == bytes(dst)[:doff] + bytes(src)[off:off + n] + bytes(dst)[doff + n:]
