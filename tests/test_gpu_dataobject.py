"""Data Object frontend through the C ABI against the oracle."""
import numpy as np
import pytest
import torch

from oracle import memcpy as om
from oracle.dataobject import DataObjects
from workloads import splitmix
from tests.gpu_util import fill_key, h, inst, slot_bytes  # noqa: F401

pytestmark = pytest.mark.gpu


def test_publish_get_release_match_oracle(h, inst):
    sizes = [1 << 20, 1 << 19]
    ids = []
    for s, sz in enumerate(sizes):
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, sz)
        assert h.hicr_util_fill(inst, sid, 0, sz, fill_key(4, s)) == 0
        ids.append(sid)
    cm = om.CommManager()
    oids = [cm.register(om.SPACE_HBM, splitmix.fill_bytes(4, s, 0, sz)) for s, sz in enumerate(sizes)]
    do = DataObjects(cm)
    rng = np.random.default_rng(1)
    objs = []
    for k in range(40):
        n = int(rng.integers(0, 20000))
        off = int(rng.integers(0, sizes[0] - n + 1))
        st, oid = h.hicr_dobj_publish(inst, ids[0], off, n)
        est, eid = do.publish(oids[0], off, n)
        assert (st, oid) == (est, eid)
        objs.append((oid, n))
    assert h.hicr_dobj_publish(inst, ids[0], sizes[0] - 3, 4)[0] == h.HICR_ERR_BOUNDS
    cursor = 0
    for oid, n in objs[:30]:
        st, hd = h.hicr_dobj_get_handle(inst, oid)
        assert st == 0 and (hd.id, hd.size, hd.space) == do.get_handle(oid)[1]
        assert h.hicr_dobj_get(inst, hd, ids[1], cursor) == do.get(oid, oids[1], cursor)
        cursor += n + int(rng.integers(0, 100))
    assert h.hicr_fence(inst, 0, 10_000_000_000) == 0
    assert (slot_bytes(h, inst, ids[1]) == cm.slots[oids[1]].data).all()
    assert h.hicr_slot_counters(inst, ids[1])[1:] == cm.counters(oids[1])
    oid = objs[0][0]
    assert h.hicr_dobj_release(inst, oid) == do.release(oid) == 0
    assert h.hicr_dobj_get_handle(inst, oid)[0] == h.HICR_ERR_INVALID
    assert h.hicr_dobj_release(inst, oid) == h.HICR_ERR_INVALID
