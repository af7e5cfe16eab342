"""hicr_memcpy_batch_noalloc against the regular device-validated batch.

Some callers cannot allocate GPU memory at the moment they issue copies (a
framework whose own pool owns all device memory, a latency-critical loop that
cannot absorb cudaMalloc's implicit synchronisation). They use
hicr_memcpy_batch_noalloc, whose scratch is a static device array instead of
cudaMalloc'd memory. Here both entry points run the same op tables on two
identically filled sets of slots and must leave identical bytes and counters,
on two calls in a row, and both must equal the CPU oracle byte for byte; a
batch of exactly the maximum op count runs, an oversized batch is rejected,
an invalid batch (also one whose bad op is the last of a maximum-size table)
reports its error and index without disturbing the next call, and repeated
calls leave the device's free memory unchanged.

This file is collected last so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, h, inst, slot_bytes  # noqa: F401

pytestmark = pytest.mark.gpu

T = 60_000_000_000


def _slots(h, inst, w, seed):
    ids = []
    for s, sz in enumerate(w.slot_sizes):
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, int(sz))
        assert st == 0
        assert h.hicr_util_fill(inst, sid, 0, int(sz), splitmix.fill_key_base(seed, s)) == 0
        ids.append(sid)
    return ids


def _table(ops, ids):
    o = ops.copy()
    m = np.asarray(ids, dtype=np.uint32)
    o["dst"], o["src"] = m[ops["dst"]], m[ops["src"]]
    return torch.from_numpy(o.view(np.uint8).copy()).cuda()


def _oracle(w, seed):
    cm = om.CommManager()
    for s, sz in enumerate(w.slot_sizes):
        assert cm.register(om.SPACE_HBM, splitmix.fill_bytes(seed, s, 0, int(sz))) == s
    return cm


def _matches_oracle(h, inst, ids, cm):
    for k, sid in enumerate(ids):
        assert (slot_bytes(h, inst, sid) == cm.slots[k].data).all(), f"slot {k} differs from the oracle"
        assert h.hicr_slot_counters(inst, sid)[1:] == cm.counters(k), k


def _same(h, inst, a_ids, b_ids):
    for a, b in zip(a_ids, b_ids):
        _, pa, na, _, _ = h.hicr_slot_info(inst, a)
        _, pb, nb, _, _ = h.hicr_slot_info(inst, b)
        torch.cuda.synchronize()
        assert na == nb and torch.equal(device_bytes(pa, na), device_bytes(pb, nb))
        assert h.hicr_slot_counters(inst, a)[1:] == h.hicr_slot_counters(inst, b)[1:]


@pytest.mark.parametrize("engine", [0, 1])
def test_noalloc_matches_device_batch_twice(h, inst, engine):
    if engine == 1:  # the TMA engine (its stages are shared memory, still no allocation)
        st, c = h.hicr_batch_get_config(inst)
        c.engine, c.threads, c.blocks_per_sm, c.tma_min_bytes = 1, 256, 1, 4096
        assert h.hicr_batch_set_config(inst, c) == 0
    w = configs.batched(5, n_slots=6, total_bytes=48 << 20, slot_lo=4 << 20, slot_hi=16 << 20,
                        n_ops=6000, n_lo=16, n_hi=512 << 10)
    assert len(w.epochs) >= 2
    a_ids = _slots(h, inst, w, 5)   # written by the no-allocation entry point
    b_ids = _slots(h, inst, w, 5)   # written by hicr_memcpy_batch_device
    cm = _oracle(w, 5)
    for call, (lo, hi) in enumerate(w.epochs[:2]):
        count = min(hi - lo, h.HICR_NOALLOC_MAX_OPS)
        ta, tb = _table(w.ops[lo:lo + count], a_ids), _table(w.ops[lo:lo + count], b_ids)
        assert h.hicr_memcpy_batch_noalloc(inst, ta.data_ptr(), count) == 0
        assert h.hicr_fence(inst, 0, T) == 0
        assert h.hicr_memcpy_batch_device(inst, tb.data_ptr(), count) == 0
        assert h.hicr_fence(inst, 0, T) == 0
        _same(h, inst, a_ids, b_ids)
        assert cm.memcpy_batch(w.ops[lo:lo + count]) == (om.OK, None)
        _matches_oracle(h, inst, a_ids, cm)
        s, r = h.hicr_slot_counters_range(inst, a_ids[0], len(a_ids))[1:]
        assert int(s.sum()) == int(r.sum()) > 0


def test_noalloc_at_the_op_limit(h, inst):
    """Exactly HICR_NOALLOC_MAX_OPS ops: the last words of the static array's
    regions (prefix sums, piece counters) are in use, and the single-CTA scan
    runs full per-thread runs. A bad op at the last index is reported with
    that index and copies nothing; the good table then equals the oracle."""
    n = h.HICR_NOALLOC_MAX_OPS
    w = configs.tiny(9, slot_bytes=2 << 20, n_ops=n, max_n=48)
    assert len(w.ops) == n
    ids = _slots(h, inst, w, 9)
    cm = _oracle(w, 9)
    bad = w.ops.copy()
    bad["n"][n - 1] = int(w.slot_sizes[bad["src"][n - 1]]) + 1
    tbad = _table(bad, ids)
    assert h.hicr_memcpy_batch_noalloc(inst, tbad.data_ptr(), n) == 0
    assert h.hicr_batch_error(inst) == (0, h.HICR_ERR_BOUNDS, n - 1)
    assert h.hicr_fence(inst, 0, T) == 0
    _matches_oracle(h, inst, ids, cm)  # nothing copied, counters untouched
    t = _table(w.ops, ids)
    for _ in range(2):
        assert h.hicr_memcpy_batch_noalloc(inst, t.data_ptr(), n) == 0
        assert h.hicr_fence(inst, 0, T) == 0
        assert cm.memcpy_batch(w.ops) == (om.OK, None)
        _matches_oracle(h, inst, ids, cm)


def test_noalloc_calls_leave_device_memory_untouched(h, inst):
    """The point of the entry point: after a first call, further calls (and
    the fences that complete them) do not change the device's free memory."""
    w = configs.batched(8, n_slots=4, total_bytes=32 << 20, slot_lo=4 << 20, slot_hi=16 << 20,
                        n_ops=3000, n_lo=16, n_hi=256 << 10)
    ids = _slots(h, inst, w, 8)
    lo, hi = w.epochs[0]
    t = _table(w.ops[lo:hi], ids)
    assert h.hicr_memcpy_batch_noalloc(inst, t.data_ptr(), hi - lo) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        assert h.hicr_memcpy_batch_noalloc(inst, t.data_ptr(), hi - lo) == 0
        assert h.hicr_fence(inst, 0, T) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversize_and_recovers_from_a_bad_batch(h, inst):
    w = configs.batched(6, n_slots=4, total_bytes=16 << 20, slot_lo=2 << 20, slot_hi=8 << 20,
                        n_ops=500, n_lo=16, n_hi=64 << 10)
    a_ids = _slots(h, inst, w, 6)
    b_ids = _slots(h, inst, w, 6)
    lo, hi = w.epochs[0]
    ta = _table(w.ops[lo:hi], a_ids)
    before = h.hicr_slot_counters_range(inst, a_ids[0], len(a_ids))
    assert h.hicr_memcpy_batch_noalloc(inst, ta.data_ptr(), h.HICR_NOALLOC_MAX_OPS + 1) == h.HICR_ERR_TOO_LARGE
    assert h.hicr_fence(inst, 0, T) == 0
    after = h.hicr_slot_counters_range(inst, a_ids[0], len(a_ids))
    assert (before[1] == after[1]).all() and (before[2] == after[2]).all()
    # an op past the end of its slot: the whole batch copies nothing, the
    # fence reports BOUNDS with the index, and the next call is unaffected
    bad = w.ops[lo:hi].copy()
    bad["n"][3] = int(w.slot_sizes[bad["src"][3]]) + 1
    tbad = _table(bad, a_ids)
    assert h.hicr_memcpy_batch_noalloc(inst, tbad.data_ptr(), hi - lo) == 0
    assert h.hicr_fence(inst, 0, T) == h.HICR_ERR_BOUNDS
    after_bad = h.hicr_slot_counters_range(inst, a_ids[0], len(a_ids))
    assert (after_bad[1] == after[1]).all() and (after_bad[2] == after[2]).all()
    _same(h, inst, a_ids, b_ids)
    tb = _table(w.ops[lo:hi], b_ids)
    assert h.hicr_memcpy_batch_noalloc(inst, ta.data_ptr(), hi - lo) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    assert h.hicr_memcpy_batch_device(inst, tb.data_ptr(), hi - lo) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    _same(h, inst, a_ids, b_ids)
