"""Stress parity of the batched copy: random op tables, 100 seeds.

Each seed draws a small batched workload (slot count, sizes, op count and op
size range vary with the seed; hazard-free fence epochs, 10% relatively
misaligned offsets) and a random copy configuration (either engine, chunk
size, CTA shape, per-op charge, TMA threshold). The slots are carved out of one
allocation with guard bands between them, so a write outside a slot would
land in a guard. After all epochs every slot byte equals the oracle's, every
guard byte is untouched and the counters are exact. Plus the seeded fill
against the generator on 10^6 random positions of a 256 MiB slot."""
import numpy as np
import pytest
import torch

from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, fill_key, h, inst  # noqa: F401

pytestmark = pytest.mark.gpu

T = 30_000_000_000
GUARD = 4096
GUARD_KEY = splitmix.fill_key_base(255, 4095)


def _random_workload(seed):
    rng = np.random.default_rng(1000 + seed)
    n_slots = int(rng.integers(4, 17))
    total = n_slots * int(rng.integers(512, 2049)) << 10
    n_hi = int(rng.choice([4 << 10, 64 << 10, 256 << 10]))  # every slot (>= 256 KiB) holds any op
    w = configs.batched(seed, n_slots=n_slots, total_bytes=total, slot_lo=256 << 10, slot_hi=8 << 20,
                        n_ops=int(rng.integers(50, 1500)), n_lo=1, n_hi=n_hi, max_gap=256,
                        name=f"stress{seed}")
    return w, rng


def _random_config(h, inst, rng):
    st, c = h.hicr_batch_get_config(inst)
    if rng.random() < 0.5:
        c.engine = 1
        # (threads, CTAs per SM, stages, stage bytes): shapes whose stages fit in shared memory
        c.threads, c.blocks_per_sm, c.tma_stages, c.tma_stage_bytes = [
            (256, 1, 4, 4096), (384, 1, 4, 4096), (192, 2, 4, 4096), (64, 1, 4, 4096), (192, 1, 8, 4096),
            (192, 1, 2, 16384), (512, 1, 2, 4096), (256, 2, 2, 4096), (256, 1, 2, 8192)][int(rng.integers(0, 9))]
        c.tma_min_bytes = int(rng.choice([1024, 4096, 32 << 10]))
    else:
        c.engine = 0
        c.threads, c.blocks_per_sm = [(64, 1), (256, 4), (512, 2), (1024, 1)][int(rng.integers(0, 4))]
    c.chunk_bytes = int(rng.choice([1024, 16 << 10, 128 << 10, 1 << 20]))
    c.op_cost_bytes = int(rng.choice([1, 64, 4096]))
    assert h.hicr_batch_set_config(inst, c) == 0
    return c


@pytest.mark.parametrize("seed", range(100))
def test_random_tables_with_guards(h, inst, seed):
    w, rng = _random_workload(seed)
    cfg = _random_config(h, inst, rng)
    sizes = [int(x) for x in w.slot_sizes]
    # one allocation: guard, slot 0, guard, slot 1, ..., guard (slot starts keep
    # the 16-byte alignment the workload assumes)
    offs, pos = [], GUARD
    for sz in sizes:
        offs.append(pos)
        pos += (sz + 15) // 16 * 16 + GUARD
    st, big = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, pos)
    assert st == 0
    assert h.hicr_util_fill(inst, big, 0, pos, GUARD_KEY) == 0
    st, base, _, _, _ = h.hicr_slot_info(inst, big)
    ids = []
    for k, (o, sz) in enumerate(zip(offs, sizes)):
        st, sid = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, base + o, sz)
        assert st == 0
        assert h.hicr_util_fill(inst, sid, 0, sz, fill_key(seed, k)) == 0
        ids.append(sid)
    cm = om.CommManager()
    oids = [cm.register(om.SPACE_HBM, splitmix.fill_bytes(seed, k, 0, sz)) for k, sz in enumerate(sizes)]
    lops = w.ops.copy()
    lops["dst"] = np.asarray(ids, dtype=np.uint32)[w.ops["dst"]]
    lops["src"] = np.asarray(ids, dtype=np.uint32)[w.ops["src"]]
    d = torch.from_numpy(lops.view(np.uint8).copy()).cuda()
    for a, b in w.epochs:
        assert cm.memcpy_batch(w.ops[a:b]) == (om.OK, None)
        assert h.hicr_memcpy_batch_device(inst, d.data_ptr() + 32 * a, b - a) == 0
        assert h.hicr_fence(inst, 0, T) == 0
    torch.cuda.synchronize()
    everything = device_bytes(base, pos).cpu().numpy()
    guard_ref = splitmix.fill_bytes(255, 4095, 0, pos)
    mask = np.ones(pos, dtype=bool)
    for k, (o, sz) in enumerate(zip(offs, sizes)):
        got = everything[o:o + sz]
        assert (got == cm.slots[oids[k]].data).all(), (seed, k, cfg.as_dict())
        mask[o:o + sz] = False
    assert (everything[mask] == guard_ref[mask]).all(), (seed, "guard bytes changed", cfg.as_dict())
    sent, recv = om.counters_from_ops(w.ops, len(ids))
    for k, sid in enumerate(ids):
        assert h.hicr_slot_counters(inst, sid)[1:] == (int(sent[k]), int(recv[k]))
    for sid in ids:
        assert h.hicr_slot_deregister(inst, sid) == 0
    assert h.hicr_mem_free(inst, big) == 0


def test_fill_matches_generator_on_a_million_positions(h, inst):
    size = 256 << 20
    st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size)
    assert st == 0
    assert h.hicr_util_fill(inst, sid, 0, size, fill_key(3, 77)) == 0
    st, ptr, _, _, _ = h.hicr_slot_info(inst, sid)
    pos = np.random.default_rng(4).integers(0, size, 1_000_000)
    torch.cuda.synchronize()
    got = device_bytes(ptr, size)[torch.from_numpy(pos).cuda()].cpu().numpy()
    assert (got == splitmix.fill_byte_at(3, 77, pos)).all()
    assert h.hicr_mem_free(inst, sid) == 0
