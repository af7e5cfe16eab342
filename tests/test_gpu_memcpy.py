"""GPU parity of memcpy / fence / counters against the oracle, through the C ABI.

Byte-exact comparison of every slot byte for cases the oracle finishes in
seconds; sampled positions plus op-boundary bytes at the full 16 GiB size.
"""
import numpy as np
import pytest
import torch

from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, fill_key, h, inst, slot_bytes  # noqa: F401

pytestmark = pytest.mark.gpu

T = 60_000_000_000  # fence timeout (ns)


def alloc_filled(h, inst, sizes, seed, tag=0):
    ids = []
    for s, sz in enumerate(sizes):
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, int(sz), tag)
        assert st == 0
        assert h.hicr_util_fill(inst, sid, 0, int(sz), fill_key(seed, s)) == 0
        ids.append(sid)
    return ids


def oracle_slots(sizes, seed):
    cm = om.CommManager()
    ids = [cm.register(om.SPACE_HBM, splitmix.fill_bytes(seed, s, 0, int(sz))) for s, sz in enumerate(sizes)]
    return cm, ids


def remap(ops, ids):
    """Rewrite workload slot indices into library slot handles."""
    o = ops.copy()
    m = np.asarray(ids, dtype=np.uint32)
    o["dst"] = m[ops["dst"]]
    o["src"] = m[ops["src"]]
    return o


def to_device(ops):
    return torch.from_numpy(ops.view(np.uint8).copy()).cuda()


def test_topology(h, inst):
    st, t = h.hicr_topology_query(inst)
    assert st == 0 and t.n_spaces == 2 and t.n_resources == 1
    assert t.spaces[0].kind == h.HICR_SPACE_HBM and t.spaces[0].phys_size > (100 << 30)
    # theoretical HBM bandwidth from clock x bus width: 0 (unknown) or a few TB/s
    assert t.spaces[0].peak_mbps == 0 or 1_000_000 < t.spaces[0].peak_mbps < 50_000_000
    assert t.spaces[1].peak_mbps == 0
    assert t.resources[0].sm_count > 0
    assert h.hicr_is_root(inst) == (0, 1)


def test_fill_matches_generator(h, inst):
    for off, n in [(0, 4096), (3, 1000), (8, 8), (1, 1)]:
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 8192)
        assert h.hicr_util_fill(inst, sid, off, n, fill_key(0, 7)) == 0
        got = slot_bytes(h, inst, sid)[off:off + n]
        assert (got == splitmix.fill_bytes(0, 7, off, n)).all()
        assert h.hicr_mem_free(inst, sid) == 0


def test_worked_example_through_the_abi(h, inst):
    from tests.test_oracle_memcpy import load_worked, STATUS
    slots, ops, final, counts = load_worked()
    ids = {}
    keep = []
    for name, b in slots.items():
        t = torch.tensor(list(b), dtype=torch.uint8, device="cuda")
        keep.append(t)
        st, sid = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, t.data_ptr(), t.numel())
        assert st == 0
        ids[name] = sid
    for d, doff, s, soff, n, exp in ops:
        st = h.hicr_memcpy(inst, ids.get(d, 999), doff, ids.get(s, 999), soff, n)
        assert st == STATUS[exp], (d, doff, s, soff, n)
    assert h.hicr_fence(inst, 0, T) == 0
    for name, b in final.items():
        assert bytes(slot_bytes(h, inst, ids[name])) == b
    for name, c in counts.items():
        assert h.hicr_slot_counters(inst, ids[name])[1:] == c
    assert h.hicr_tag_counter(inst, 0) == (0, 4)


def _corner_ops(size):
    """Ops over every (src mod 16, dst mod 16) residue pair for a list of
    sizes, with disjoint destination ranges (slot 1) and sources in slot 0."""
    ns = [0, 1, 2, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 129, 4095, 4096, 4097, 65535, 65537]
    rng = np.random.default_rng(5)
    dst, src, doff, soff, nn = [], [], [], [], []
    cursor = 0
    for n in ns:
        for rs in range(16):
            for rd in range(16):
                if n > 4096 and (rs, rd) not in [(0, 0), (1, 0), (0, 1), (7, 9), (15, 15), (4, 8), (8, 4), (12, 3)]:
                    continue
                s = 16 * int(rng.integers(0, (size - n - 16) // 16)) + rs
                d = ((cursor + 15) // 16) * 16 + rd
                cursor = d + n + int(rng.integers(0, 3))
                dst.append(1), src.append(0), doff.append(d), soff.append(s), nn.append(n)
    assert cursor <= size
    return configs.make_ops(dst, src, doff, soff, nn)


@pytest.mark.parametrize("path", ["batch", "device", "queue", "plain", "tma"])
def test_size_and_alignment_corners(h, inst, path):
    size = 8 << 20
    ops = _corner_ops(size)
    if path == "tma":  # the TMA engine with its smallest threshold: every co-aligned piece >= 1 KiB
        st, c = h.hicr_batch_get_config(inst)
        c.engine, c.tma_min_bytes, c.threads, c.blocks_per_sm, c.chunk_bytes = 1, 1024, 256, 1, 16 << 10
        assert h.hicr_batch_set_config(inst, c) == 0
        path = "device"
    ids = alloc_filled(h, inst, [size, size], 11)
    cm, oids = oracle_slots([size, size], 11)
    assert cm.memcpy_batch(ops) == (om.OK, None)
    dops = remap(ops, ids)
    if path == "batch":
        assert h.hicr_memcpy_batch(inst, dops) == (0, 0)
    elif path == "device":
        t = to_device(dops)
        assert h.hicr_memcpy_batch_device(inst, t.data_ptr(), len(dops)) == 0
    elif path == "queue":
        for o in dops:
            assert h.hicr_memcpy(inst, int(o["dst"]), int(o["dst_off"]), int(o["src"]), int(o["src_off"]),
                                 int(o["n"])) == 0
    else:
        assert h.hicr_memcpy_batch_plain(inst, dops) == (0, 0)
    assert h.hicr_fence(inst, 0, T) == 0
    for k in range(2):
        assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all()
    if path != "plain":
        assert h.hicr_slot_counters(inst, ids[0])[1:] == (len(ops), 0)
        assert h.hicr_slot_counters(inst, ids[1])[1:] == (0, len(ops))


@pytest.mark.parametrize("sizes", [
    [16],
    [0, 1, 17],
    [4099, 65536, 33, 262144, 5, 100_000, 2, 7],   # eight ops, one at the 256 KiB limit
    [4099, 65536, 33, 262145],                      # one op over the limit: the regular path
    [64] * 9,                                       # nine ops: the regular path
])
def test_small_batches_match_oracle(h, inst, sizes):
    """Host batches of at most 8 ops of at most 256 KiB travel as kernel
    parameters (one CTA per op, no op-table upload, no plan/scan); larger
    ones take the regular path. Both must leave the oracle's bytes and exact
    slot and tag counters, through single memcpys + fence and through
    hicr_memcpy_batch."""
    size = 4 << 20
    ids = []
    for s, tag in enumerate((3, 5)):
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size, tag)
        assert st == 0 and h.hicr_util_fill(inst, sid, 0, size, fill_key(23, s)) == 0
        ids.append(sid)
    cm, oids = oracle_slots([size, size], 23)
    rng = np.random.default_rng(len(sizes) * 31 + sum(sizes) % 97)
    c0 = [h.hicr_slot_counters(inst, i)[1:] for i in ids]
    t0 = [h.hicr_tag_counter(inst, t)[1] for t in (3, 5)]
    for rnd, path in enumerate(("queue", "batch")):
        cursor = rnd * (size // 2)
        dst, src, doff, soff = [], [], [], []
        for n in sizes:
            d = cursor + int(rng.integers(0, 16))
            cursor = d + n + 1
            dst.append(1), src.append(0), doff.append(d), soff.append(int(rng.integers(0, size - n)))
        assert cursor <= (rnd + 1) * (size // 2)
        ops = configs.make_ops(dst, src, doff, soff, sizes)
        assert cm.memcpy_batch(ops) == (om.OK, None)
        dops = remap(ops, ids)
        if path == "queue":
            for o in dops:
                assert h.hicr_memcpy(inst, int(o["dst"]), int(o["dst_off"]), int(o["src"]), int(o["src_off"]),
                                     int(o["n"])) == 0
        else:
            assert h.hicr_memcpy_batch(inst, dops) == (0, 0)
        assert h.hicr_fence(inst, 3, T) == 0  # every op touches tags 3 and 5
        for k in range(2):
            assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all(), (path, k)
        m = (rnd + 1) * len(sizes)
        assert h.hicr_slot_counters(inst, ids[0])[1:] == (c0[0][0] + m, c0[0][1])
        assert h.hicr_slot_counters(inst, ids[1])[1:] == (c0[1][0], c0[1][1] + m)
        assert [h.hicr_tag_counter(inst, t)[1] for t in (3, 5)] == [t0[0] + m, t0[1] + m]
    for i in ids:
        assert h.hicr_mem_free(inst, i) == 0


def test_tiny_config_bit_exact(h, inst):
    w = configs.tiny(0)
    ids = alloc_filled(h, inst, w.slot_sizes, 0)
    cm, oids = oracle_slots(w.slot_sizes, 0)
    assert cm.memcpy_batch(w.ops) == (om.OK, None)
    assert h.hicr_memcpy_batch(inst, remap(w.ops, ids)) == (0, 0)
    assert h.hicr_fence(inst, 0, T) == 0
    for k in range(2):
        assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all()
    assert h.hicr_slot_counters(inst, ids[0])[1:] == (1024, 0)
    assert h.hicr_slot_counters(inst, ids[1])[1:] == (0, 1024)
    assert h.hicr_tag_counter(inst, 0) == (0, 1024)
    assert h.hicr_fence_slot(inst, ids[1], 0, 1024, T) == 0
    assert h.hicr_fence_slot(inst, ids[1], 0, 1025, 2_000_000) == h.HICR_ERR_TIMEOUT


CONFIGS = [
    dict(chunk_bytes=1024, op_cost_bytes=1, blocks_per_sm=1, threads=64),
    dict(chunk_bytes=4096, op_cost_bytes=4096, blocks_per_sm=2, threads=256),
    dict(chunk_bytes=64 << 10, op_cost_bytes=2048, blocks_per_sm=2, threads=512),
    dict(chunk_bytes=1 << 20, op_cost_bytes=64, blocks_per_sm=1, threads=1024),
    # the TMA engine: small threshold (many short bodies, partial stages) and the tuned shapes
    dict(chunk_bytes=64 << 10, op_cost_bytes=4096, blocks_per_sm=1, threads=256, engine=1, tma_min_bytes=1024),
    dict(chunk_bytes=1 << 20, op_cost_bytes=64, blocks_per_sm=2, threads=192, engine=1, tma_min_bytes=32 << 10),
    dict(chunk_bytes=256 << 10, op_cost_bytes=4096, blocks_per_sm=1, threads=384, engine=1, tma_min_bytes=256 << 10),
    # other stage shapes: 8 stages of 4 KiB, 2 of 16 KiB
    dict(chunk_bytes=128 << 10, op_cost_bytes=4096, blocks_per_sm=1, threads=192, engine=1, tma_min_bytes=1024,
         tma_stages=8, tma_stage_bytes=4096),
    dict(chunk_bytes=256 << 10, op_cost_bytes=64, blocks_per_sm=1, threads=192, engine=1, tma_min_bytes=4096,
         tma_stages=2, tma_stage_bytes=16384),
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_batched_small_epochs_bit_exact(h, inst, cfg):
    w = configs.batched_small(0)
    st, c = h.hicr_batch_get_config(inst)
    for k, v in cfg.items():
        setattr(c, k, v)
    assert h.hicr_batch_set_config(inst, c) == 0
    ids = alloc_filled(h, inst, w.slot_sizes, 0)
    cm, oids = oracle_slots(w.slot_sizes, 0)
    dops = to_device(remap(w.ops, ids))
    for a, b in w.epochs:
        assert cm.memcpy_batch(w.ops[a:b]) == (om.OK, None)
        assert h.hicr_memcpy_batch_device(inst, dops.data_ptr() + 32 * a, b - a) == 0
        assert h.hicr_fence(inst, 0, T) == 0
    for k in range(len(ids)):
        assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all(), k
    sent, recv = om.counters_from_ops(w.ops, len(ids))
    for k in range(len(ids)):
        assert h.hicr_slot_counters(inst, ids[k])[1:] == (int(sent[k]), int(recv[k]))


def test_graph_replay_and_profile(h, inst):
    w = configs.batched_small(1)
    ids = alloc_filled(h, inst, w.slot_sizes, 1)
    cm, oids = oracle_slots(w.slot_sizes, 1)
    for a, b in w.epochs:
        cm.memcpy_batch(w.ops[a:b])
    dops = to_device(remap(w.ops, ids))
    assert h.hicr_batch_reserve(inst, len(w.ops)) == 0
    assert h.hicr_profile_enable(inst, 1) == 0
    assert h.hicr_graph_begin(inst) == 0
    for a, b in w.epochs:
        assert h.hicr_memcpy_batch_device(inst, dops.data_ptr() + 32 * a, b - a) == 0
    st, g = h.hicr_graph_end(inst)
    assert st == 0
    for rep in range(3):
        assert h.hicr_graph_launch(inst, g) == 0
        assert h.hicr_fence(inst, 0, T) == 0
        st, ms, n = h.hicr_profile_read(inst)
        assert st == 0 and n == len(w.epochs) and ms > 0
    # sources are never written, so replays reproduce the single application
    for k in range(len(ids)):
        assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all(), k
    sent, recv = om.counters_from_ops(w.ops, len(ids))
    for k in range(len(ids)):
        assert h.hicr_slot_counters(inst, ids[k])[1:] == (3 * int(sent[k]), 3 * int(recv[k]))
    assert h.hicr_graph_destroy(inst, g) == 0


def test_device_validation_rejects_whole_batch(h, inst):
    size = 1 << 20
    ids = alloc_filled(h, inst, [size, size], 2)
    before = [slot_bytes(h, inst, i) for i in ids]
    good = configs.make_ops([ids[1]] * 3, [ids[0]] * 3, [0, 100, 200], [0, 0, 0], [10, 10, 10])
    cases = [
        (1, dict(n=size), h.HICR_ERR_BOUNDS),
        (2, dict(dst=999), h.HICR_ERR_INVALID),
        (0, dict(dst=ids[0], dst_off=5), h.HICR_ERR_OVERLAP),
        (1, dict(src_off=(1 << 64) - 1), h.HICR_ERR_BOUNDS),
    ]
    for idx, patch, code in cases:
        ops = good.copy()
        for k, v in patch.items():
            ops[k][idx] = v
        t = to_device(ops)
        assert h.hicr_memcpy_batch_device(inst, t.data_ptr(), len(ops)) == 0
        assert h.hicr_fence(inst, 0, T) == code
        assert h.hicr_batch_error(inst) == (0, 0, 0)  # cleared by the fence
        st, bad = h.hicr_memcpy_batch(inst, ops)
        assert (st, bad) == (code, idx)
    for i, b in zip(ids, before):
        assert (slot_bytes(h, inst, i) == b).all()
        assert h.hicr_slot_counters(inst, i)[1:] == (0, 0)


def test_host_validation_matches_oracle(h, inst):
    rng = np.random.default_rng(9)
    sizes = [64, 100, 1 << 12]
    ids = alloc_filled(h, inst, sizes, 3)
    cm, oids = oracle_slots(sizes, 3)
    st, hs = h.hicr_mem_alloc(inst, h.HICR_SPACE_HOST, 64)
    assert st == 0
    ho = cm.register(om.SPACE_HOST, np.zeros(64, dtype=np.uint8))
    lib_ids = ids + [hs]
    or_ids = oids + [ho]
    for _ in range(3000):
        d, s = int(rng.integers(0, 5)), int(rng.integers(0, 5))
        n = int(rng.choice([0, 1, 5, 30, 64, 100, 5000]))
        doff, soff = int(rng.integers(0, 120)), int(rng.integers(0, 120))
        exp = cm.validate(or_ids[d] if d < 4 else 77, doff, or_ids[s] if s < 4 else 77, soff, n)
        got = h.hicr_memcpy(inst, lib_ids[d] if d < 4 else 4000, doff, lib_ids[s] if s < 4 else 4000, soff, n)
        assert got == exp, (d, doff, s, soff, n)
        if exp == om.OK:
            cm._apply(or_ids[d], doff, or_ids[s], soff, n)
            assert h.hicr_fence(inst, 0, T) == 0  # keep ops of an epoch hazard-free
    for k in range(3):
        assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all()
        assert h.hicr_slot_counters(inst, ids[k])[1:] == cm.counters(oids[k])


def test_checked_mode_hazard_index_matches_oracle(h, inst):
    rng = np.random.default_rng(4)
    ids = alloc_filled(h, inst, [256, 256], 4)
    assert h.hicr_set_checked(inst, 1) == 0
    seen = 0
    for _ in range(400):
        k = int(rng.integers(2, 7))
        ops = configs.make_ops(rng.integers(0, 2, k), rng.integers(0, 2, k), rng.integers(0, 200, k),
                               rng.integers(0, 200, k), rng.integers(0, 40, k))
        ok = all(om.CommManager.validate(_two_slot_cm(), int(o["dst"]), int(o["dst_off"]), int(o["src"]),
                                         int(o["src_off"]), int(o["n"])) == om.OK for o in ops)
        if not ok:
            continue
        exp = om.first_hazard(ops)
        st, bad = h.hicr_memcpy_batch(inst, remap(ops, ids))
        if exp is None:
            assert st == 0
            assert h.hicr_fence(inst, 0, T) == 0
        else:
            seen += 1
            assert (st, bad) == (h.HICR_ERR_HAZARD, exp)
    assert seen > 50


def _two_slot_cm():
    cm = om.CommManager()
    cm.register(om.SPACE_HBM, np.zeros(256, dtype=np.uint8))
    cm.register(om.SPACE_HBM, np.zeros(256, dtype=np.uint8))
    return cm


def test_registered_torch_tensors_and_deregister(h, inst):
    a = torch.arange(4096, device="cuda", dtype=torch.int32).view(torch.uint8)
    b = torch.zeros(16384, device="cuda", dtype=torch.uint8)
    st, sa = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, a.data_ptr(), a.numel(), 3)
    st2, sb = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, b.data_ptr(), b.numel(), 5)
    assert st == 0 and st2 == 0
    assert h.hicr_memcpy(inst, sb, 7, sa, 3, 10000) == 0
    assert h.hicr_fence(inst, 5, T) == 0
    exp = np.zeros(16384, dtype=np.uint8)
    exp[7:10007] = a.cpu().numpy()[3:10003]
    assert (b.cpu().numpy() == exp).all()
    assert h.hicr_tag_counter(inst, 3) == (0, 1) and h.hicr_tag_counter(inst, 5) == (0, 1)
    assert h.hicr_slot_deregister(inst, sa) == 0
    assert h.hicr_memcpy(inst, sb, 0, sa, 0, 1) == h.HICR_ERR_INVALID
    assert h.hicr_mem_free(inst, sb) == h.HICR_ERR_INVALID  # registered, not allocated


def test_exec_units_fill_and_digest(h, inst):
    from oracle import digest as od
    st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 1 << 20)
    st, ptr, size, _, _ = h.hicr_slot_info(inst, sid)
    st, unit = h.hicr_exec_unit_builtin("fill_seeded")
    assert st == 0 and unit.n_args == 4
    import ctypes as C
    args = [C.c_void_p(ptr), C.c_uint64(0), C.c_uint64(size), C.c_uint64(fill_key(0, 3))]
    st, pu = h.hicr_pu_create(inst)
    st, e = h.hicr_exec_launch(inst, pu, unit, args)
    assert st == 0
    assert h.hicr_exec_await(inst, e, T) == 0
    assert h.hicr_exec_await(inst, e, T) == h.HICR_ERR_INVALID  # finished states are released
    assert (slot_bytes(h, inst, sid) == splitmix.fill_bytes(0, 3, 0, size)).all()
    for off, n in [(0, size), (5, 1001), (8, 0)]:
        st, dg = h.hicr_util_digest(inst, sid, off, n)
        assert st == 0 and dg == od.byte_digest(splitmix.fill_bytes(0, 3, off, n))
    assert h.hicr_pu_destroy(inst, pu) == 0
    assert h.hicr_exec_unit_builtin("nope")[0] == h.HICR_ERR_INVALID


def test_torch_stream_as_processing_unit(h, inst):
    s = torch.cuda.Stream()
    st, pu = h.hicr_pu_create(inst, s.cuda_stream)
    assert st == 0 and h.hicr_pu_stream(inst, pu) == (0, s.cuda_stream)
    ids = alloc_filled(h, inst, [1 << 20, 1 << 20], 6)
    assert h.hicr_comm_set_pu(inst, pu) == 0
    assert h.hicr_memcpy(inst, ids[1], 0, ids[0], 0, 1 << 20) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    assert (slot_bytes(h, inst, ids[1]) == splitmix.fill_bytes(6, 0, 0, 1 << 20)).all()
    assert h.hicr_comm_set_pu(inst, 0) == 0
    assert h.hicr_pu_destroy(inst, pu) == 0


def test_bounded_device_wait_gives_up(h, inst):
    """Every spin in the library ends at a %globaltimer deadline: a wait on a
    flag that nothing sets must return TIMEOUT after about the set time."""
    st, status, waited = h.hicr_util_wait_test(inst, 200_000_000)
    assert st == 0 and status == h.HICR_ERR_TIMEOUT
    assert 200_000_000 <= waited < 2_000_000_000


def test_autotune_cache_round_trip(h, inst, tmp_path, monkeypatch):
    """With HICR_TUNE_CACHE set, the first autotune appends its winner to the
    file; a later autotune of a table with the same key installs the cached
    configuration without trials."""
    import json
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("HICR_TUNE_CACHE", str(path))
    w = configs.batched_small(2)
    ids = alloc_filled(h, inst, w.slot_sizes, 2)
    a, b = w.epochs[0]
    dops = to_device(remap(w.ops[a:b], ids))
    st, c1, ms1 = h.hicr_batch_autotune(inst, dops.data_ptr(), b - a, 2)
    assert st == 0
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["engine"] == c1.engine and rec["chunk_bytes"] == c1.chunk_bytes and rec["ops_log2"] >= 0
    other = h.hicr_batch_get_config(inst)[1]
    other.engine, other.chunk_bytes, other.threads, other.blocks_per_sm = 0, 4096, 64, 1
    assert h.hicr_batch_set_config(inst, other) == 0
    st, c2, ms2 = h.hicr_batch_autotune(inst, dops.data_ptr(), b - a, 2)
    assert st == 0 and c2.as_dict() == c1.as_dict() and abs(ms2 - ms1) < 1e-3 * max(ms1, 1.0)
    assert h.hicr_batch_get_config(inst)[1].as_dict() == c1.as_dict()
    assert len(path.read_text().splitlines()) == 1


@pytest.mark.parametrize("n_ops,bad_at", [(20_000, 19_999), (20_000, 0), (50_000, 31_337), (8_192, 4_096)])
def test_large_host_batch_reports_the_first_invalid_op(h, inst, n_ops, bad_at):
    """Host tables of 8,192 ops or more are validated by several host
    threads; the reported op is still the first invalid one in issue order,
    nothing of the batch runs, and the same table without the bad ops runs
    exactly as the oracle says."""
    size = 1 << 20
    ids = alloc_filled(h, inst, [size, size], 4)
    cm, oids = oracle_slots([size, size], 4)
    rng = np.random.default_rng(n_ops + bad_at)
    n = rng.integers(0, 16, n_ops)
    doff = np.arange(n_ops, dtype=np.uint64) * np.uint64(16)  # disjoint destinations
    soff = rng.integers(0, size - 16, n_ops)
    ops = configs.make_ops([1] * n_ops, [0] * n_ops, doff, soff, n)
    bad = ops.copy()
    bad["n"][bad_at] = size + 1                       # out of bounds
    bad["n"][min(bad_at + 7, n_ops - 1)] = size + 1   # a later one is not the one reported
    st, first = h.hicr_memcpy_batch(inst, remap(bad, ids))
    assert (st, first) == (h.HICR_ERR_BOUNDS, bad_at)
    assert cm.memcpy_batch(bad) == (om.ERR_BOUNDS, bad_at)
    assert h.hicr_fence(inst, 0, T) == 0
    assert h.hicr_slot_counters(inst, ids[1])[1:] == (0, 0)   # the rejected batch did nothing
    assert h.hicr_memcpy_batch(inst, remap(ops, ids)) == (0, 0)
    assert cm.memcpy_batch(ops) == (om.OK, None)
    assert h.hicr_fence(inst, 0, T) == 0
    for k in range(2):
        assert (slot_bytes(h, inst, ids[k]) == cm.slots[oids[k]].data).all()
    assert h.hicr_slot_counters(inst, ids[1])[1:] == (0, n_ops)
