"""fence(tag) and fence_slot against the memcpy oracle (HiCR paper Sec. 3.1.4).

fence(tag) waits for every op issued before it that touches a slot of that
tag, and only for those: each memcpy launch ends with a completion signal the
device writes into mapped host memory, and the fence polls for the signal of
the last launch that holds an op of its tag. A fence on one tag therefore
returns while a long batch of another tag, issued after it, still runs. The
counters after the fences are exact against the oracle; fences after other
work on the communication stream (fills) still cover it; fence_slot waits
for the expected counts and reports TIMEOUT when issued work cannot reach
them; a failed device batch is reported once by the next fence of any tag.
"""
import json
import os
import subprocess
import time

import numpy as np
import pytest
import torch

from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, h, inst, slot_bytes  # noqa: F401

pytestmark = pytest.mark.gpu

T = 60_000_000_000
GiB = 1 << 30


def test_fence_on_one_tag_returns_while_another_tag_runs(h, inst):
    # tag 1: a small copy issued first; tag 2: 5 batches of 8 GiB issued after it
    st, a_src = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 1 << 20, 1)
    st2, a_dst = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 1 << 20, 1)
    st3, b_src = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 256 << 20, 2)
    st4, b_dst = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 8 * GiB, 2)
    assert (st, st2, st3, st4) == (0, 0, 0, 0)
    assert h.hicr_util_fill(inst, a_src, 0, 1 << 20, splitmix.fill_key_base(1, 0)) == 0
    assert h.hicr_util_fill(inst, b_src, 0, 256 << 20, splitmix.fill_key_base(1, 1)) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    big = configs.make_ops([b_dst] * 32, [b_src] * 32, np.arange(32, dtype=np.uint64) * (256 << 20),
                           [0] * 32, [256 << 20] * 32)
    # warm-up of both paths
    assert h.hicr_memcpy(inst, a_dst, 0, a_src, 0, 4096) == 0
    assert h.hicr_memcpy_batch(inst, big) == (0, 0)
    assert h.hicr_fence(inst, 2, T) == 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert h.hicr_memcpy(inst, a_dst, 4096, a_src, 4096, 65536) == 0
    assert h.hicr_flush(inst) == 0
    for _ in range(5):
        assert h.hicr_memcpy_batch(inst, big) == (0, 0)
    t_issue = time.perf_counter()
    assert h.hicr_fence(inst, 1, T) == 0
    t_a = time.perf_counter()
    # tag 2 has about 80 GB of copies behind the tag-1 op: still running now
    assert h.hicr_fence(inst, 2, 0) == h.HICR_ERR_TIMEOUT
    assert h.hicr_fence(inst, 2, T) == 0
    t_b = time.perf_counter()
    print(f"issue {1e3 * (t_issue - t0):.2f} ms, fence(1) {1e3 * (t_a - t_issue):.3f} ms, "
          f"fence(2) {1e3 * (t_b - t_a):.2f} ms", flush=True)
    assert t_b - t_a > 5 * (t_a - t_issue)
    # bytes and counters against the oracle
    cm = om.CommManager()
    oa = cm.register(om.SPACE_HBM, splitmix.fill_bytes(1, 0, 0, 1 << 20), 1)
    od_ = cm.register(om.SPACE_HBM, np.zeros(1 << 20, dtype=np.uint8), 1)
    assert cm.memcpy(od_, 0, oa, 0, 4096) == om.OK
    assert cm.memcpy(od_, 4096, oa, 4096, 65536) == om.OK
    got = slot_bytes(h, inst, a_dst)
    assert (got[:4096 + 65536] == cm.slots[od_].data[:4096 + 65536]).all()
    assert h.hicr_slot_counters(inst, a_src)[1:] == (2, 0)
    assert h.hicr_slot_counters(inst, a_dst)[1:] == (0, 2)
    assert h.hicr_slot_counters(inst, b_src)[1:] == (6 * 32, 0)
    assert h.hicr_slot_counters(inst, b_dst)[1:] == (0, 6 * 32)
    assert h.hicr_tag_counter(inst, 1) == (0, 2) and h.hicr_tag_counter(inst, 2) == (0, 6 * 32)
    pos = np.arange(0, 8 * GiB, 1 << 24, dtype=np.int64) + 12345
    exp = splitmix.fill_byte_at(1, 1, pos % (256 << 20))
    st, ptr, size, _, _ = h.hicr_slot_info(inst, b_dst)
    got = device_bytes(ptr, size)[torch.from_numpy(pos).cuda()].cpu().numpy()
    assert (got == exp).all()
    for s in (a_src, a_dst, b_src, b_dst):
        assert h.hicr_mem_free(inst, s) == 0


def test_fences_per_tag_match_the_oracle(h, inst):
    """Three tags, slots of mixed tags, host batches, single memcpys and a
    device batch (whose tags the host does not read) interleaved with fences
    on each tag: after every fence the slots of that tag hold the oracle's
    bytes and counters (read without any device-wide synchronisation), and at
    the end every slot and tag counter equals the oracle's."""
    rng = np.random.default_rng(5)
    tags = [0, 1, 1, 2, 2, 0]
    size = 1 << 20
    ids = []
    cm = om.CommManager()
    for s, tg in enumerate(tags):
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size, tg)
        assert st == 0 and h.hicr_util_fill(inst, sid, 0, size, splitmix.fill_key_base(2, s)) == 0
        ids.append(sid)
        cm.register(om.SPACE_HBM, splitmix.fill_bytes(2, s, 0, size), tg)
    for rnd in range(12):
        n_ops = int(rng.integers(1, 40))
        cursor = {}
        dst, src, doff, soff, n = [], [], [], [], []
        for _ in range(n_ops):
            d, s_ = rng.choice(len(tags), 2, replace=False)
            k = int(rng.integers(0, 20000))
            c = cursor.get(int(d), 0)
            if c + k > size // 2:
                continue
            dst.append(int(d)), src.append(int(s_)), doff.append(c), soff.append(size // 2 + int(rng.integers(0, size // 2 - k)))
            n.append(k)
            cursor[int(d)] = c + k + int(rng.integers(0, 64))
        if not n:
            continue
        ops = configs.make_ops(dst, src, doff, soff, n)
        assert cm.memcpy_batch(ops) == (om.OK, None)
        g = ops.copy()
        g["dst"] = np.asarray(ids, dtype=np.uint32)[ops["dst"]]
        g["src"] = np.asarray(ids, dtype=np.uint32)[ops["src"]]
        how = rnd % 3
        if how == 0:
            assert h.hicr_memcpy_batch(inst, g) == (0, 0)
        elif how == 1:
            for o in g:
                assert h.hicr_memcpy(inst, int(o["dst"]), int(o["dst_off"]), int(o["src"]), int(o["src_off"]),
                                     int(o["n"])) == 0
        else:
            d = torch.from_numpy(g.view(np.uint8).copy()).cuda()
            assert h.hicr_memcpy_batch_device(inst, d.data_ptr(), len(g)) == 0
        tag = int(rng.integers(0, 3))
        assert h.hicr_fence(inst, tag, T) == 0
        # every op touching a slot of this tag is an op of this tag: the slot
        # is final now. Read it on torch's stream, which is not ordered after
        # the communication stream, so only the fence makes the bytes final.
        for k, sid in enumerate(ids):
            if tags[k] != tag:
                continue
            st, ptr, sz, _, _ = h.hicr_slot_info(inst, sid)
            assert (device_bytes(ptr, sz).cpu().numpy() == cm.slots[k].data).all(), (rnd, k)
            assert h.hicr_slot_counters(inst, sid)[1:] == cm.counters(k), (rnd, k)
    for tg in range(3):
        assert h.hicr_fence(inst, tg, T) == 0
        assert h.hicr_tag_counter(inst, tg) == (0, cm.tag_ops.get(tg, 0))
    for k, sid in enumerate(ids):
        assert (slot_bytes(h, inst, sid) == cm.slots[k].data).all(), k
        assert h.hicr_slot_counters(inst, sid)[1:] == cm.counters(k), k


def test_fence_slot_and_errors(h, inst):
    size = 1 << 20
    st, a = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size, 4)
    st2, b = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size, 4)
    assert st == 0 and st2 == 0
    for i in range(10):
        assert h.hicr_memcpy(inst, b, 100 * i, a, 0, 64) == 0
    assert h.hicr_fence_slot(inst, b, 0, 10, T) == 0
    assert h.hicr_fence_slot(inst, a, 10, 0, T) == 0
    t0 = time.perf_counter()
    assert h.hicr_fence_slot(inst, b, 0, 11, T) == h.HICR_ERR_TIMEOUT  # no issued op can reach 11
    assert time.perf_counter() - t0 < 5.0
    # a device batch with a bad op: the next fence of any tag reports it once
    bad = configs.make_ops([b], [a], [0], [size - 8], [16])
    d = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    assert h.hicr_memcpy_batch_device(inst, d.data_ptr(), 1) == 0
    assert h.hicr_fence(inst, 7, T) == h.HICR_ERR_BOUNDS
    assert h.hicr_fence(inst, 4, T) == 0
    assert h.hicr_slot_counters(inst, b)[1:] == (0, 10)
    # a fill (other work on the communication stream) followed by a fence of
    # an unrelated tag: the fence still covers it
    assert h.hicr_util_fill(inst, a, 0, size, splitmix.fill_key_base(4, 0)) == 0
    assert h.hicr_fence(inst, 9, T) == 0
    assert (slot_bytes(h, inst, a) == splitmix.fill_bytes(4, 0, 0, size)).all()


def test_c_latency_harness(h, inst):
    """The C harness times small synchronous operations through the C ABI
    only; it must run to the end and print every case."""
    from paper_2509_01425_gb300 import build
    exe = build.LATENCY_BIN
    assert os.path.exists(exe)
    r = subprocess.run([exe, "0", "200"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout)
    print(d, flush=True)
    for k in ("memcpy16_fence", "fence_idle", "exec_await", "spsc_push_pop", "dobj_get_fence",
              "memcpy16_fence_latency_mode", "dobj_get_fence_latency_mode", "spsc_push_pop_latency_mode"):
        assert 0 < d[k]["p50_us"] <= d[k]["p99_us"] <= d[k]["max_us"]


@pytest.mark.parametrize("idle_us", [50, 5000])
def test_latency_mode_matches_the_oracle(h, inst, idle_us):
    """Latency mode: small host batches go to the persistent server (which
    ends after idle_us without work, so the short window also exercises its
    relaunch), large ones to the stream; fences on each tag, slot
    deregistration and freeing interleave with them. Bytes (read without
    device-wide synchronisation) and counters equal the oracle's after every
    fence; at the end the mode is turned off and everything still matches.
    The server runs beside the stream, so the program respects the model's
    rule that ops not separated by a fence of their tag are unordered: no
    destination byte is written twice between two fences on all tags."""
    rng = np.random.default_rng(idle_us)
    assert h.hicr_set_latency_mode(inst, idle_us) == 0
    tags = [0, 1, 2, 0, 1, 2]
    size = 4 << 20
    ids = []
    cm = om.CommManager()
    for s_, tg in enumerate(tags):
        st, sid = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size, tg)
        assert st == 0 and h.hicr_util_fill(inst, sid, 0, size, splitmix.fill_key_base(6, s_)) == 0
        ids.append(sid)
        cm.register(om.SPACE_HBM, splitmix.fill_bytes(6, s_, 0, size), tg)
    cursor = {}  # per slot: destination bytes below it were written since the last fence on all tags
    for rnd in range(60):
        big = rnd % 7 == 3
        n_ops = int(rng.integers(9, 30)) if big else int(rng.integers(1, 9))
        if max(cursor.values(), default=0) > size // 4:
            for tg in range(3):
                assert h.hicr_fence(inst, tg, T) == 0
            cursor = {}
        dst, src, doff, soff, n = [], [], [], [], []
        for _ in range(n_ops):
            d, s_ = rng.choice(len(tags), 2, replace=False)
            k = int(rng.integers(0, 300_000 if big else 70_000))
            c = cursor.get(int(d), 0)
            if c + k > size // 2:
                continue
            dst.append(int(d)), src.append(int(s_)), doff.append(c), n.append(k)
            soff.append(size // 2 + int(rng.integers(0, size // 2 - k)))
            cursor[int(d)] = c + k + int(rng.integers(0, 64))
        if not n:
            continue
        ops = configs.make_ops(dst, src, doff, soff, n)
        assert cm.memcpy_batch(ops) == (om.OK, None)
        g = ops.copy()
        g["dst"] = np.asarray(ids, dtype=np.uint32)[ops["dst"]]
        g["src"] = np.asarray(ids, dtype=np.uint32)[ops["src"]]
        if rnd % 2:
            assert h.hicr_memcpy_batch(inst, g) == (0, 0)
        else:
            for o in g:
                assert h.hicr_memcpy(inst, int(o["dst"]), int(o["dst_off"]), int(o["src"]), int(o["src_off"]),
                                     int(o["n"])) == 0
        if rnd % 3 == 0:
            time.sleep(0.002)  # sometimes longer than the idle window: the server ends and restarts
        tag = int(rng.integers(0, 3))
        assert h.hicr_fence(inst, tag, T) == 0
        for k, sid in enumerate(ids):
            if tags[k] != tag:
                continue
            st, ptr, sz, _, _ = h.hicr_slot_info(inst, sid)
            assert (device_bytes(ptr, sz).cpu().numpy() == cm.slots[k].data).all(), (rnd, k)
            assert h.hicr_slot_counters(inst, sid)[1:] == cm.counters(k), (rnd, k)
    for tg in range(3):
        assert h.hicr_fence(inst, tg, T) == 0
        assert h.hicr_tag_counter(inst, tg) == (0, cm.tag_ops.get(tg, 0))
    # a registered slot leaves only when the server has finished with it
    t = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    st, r = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, t.data_ptr(), 4096, 0)
    ro = cm.register(om.SPACE_HBM, np.zeros(4096, dtype=np.uint8), 0)
    assert cm.memcpy(ro, 0, 0, 0, 4096) == om.OK
    assert st == 0 and h.hicr_memcpy(inst, r, 0, ids[0], 0, 4096) == 0 and h.hicr_flush(inst) == 0
    assert h.hicr_fence(inst, 0, T) == 0 and h.hicr_slot_deregister(inst, r) == 0
    assert (t.cpu().numpy() == cm.slots[ro].data).all()
    assert h.hicr_set_latency_mode(inst, 0) == 0
    for k, sid in enumerate(ids):
        assert (slot_bytes(h, inst, sid) == cm.slots[k].data).all(), k
        assert h.hicr_slot_counters(inst, sid)[1:] == cm.counters(k), k
        assert h.hicr_mem_free(inst, sid) == 0
    assert h.hicr_set_latency_mode(inst, 2_000_000) == h.HICR_ERR_INVALID


def test_latency_mode_beside_cooperative_runs(h, inst):
    """A live latency-mode server does not get in the way of this library's
    cooperative runs (they end it first): small copies, then an SPSC stream
    and a ping-pong, then more small copies, all correct."""
    size = 1 << 20
    st, a = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size)
    st2, b = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size)
    assert st == 0 and st2 == 0
    assert h.hicr_util_fill(inst, a, 0, size, splitmix.fill_key_base(8, 0)) == 0
    assert h.hicr_set_latency_mode(inst, 1_000_000) == 0  # a server that would stay for a second
    for i in range(4):
        assert h.hicr_memcpy(inst, b, 4096 * i, a, 4096 * i, 4096) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    chans = [h.hicr_spsc_create(inst, 64, 256)[1] for _ in range(sms // 2)]  # a CTA on every SM
    st, res = h.hicr_spsc_stream(inst, chans, 2000, 64)
    assert st == 0 and all(r.popped == 2000 and r.mismatches == 0 for r in res)
    st, r = h.hicr_pingpong(inst, a, 0, 1 << 16, 10, 2, 152)
    assert st == 0 and r.status == 0
    for i in range(4, 8):
        assert h.hicr_memcpy(inst, b, 4096 * i, a, 4096 * i, 4096) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    assert (slot_bytes(h, inst, b)[:8 * 4096] == splitmix.fill_bytes(8, 0, 0, 8 * 4096)).all()
    assert h.hicr_slot_counters(inst, b)[1:] == (0, 8)
    assert h.hicr_set_latency_mode(inst, 0) == 0
    for c in chans:
        assert h.hicr_channel_destroy(inst, c) == 0