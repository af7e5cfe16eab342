"""Serving loop: every request's result is the same alone and in the mix.

A request is a memcpy batch into its own destination region or an MPSC burst
drained by a channel consumer. Its result digest (memcpy: ordered combination
of the word digests of its ops' destination bytes; burst: ordered combination
of the consumed messages' digests) must be bit-identical when the requests
run one at a time and when they arrive together and overlap on the device,
and both must equal the digest the oracle computes from the seeded sources.
In the mix, every request's delivered bytes are also compared with the
oracle's byte by byte: each memcpy request's destination region (kept after
the run and read from the arena) against the memcpy oracle applying the
template's ops, and every burst message as the consumer took it from the
channel (the capture form) against the channel oracle's delivery.
"""
import numpy as np
import pytest
import torch

import bench
from oracle import channels as oc
from oracle import digest as od
from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, h, inst  # noqa: F401

pytestmark = pytest.mark.gpu

SEED = 3
T = 30_000_000_000


def small_setup(h, inst, verify=True, budget=512 << 20, ring_bytes=8 << 20):
    src_w = configs.batched(SEED, n_slots=8, total_bytes=64 << 20, slot_lo=1 << 20, slot_hi=16 << 20, n_ops=50,
                            n_hi=64 << 10)
    tmpl = configs.serve_templates(SEED, src_w, n_templates=16, max_ops=48, max_msgs=24, n_hi=256 << 10,
                                   msg_hi=16 << 10)
    assert tmpl.region_bytes.max() <= 16 << 20
    ss = bench.ServeSetup(h, inst, src_w, tmpl, seed=SEED, budget=budget, n_channels=4, ring_bytes=ring_bytes,
                          max_msgs=1024, chunk_bytes=64 << 10, op_cost_bytes=2048, verify=verify)
    return src_w, tmpl, ss


def expected_digest(tmpl, kind, t):
    if kind == 0:
        a, b = int(tmpl.op_start[t]), int(tmpl.op_start[t + 1])
        ds = [od.byte_digest(splitmix.fill_bytes(SEED, int(o["src"]), int(o["src_off"]), int(o["n"])))
              for o in tmpl.ops[a:b]]
    else:
        a, b = int(tmpl.msg_start[t]), int(tmpl.msg_start[t + 1])
        ds = [od.byte_digest(splitmix.mpsc_payload_bytes(t, m, int(tmpl.msg_sizes[a + m]))) for m in range(b - a)]
    return od.combine(ds)


def test_alone_equals_mix_equals_oracle(h, inst):
    src_w, tmpl, ss = small_setup(h, inst)
    tr = configs.serve_trace(SEED, rate=200_000.0, duration_s=0.002, n_templates=16)
    reqs = ss.requests(tr)
    assert len(reqs) > 200 and (reqs["kind"] == 1).any() and (reqs["kind"] == 0).any()
    st, alone, s_alone = h.hicr_serve_run(inst, ss.srv, reqs, 1, T)
    print("alone:", st, s_alone.as_dict(), flush=True)
    assert st == 0 and s_alone.completed == len(reqs) and s_alone.max_inflight == 1
    assert h.hicr_serve_digests(inst, ss.srv, reqs, alone) == 0
    st, mix, s_mix = h.hicr_serve_run(inst, ss.srv, reqs, 0, T)
    print("mix:", st, s_mix.as_dict(), h.hicr_last_error_string(inst), flush=True)
    assert st == 0 and s_mix.completed == len(reqs), (st, s_mix.as_dict(), h.hicr_last_error_string(inst))
    assert s_mix.max_inflight > 1, "requests did not overlap on the device"
    assert h.hicr_serve_digests(inst, ss.srv, reqs, mix) == 0
    assert (alone["digest"] == mix["digest"]).all()
    cache = {}
    for i, r in enumerate(reqs):
        key = (int(r["kind"]), int(r["tmpl"]))
        if key not in cache:
            cache[key] = expected_digest(tmpl, *key)
        assert int(mix["digest"][i]) == cache[key], (i, key)
    assert (mix["latency_ns"] > 0).all()
    ss.free()


def _oracle_region(src_w, tmpl, t):
    """The memcpy oracle applies template t's ops to a fresh region slot: the
    expected bytes of every op's destination range."""
    a, b = int(tmpl.op_start[t]), int(tmpl.op_start[t + 1])
    cm = om.CommManager()
    ids = {}
    for o in tmpl.ops[a:b]:
        sl = int(o["src"])
        if sl not in ids:
            ids[sl] = cm.register(om.SPACE_HBM, splitmix.fill_bytes(SEED, sl, 0, int(src_w.slot_sizes[sl])))
    dst = cm.register(om.SPACE_HBM, np.zeros(max(int(tmpl.region_bytes[t]), 1), dtype=np.uint8))
    ops = tmpl.ops[a:b].copy()
    ops["dst"] = dst
    ops["src"] = [ids[int(x)] for x in tmpl.ops[a:b]["src"]]
    assert cm.memcpy_batch(ops) == (om.OK, None)
    return cm.slots[dst].data


def _oracle_burst(tmpl, t, ring=8 << 20, max_msgs=1024):
    """The channel oracle's delivery of burst template t: its messages pushed
    in order by one producer into an MPSC channel and popped one by one."""
    a, b = int(tmpl.msg_start[t]), int(tmpl.msg_start[t + 1])
    orc = oc.MpscOracle(1, ring, max_msgs)
    out = []
    for m in range(b - a):
        data = splitmix.mpsc_payload_bytes(t, m, int(tmpl.msg_sizes[a + m]))
        if orc.push(0, data) == om.ERR_FULL:
            while orc.depth()[0]:
                out.append(orc.payload(0))
                orc.pop(1)
            assert orc.push(0, data) == om.OK
    while orc.depth()[0]:
        out.append(orc.payload(0))
        orc.pop(1)
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint8)


@pytest.mark.parametrize("ring_bytes", [8 << 20, 32 << 10])
def test_mix_delivers_the_oracle_bytes(h, inst, ring_bytes):
    """Every memcpy region and every burst message of a mix, byte for byte.
    With 8 MiB rings every burst is reserved whole (its groups copy side by
    side); with 32 KiB rings the bursts above half a ring reserve group by
    group, and wrap the ring often."""
    src_w, tmpl, ss = small_setup(h, inst, verify=False, budget=2 << 30, ring_bytes=ring_bytes)  # room for every kept region
    bb16 = np.array([int(((tmpl.msg_sizes[tmpl.msg_start[t]:tmpl.msg_start[t + 1]].astype(np.int64) + 15) // 16 * 16).sum())
                     for t in range(16)])
    if ring_bytes == 32 << 10:
        assert (bb16 > ring_bytes // 2).any() and (bb16 <= ring_bytes // 2).any()  # both reservation forms
    tr = configs.serve_trace(SEED + 2, rate=200_000.0, duration_s=0.002, n_templates=16)
    reqs = ss.requests(tr)
    burst = reqs["kind"] == 1
    assert burst.any() and (~burst).any()
    bbytes = np.array([int(tmpl.msg_sizes[tmpl.msg_start[t]:tmpl.msg_start[t + 1]].sum()) for t in range(16)])
    cap_off = np.full(len(reqs), np.iinfo(np.uint64).max, dtype=np.uint64)
    sizes = np.where(burst, bbytes[reqs["tmpl"]], 0).astype(np.uint64)
    cap_off[burst] = (np.cumsum(sizes) - sizes)[burst]
    cap = torch.zeros(max(int(sizes.sum()), 16), dtype=torch.uint8, device="cuda")
    d_off = torch.from_numpy(cap_off.view(np.int64).copy()).cuda()
    keep = (~burst).astype(np.uint8)
    st, res, stats = h.hicr_serve_run_ex(inst, ss.srv, reqs, 0, T, keep=keep, d_capture=cap, d_cap_off=d_off)
    assert st == 0 and stats.completed == len(reqs), (st, stats.as_dict(), h.hicr_last_error_string(inst))
    assert stats.max_inflight > 1
    st, arena = h.hicr_serve_arena(inst, ss.srv)
    st, aptr, asize, _, _ = h.hicr_slot_info(inst, arena)
    torch.cuda.synchronize()
    got_cap = cap.cpu().numpy()
    regions, bursts = {}, {}
    for i, r in enumerate(reqs):
        t = int(r["tmpl"])
        if r["kind"] == 0:
            if t not in regions:
                regions[t] = _oracle_region(src_w, tmpl, t)
            n = int(tmpl.region_bytes[t])
            got = device_bytes(aptr + int(res["dst_offset"][i]), n).cpu().numpy()
            a, b = int(tmpl.op_start[t]), int(tmpl.op_start[t + 1])
            for o in tmpl.ops[a:b]:
                d0, k = int(o["dst_off"]), int(o["n"])
                assert (got[d0:d0 + k] == regions[t][d0:d0 + k]).all(), (i, t, d0)
        else:
            if t not in bursts:
                bursts[t] = _oracle_burst(tmpl, t)
            o = int(cap_off[i])
            assert (got_cap[o:o + len(bursts[t])] == bursts[t]).all(), (i, t)
    # the digests agree with the bytes
    assert h.hicr_serve_digests(inst, ss.srv, reqs, res) == 0
    for i, r in enumerate(reqs):
        assert int(res["digest"][i]) == expected_digest(tmpl, int(r["kind"]), int(r["tmpl"])), i
    ss.free()


def test_budget_limits_admission_and_everything_completes(h, inst):
    # the arena holds only a few regions at once: requests queue for memory
    src_w, tmpl, ss = small_setup(h, inst, verify=False, budget=(4 * (8 << 20)) + (2 << 20))
    tr = configs.serve_trace(SEED + 1, rate=500_000.0, duration_s=0.001, n_templates=16)
    reqs = ss.requests(tr)
    st, res, stats = h.hicr_serve_run(inst, ss.srv, reqs, 0, 20_000_000_000)
    print("budget run:", st, stats.as_dict(), h.hicr_last_error_string(inst), flush=True)
    assert st == 0 and stats.completed == len(reqs), (st, stats.as_dict(), h.hicr_last_error_string(inst))
    assert stats.max_region_bytes <= 2 << 20
    assert (res["admit_ns"] > 0).any(), "no request had to wait for memory"
    burst = reqs["kind"] == 1
    for i in np.nonzero(burst)[0][:50]:
        assert int(res["digest"][i]) == expected_digest(tmpl, 1, int(reqs["tmpl"][i]))
    # the device clock at each completion: every request has one, and their
    # spread fits the host-observed span of the run (first arrival to last
    # completion seen; the two clocks share no origin, only differences)
    dev = res["device_done_ns"].astype(np.int64)
    assert (dev > 0).all()
    assert dev.max() - dev.min() <= int(stats.wall_ns) + 1_000_000
    # the host loop's longest pause ends inside the run, after it began
    assert 0 < stats.max_poll_gap_ns <= stats.max_poll_gap_at_ns
    st, pres, pstats = h.hicr_serve_run_plain(inst, ss.srv, reqs, int(1e12), T)
    assert st == 0 and pstats.completed == len(reqs)
    assert (pres["device_done_ns"] == 0).all()  # the plain form has no device clock per request
    assert 0 < pstats.max_poll_gap_ns <= pstats.max_poll_gap_at_ns
    ss.free()


def test_serve_rejects_bad_requests(h, inst):
    src_w, tmpl, ss = small_setup(h, inst)
    reqs = np.zeros(2, dtype=h.SERVE_REQ_DTYPE)
    reqs["tmpl"] = [0, 999]
    assert h.hicr_serve_run(inst, ss.srv, reqs, 0, T)[0] == h.HICR_ERR_INVALID
    reqs["tmpl"] = [0, 0]
    reqs["arrival_ns"] = [10, 5]
    assert h.hicr_serve_run(inst, ss.srv, reqs, 0, T)[0] == h.HICR_ERR_INVALID
    ss.free()


def test_finalize_releases_an_engine_left_alive(h):
    """An engine the caller never destroys is released with its instance:
    its arena and rings (here 8 GiB) return to the device."""
    import torch
    torch.cuda.synchronize()
    st, i2 = h.hicr_init(0)
    assert st == 0
    free0 = torch.cuda.mem_get_info()[0]
    cfg = dict(budget_bytes=8 << 30, n_channels=4, max_msgs=1024, ring_bytes=256 << 20, chunk_bytes=64 << 10,
               op_cost_bytes=2048, verify=0)
    h.check(h.hicr_serve_create(i2, cfg), "serve_create")
    assert torch.cuda.mem_get_info()[0] < free0 - (7 << 30)
    assert h.hicr_finalize(i2) == 0
    assert torch.cuda.mem_get_info()[0] > free0 - (256 << 20)
