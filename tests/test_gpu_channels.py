"""GPU parity of the SPSC / MPSC channels against the channel oracle.

Host calls (push / peek / pop / depth) are deterministic and must match the
oracle exactly: statuses, ring offsets, sizes, producers, sequence numbers
and payload bytes. Device streaming runs interleave producers freely: the
SPSC stream must deliver the exact token stream, the MPSC stream must pass
the interleaving-agnostic checker (multiset, per-producer order, sizes, ring
offsets replayed from the placement rule) without ever exceeding capacity.
What the consumers received is compared with what the oracle delivers byte
by byte: the streams' capture forms store every consumed token or message,
and the ping-pong's capture form both agents' buffers. The digests are
checked as well, as an extra.
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

ST = {"OK": om.OK, "FULL": om.ERR_FULL, "EMPTY": om.ERR_EMPTY, "TOO_LARGE": om.ERR_TOO_LARGE}


def ring_bytes(h, inst, ch, off, n):
    st, rs = h.hicr_channel_ring(inst, ch)
    st, ptr, size, _, _ = h.hicr_slot_info(inst, rs)
    torch.cuda.synchronize()
    return device_bytes(ptr + off, n).cpu().numpy()


def src_slot(h, inst, data: np.ndarray):
    t = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    st, s = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, t.data_ptr(), t.numel())
    assert st == 0
    return s, t


def _rewrite_pool(h, inst, rng, s, pool, s2, other):
    """Overwrite a random range of the source slot by a memcpy from a second
    slot (a small batch: in latency mode the server takes it) and mirror it in
    the oracle's copy of the pool. The next push reads the new bytes: a
    channel call comes after everything issued before it. The fence first
    completes the previous rewrite: two copies that write the same bytes in
    one epoch are unordered (the oracle would apply them in issue order)."""
    assert h.hicr_fence(inst, 0, 10**10) == 0
    n = int(rng.integers(1, min(len(pool), 512) + 1))
    d = int(rng.integers(0, len(pool) - n + 1))
    o = int(rng.integers(0, len(other) - n + 1))
    assert h.hicr_memcpy(inst, s, d, s2, o, n) == 0
    pool[d:d + n] = other[o:o + n]


LATENCY = pytest.mark.parametrize("idle_us", [0, 3000], ids=["launch", "latency_mode"])


@LATENCY
@pytest.mark.parametrize("seed,ts,cap", [(0, 8, 5), (1, 24, 7), (2, 64, 16)])
def test_spsc_host_calls_match_oracle(h, inst, seed, ts, cap, idle_us):
    """Statuses, offsets and token bytes of push / peek / pop / depth match
    the SPSC oracle; with latency mode on, the calls go to the server kernel
    and the pool is rewritten by server-side copies between them."""
    rng = np.random.default_rng(seed)
    assert h.hicr_set_latency_mode(inst, idle_us) == 0
    st, ch = h.hicr_spsc_create(inst, ts, cap)
    assert st == 0
    orc = oc.SpscOracle(ts, cap)
    pool = rng.integers(0, 256, ts * 4 * cap, dtype=np.uint8)
    s, keep = src_slot(h, inst, pool)
    other = rng.integers(0, 256, 4096, dtype=np.uint8)
    s2, keep2 = src_slot(h, inst, other)
    for step in range(300):
        r = rng.random()
        if r < 0.08:
            _rewrite_pool(h, inst, rng, s, pool, s2, other)
        elif r < 0.45:
            k = int(rng.integers(0, cap + 2))
            off = int(rng.integers(0, len(pool) - k * ts + 1))
            exp = orc.push(pool[off:off + k * ts])
            assert h.hicr_channel_push(inst, ch, 0, s, off, k) == exp, step
        elif r < 0.7:
            k = int(rng.integers(0, cap + 2))
            assert h.hicr_channel_pop(inst, ch, k) == orc.pop(k), step
        elif r < 0.9:
            k = int(rng.integers(0, cap + 1))
            est, info = orc.peek(k)
            gst, ginfo = h.hicr_channel_peek(inst, ch, k)
            assert gst == est, step
            if est == om.OK:
                assert ginfo == info
                assert (ring_bytes(h, inst, ch, ginfo[0], ts) == orc.token(k)).all()
        else:
            assert h.hicr_channel_depth(inst, ch)[1:] == orc.depth()
    assert h.hicr_channel_push(inst, ch, 1, s, 0, 1) == h.HICR_ERR_INVALID  # SPSC has producer 0 only
    assert h.hicr_channel_push(inst, ch, 0, s, len(pool), 1) == h.HICR_ERR_BOUNDS
    assert h.hicr_channel_destroy(inst, ch) == 0
    assert h.hicr_channel_depth(inst, ch)[0] == h.HICR_ERR_INVALID


def test_latency_mode_push_after_a_stream_copy_reads_its_bytes(h, inst):
    """In latency mode a channel call goes to the server only while the
    communication stream is quiet. A 4 MiB memcpy is beyond the server's
    small-op limit, so the stream runs it; the push issued right after it
    must come behind it (a launch after the copy) and carry the new bytes."""
    rng = np.random.default_rng(11)
    assert h.hicr_set_latency_mode(inst, 3000) == 0
    ts, cap, n = 64, 64, 4 << 20
    st, ch = h.hicr_spsc_create(inst, ts, cap)
    assert st == 0
    orc = oc.SpscOracle(ts, cap)
    pool = np.zeros(n, dtype=np.uint8)
    s, keep = src_slot(h, inst, pool)
    other = rng.integers(0, 256, n, dtype=np.uint8)
    s2, keep2 = src_slot(h, inst, other)
    for rep in range(6):
        fresh = rng.integers(0, 256, n, dtype=np.uint8)
        keep2.copy_(torch.from_numpy(fresh))
        torch.cuda.synchronize()
        assert h.hicr_memcpy(inst, s, 0, s2, 0, n) == 0
        off = int(rng.integers(0, n // ts - 8)) * ts
        assert h.hicr_channel_push(inst, ch, 0, s, off, 8) == orc.push(fresh[off:off + 8 * ts]), rep
        for j in range(8):
            gst, info = h.hicr_channel_peek(inst, ch, j)
            est, einfo = orc.peek(j)
            assert gst == est == om.OK and info == einfo, (rep, j)
            assert (ring_bytes(h, inst, ch, info[0], ts) == orc.token(j)).all(), (rep, j)
        assert h.hicr_channel_pop(inst, ch, 8) == orc.pop(8) == om.OK
        assert h.hicr_fence(inst, 0, 10**10) == 0
    assert h.hicr_set_latency_mode(inst, 0) == 0
    assert h.hicr_channel_destroy(inst, ch) == 0


def test_mpsc_golden_wraparound_through_the_abi(h, inst):
    from tests.test_oracle_channels import load_mpsc_golden
    prog = load_mpsc_golden()
    R, M, P = map(int, prog[0][1:])
    st, ch = h.hicr_mpsc_create(inst, P, R, M)
    assert st == 0
    pool = np.concatenate([splitmix.mpsc_payload_bytes(p, q, 128) for p in range(P) for q in range(8)])
    s, keep = src_slot(h, inst, pool)
    seq = [0] * P
    for f in prog[1:]:
        if f[0] == "push":
            p, n = int(f[1]), int(f[2])
            off = (p * 8 + seq[p]) * 128
            got = h.hicr_channel_push(inst, ch, p, s, off, n)
            assert got == ST[f[3]], f
            if got == om.OK:
                seq[p] += 1
        elif f[0] == "pop":
            assert h.hicr_channel_pop(inst, ch, int(f[1])) == ST[f[2]], f
        elif f[0] == "peek":
            gst, info = h.hicr_channel_peek(inst, ch, int(f[1]))
            assert gst == ST[f[2]], f
            if gst == om.OK:
                assert list(info) == [int(x) for x in f[3:7]], f
                o, n, p, q = info
                assert (ring_bytes(h, inst, ch, o, n) == pool[(p * 8 + q) * 128:(p * 8 + q) * 128 + n]).all()
        elif f[0] == "depth":
            assert h.hicr_channel_depth(inst, ch)[1:] == (int(f[1]), int(f[2])), f


@LATENCY
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mpsc_host_calls_match_oracle(h, inst, seed, idle_us):
    rng = np.random.default_rng(seed)
    assert h.hicr_set_latency_mode(inst, idle_us) == 0
    P, R, M = 4, 1 << 12, 8
    st, ch = h.hicr_mpsc_create(inst, P, R, M)
    assert st == 0
    orc = oc.MpscOracle(P, R, M)
    pool = rng.integers(0, 256, 1 << 16, dtype=np.uint8)
    s, keep = src_slot(h, inst, pool)
    other = rng.integers(0, 256, 4096, dtype=np.uint8)
    s2, keep2 = src_slot(h, inst, other)
    for step in range(400):
        r = rng.random()
        if r < 0.06:
            _rewrite_pool(h, inst, rng, s, pool, s2, other)
        elif r < 0.5:
            p = int(rng.integers(0, P))
            n = int(rng.choice([0, 1, 7, 16, 17, 100, 500, 1500, 2100, 4096, 5000]))
            off = int(rng.integers(0, len(pool) - n + 1))
            exp = orc.push(p, pool[off:off + n])
            assert h.hicr_channel_push(inst, ch, p, s, off, n) == exp, (step, p, n)
        elif r < 0.75:
            k = int(rng.integers(0, 4))
            assert h.hicr_channel_pop(inst, ch, k) == orc.pop(k), step
        elif r < 0.92:
            k = int(rng.integers(0, M + 1))
            est, info = orc.peek(k)
            gst, ginfo = h.hicr_channel_peek(inst, ch, k)
            assert gst == est, step
            if est == om.OK:
                assert ginfo == info, step
                assert (ring_bytes(h, inst, ch, ginfo[0], ginfo[1]) == orc.payload(k)).all()
        else:
            assert h.hicr_channel_depth(inst, ch)[1:] == orc.depth(), step
    assert h.hicr_channel_push(inst, ch, P, s, 0, 8) == h.HICR_ERR_INVALID
    assert h.hicr_mpsc_create(inst, 2, 3000, 8)[0] == h.HICR_ERR_INVALID   # ring not a power of two


def _spsc_expected_digest(channel, tokens, wpt=8):
    d = 0
    step = 1 << 20
    for t0 in range(0, tokens, step):
        n = min(step, tokens - t0)
        d = (d + od.word_digest(splitmix.spsc_token_words(channel, t0, n, wpt), t0 * wpt)) % (1 << 64)
    return d


def _spsc_through_oracle(stream: np.ndarray, ts: int, cap: int) -> np.ndarray:
    """Push the tokens of `stream` through the SPSC oracle (capacity `cap`) in
    batches of up to `cap` tokens, popping each batch: the bytes the oracle
    delivers, in order."""
    orc = oc.SpscOracle(ts, cap)
    out = []
    n = len(stream) // ts
    for t0 in range(0, n, cap):
        k = min(cap, n - t0)
        assert orc.push(stream[t0 * ts:(t0 + k) * ts]) == om.OK
        out.extend(orc.token(j) for j in range(k))
        assert orc.pop(k) == om.OK
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint8)


def _rule_stream(channel, tokens, ts):
    return splitmix.spsc_token_words(channel, 0, tokens, ts // 8).astype("<u8").view(np.uint8)


@pytest.mark.parametrize("digest_only", [False, True], ids=["verify", "digest_only"])
@pytest.mark.parametrize("n_ch,cap,ts,tokens,batch", [
    (64, 4096, 64, 100_000, 256),
    (8, 16, 64, 1003, 16),
    (4, 64, 32, 5000, 1),
    (2, 4096, 128, 70_000, 4096),
    (3, 100, 48, 2_000, 7),          # 3 vectors per token: the general (non-divisible) layout
])
def test_spsc_stream_exact_token_stream(h, inst, n_ch, cap, ts, tokens, batch, digest_only):
    """The consumers' captured streams equal, token by token, the payload-rule
    stream pushed through the SPSC oracle (every channel of the small cases;
    the first and last channel of the 64-channel case, whose other channels
    are compared with the payload rule's words directly). Both consumer forms:
    checking every word against the rule, and digesting only."""
    chans = [h.hicr_spsc_create(inst, ts, cap)[1] for _ in range(n_ch)]
    cap_buf = torch.zeros(n_ch * tokens * ts, dtype=torch.uint8, device="cuda")
    st, res = h.hicr_spsc_stream_ex(inst, chans, tokens, batch, d_capture=cap_buf.data_ptr(),
                                    capture_stride=tokens * ts,
                                    flags=h.HICR_SPSC_DIGEST_ONLY if digest_only else 0)
    assert st == 0
    got = cap_buf.cpu().numpy().reshape(n_ch, tokens * ts)
    for i, r in enumerate(res):
        assert (r.pushed, r.popped, r.mismatches, r.status) == (tokens, tokens, 0, 0)
        assert 0 < r.max_occupancy <= cap
        assert r.digest == _spsc_expected_digest(i, tokens, ts // 8), i
        assert h.hicr_channel_depth(inst, chans[i])[1] == 0
        exp = _rule_stream(i, tokens, ts)
        if n_ch <= 8 or i in (0, n_ch - 1):
            exp = _spsc_through_oracle(exp, ts, cap)
        bad = np.nonzero(got[i] != exp)[0]
        assert len(bad) == 0, f"channel {i}: {len(bad)} bytes differ, first in token {bad[0] // ts}"
    # a second run continues from the channels' counters
    st, res2 = h.hicr_spsc_stream(inst, chans[:1], 100, min(batch, 100))
    assert st == 0 and res2[0].digest == _spsc_expected_digest(0, 100, ts // 8)


@pytest.mark.parametrize("n_ch,cap,ts,tokens,batch,staged", [
    (16, 4096, 64, 50_000, 256, 4096),
    (4, 16, 64, 1003, 16, 7),
    (3, 64, 32, 5000, 1, 64),
    (2, 100, 48, 2_000, 7, 33),      # the general layout
    (1, 8, 16, 333, 8, 1),
    (1, 4096, 64, 20_000, 2048, 1),  # one staged token
    (76, 64, 64, 3_000, 32, 64),     # as many channels as can be resident: one CTA on every SM
])
def test_spsc_copy_producers_deliver_the_staged_tokens(h, inst, n_ch, cap, ts, tokens, batch, staged):
    """Producers that push by copying from a memory slot (Sec. 4.3): token s
    of channel i is staged token (s mod staged) of that channel; the captured
    stream equals that sequence pushed through the SPSC oracle, and the digest
    equals the oracle digest of those words."""
    rng = np.random.default_rng(ts * 1000 + n_ch)
    pool = rng.integers(0, 256, n_ch * staged * ts + 16, dtype=np.uint8)
    s, keep = src_slot(h, inst, pool)
    chans = [h.hicr_spsc_create(inst, ts, cap)[1] for _ in range(n_ch)]
    cap_buf = torch.zeros(n_ch * tokens * ts, dtype=torch.uint8, device="cuda")
    st, res = h.hicr_spsc_stream_ex(inst, chans, tokens, batch, src=s, src_off=16, src_tokens=staged,
                                    d_capture=cap_buf.data_ptr(), capture_stride=tokens * ts)
    assert st == 0
    got = cap_buf.cpu().numpy().reshape(n_ch, tokens * ts)
    for i, r in enumerate(res):
        assert (r.pushed, r.popped, r.mismatches, r.status) == (tokens, tokens, 0, 0)
        mine = pool[16 + i * staged * ts:16 + (i + 1) * staged * ts].reshape(staged, ts)
        pushed = mine[np.arange(tokens) % staged].reshape(-1)
        exp = _spsc_through_oracle(pushed, ts, cap) if tokens * n_ch <= 200_000 else pushed
        assert (got[i] == exp).all(), i
        assert r.digest == od.byte_digest(exp), i
    # without capture the same run gives the same digests
    st, res2 = h.hicr_spsc_stream_ex(inst, chans, tokens, batch, src=s, src_off=16, src_tokens=staged)
    assert st == 0 and [r.digest for r in res2] == [r.digest for r in res]
    # staged tokens outside the slot, and an unaligned staging address
    assert h.hicr_spsc_stream_ex(inst, chans, tokens, batch, src=s, src_off=32, src_tokens=staged)[0] == \
        h.HICR_ERR_BOUNDS
    assert h.hicr_spsc_stream_ex(inst, chans, tokens, batch, src=s, src_off=8, src_tokens=staged)[0] == \
        h.HICR_ERR_INVALID


def test_spsc_stream_rejects_unknown_flags(h, inst):
    ch = h.hicr_spsc_create(inst, 64, 64)[1]
    assert h.hicr_spsc_stream_ex(inst, [ch], 10, 8, flags=2)[0] == h.HICR_ERR_INVALID
    st, res = h.hicr_spsc_stream_ex(inst, [ch], 10, 8, flags=h.HICR_SPSC_DIGEST_ONLY)
    assert st == 0 and res[0].popped == 10 and res[0].digest == _spsc_expected_digest(0, 10)


def test_spsc_stream_rejects_more_channels_than_can_be_resident(h, inst):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    chans = [h.hicr_spsc_create(inst, 64, 64)[1] for _ in range(sms // 2 + 1)]
    assert h.hicr_spsc_stream(inst, chans, 100, 16)[0] == h.HICR_ERR_INVALID
    assert h.hicr_spsc_stream(inst, chans[:-1], 100, 16)[0] == h.HICR_OK
    for c in chans:
        assert h.hicr_channel_destroy(inst, c) == 0


def _oracle_deliveries(w, ring, max_msgs, nonlocking):
    """What the channel oracle delivers, message by message: for each consumer
    c, its producers (c, c + C, ...) push their messages round-robin into one
    oracle channel (locking: MpscOracle, one shared ring; non-locking:
    MpscNonLockingOracle, a ring per producer); whenever a push finds no room
    the consumer pops everything buffered, and it drains the channel at the
    end. Returns {(producer, seq): the payload bytes popped}."""
    P, M = w.sizes.shape
    out = {}
    for c in range(w.n_consumers):
        prods = list(range(c, P, w.n_consumers))
        orc = (oc.MpscNonLockingOracle if nonlocking else oc.MpscOracle)(len(prods), ring, max_msgs)

        def drain():
            while orc.depth()[0]:
                st, (_, n, k, s) = orc.peek(0)
                out[(prods[k], s)] = orc.payload(0)
                assert len(out[(prods[k], s)]) == n and orc.pop(1) == om.OK

        for s in range(M):
            for k, p in enumerate(prods):
                data = splitmix.mpsc_payload_bytes(p, s, int(w.sizes[p, s]))
                st = orc.push(k, data)
                if st == om.ERR_FULL:
                    drain()
                    st = orc.push(k, data)
                assert st == om.OK, (c, p, s, st)
        drain()
    return out


def _check_capture(w, run, deliveries):
    """The capture buffer holds every message the GPU consumers received at
    its staging offset, and zeros elsewhere: compare it with the oracle's
    deliveries byte by byte."""
    got = run.capture.cpu().numpy()
    exp = np.zeros_like(got)
    P, M = w.sizes.shape
    assert len(deliveries) == P * M
    for (p, s), data in deliveries.items():
        o = int(run.offs[p * M + s])
        exp[o:o + len(data)] = data
    bad = np.nonzero(got != exp)[0]
    assert len(bad) == 0, f"{len(bad)} captured bytes differ from the oracle's deliveries, first at {bad[0]}"


def _check_mpsc(w, logs, res, ring, sample=1.0, seed=0):
    rng = np.random.default_rng(seed)
    C = w.n_consumers
    for c in range(C):
        n = int(res[c].consumed)
        L = logs[c][:n]
        assert res[c].status == 0
        assert int(res[c].max_inflight_bytes) <= ring
        assert int(res[c].max_inflight_msgs) <= w.max_msgs
        probs = oc.check_mpsc_log(w.sizes, C, c, list(zip(L["producer"], L["seq"], L["size"], L["offset"])), ring)
        assert probs == [], (c, probs[:5])
        assert int(res[c].bytes) == int(L["size"].astype(np.int64).sum())
        idx = np.nonzero(rng.random(n) < sample)[0]
        for j in idx:
            p, q, sz = int(L["producer"][j]), int(L["seq"][j]), int(L["size"][j])
            assert int(L["digest"][j]) == od.byte_digest(splitmix.mpsc_payload_bytes(p, q, sz)), (c, j)


@pytest.mark.parametrize("P,C,M,ring,max_msgs,hi,group,ctas", [
    (64, 4, 64, 1 << 20, 256, 16 << 10, 4, 1),
    (48, 3, 40, 1 << 16, 64, 4 << 10, 1, 3),
    (33, 5, 17, 1 << 14, 32, 2 << 10, 8, 2),
    (64, 2, 100, 1 << 15, 16, 4 << 10, 2, 5),
])
def test_mpsc_stream_checker_and_payloads(h, inst, P, C, M, ring, max_msgs, hi, group, ctas):
    w = configs.mpsc(7, n_producers=P, n_consumers=C, msgs_per_producer=M, ring_bytes=ring, max_msgs=max_msgs,
                     hi=hi)
    run = bench.MpscRun(h, inst, w, group=group, consumer_ctas=ctas)
    st, res = run.run(capture=True)
    assert st == 0
    _check_mpsc(w, run.logs(), res, ring)
    _check_capture(w, run, _oracle_deliveries(w, ring, max_msgs, False))
    # the rings wrapped (skip-to-start exercised) and are empty again
    assert sum(int(r.bytes) for r in res) > ring
    for ch in run.chans:
        assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    # a second run continues from the channels' counters
    st, res = run.run()
    assert st == 0 and sum(int(r.consumed) for r in res) == P * M
    for ch in run.chans:
        assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    run.free()


@pytest.mark.parametrize("nonlocking", [False, True])
@pytest.mark.parametrize("gap", [None, 3])
def test_mpsc_stream_odd_staging_and_empty_messages(h, inst, nonlocking, gap):
    """Every fifth message is empty (zero-byte bodies inside the producers'
    group copies and the consumers' digest walks); with gap = 3 the staged
    payloads sit at arbitrary alignments, so the producers' bulk copies fall
    back to the warp copy for most messages of a group but not all."""
    ring, max_msgs = 1 << 16, (8 if nonlocking else 64)
    w = configs.mpsc(13, n_producers=40, n_consumers=4, msgs_per_producer=50, ring_bytes=ring, max_msgs=max_msgs,
                     hi=8 << 10)
    w.sizes[:, ::5] = 0
    run = bench.MpscRun(h, inst, w, group=8, nonlocking=nonlocking, consumer_ctas=2, ring_bytes=ring,
                        max_msgs=max_msgs, stage_gap=gap)
    st, res = run.run(capture=True)
    assert st == 0
    if nonlocking:
        _check_mpsc_nl(w, run, res)
    else:
        _check_mpsc(w, run.logs(), res, ring)
    _check_capture(w, run, _oracle_deliveries(w, ring, max_msgs, nonlocking))
    assert sum(int(r.consumed) for r in res) == w.sizes.size
    run.free()


@pytest.mark.parametrize("nbytes,ctas,off", [
    (1, 1, 7), (17, 1, 7), (4096, 2, 7), ((1 << 20) + 3, 8, 7), ((64 << 20) + 5, 152, 7),
    # agents of at most half the SMs with >= 64 KiB per warp: the bulk-copy form
    # (from an unaligned source the send falls back to the warp copy, the echo does not)
    (64 << 20, 32, 7), ((128 << 20) + 9, 64, 0), ((96 << 20) + 1, 76, 16),
])
def test_pingpong_delivers_the_message(h, inst, nbytes, ctas, off):
    """Test Case 1 restated on one GPU: after the round trips both
    single-message buffers hold exactly the message (oracle digest)."""
    size = nbytes + 100
    st, s = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size)
    assert h.hicr_util_fill(inst, s, 0, size, splitmix.fill_key_base(5, 1)) == 0
    out_a = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out_b = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    st, r = h.hicr_pingpong_capture(inst, s, off, nbytes, out_a.data_ptr(), out_b.data_ptr(), reps=10, warmup=2,
                                    ctas_per_side=ctas)
    assert st == 0 and r.status == 0
    # the oracle: A pushes the message into B's single-message channel, B pops
    # it and pushes it back into A's, A pops it (two rounds suffice: every
    # round leaves the same bytes)
    msg = splitmix.fill_bytes(5, 1, off, nbytes)
    ab, ba = oc.SpscOracle(nbytes, 1), oc.SpscOracle(nbytes, 1)
    for _ in range(2):
        assert ab.push(msg) == om.OK
        got_b = ab.token(0)
        assert ab.pop(1) == om.OK and ba.push(got_b) == om.OK
        got_a = ba.token(0)
        assert ba.pop(1) == om.OK
    assert (out_b.cpu().numpy() == got_b).all() and (out_a.cpu().numpy() == got_a).all()
    exp = od.byte_digest(msg)
    assert r.digest_a == exp and r.digest_b == exp
    assert r.half_rtt_ns > 0 and r.goodput_gbs > 0
    assert h.hicr_pingpong(inst, s, 200, size, 1, 0, 1)[0] == h.HICR_ERR_BOUNDS
    assert h.hicr_pingpong(inst, s, 0, 16, 1, 0, 257)[0] == h.HICR_ERR_INVALID
    assert h.hicr_mem_free(inst, s) == 0


@LATENCY
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_nonlocking_host_calls_match_oracle(h, inst, seed, idle_us):
    """Non-locking MPSC (one ring per producer): statuses, offsets within the
    producer's ring, sizes, producers, sequence numbers and payloads match the
    non-locking oracle under random programs that fill and wrap the rings."""
    rng = np.random.default_rng(seed)
    assert h.hicr_set_latency_mode(inst, idle_us) == 0
    P, R, M = 3, 1 << 10, 4
    st, ch = h.hicr_mpsc_nl_create(inst, P, R, M)
    assert st == 0
    orc = oc.MpscNonLockingOracle(P, R, M)
    pool = rng.integers(0, 256, 1 << 14, dtype=np.uint8)
    s, keep = src_slot(h, inst, pool)
    other = rng.integers(0, 256, 4096, dtype=np.uint8)
    s2, keep2 = src_slot(h, inst, other)
    for step in range(400):
        r = rng.random()
        if r < 0.06:
            _rewrite_pool(h, inst, rng, s, pool, s2, other)
        elif r < 0.5:
            p = int(rng.integers(0, P))
            n = int(rng.choice([0, 1, 9, 16, 100, 333, 512, 700, 1024, 1100]))
            off = int(rng.integers(0, len(pool) - n + 1))
            exp = orc.push(p, pool[off:off + n])
            assert h.hicr_channel_push(inst, ch, p, s, off, n) == exp, (step, p, n)
        elif r < 0.72:
            k = int(rng.integers(0, 5))
            assert h.hicr_channel_pop(inst, ch, k) == orc.pop(k), step
        elif r < 0.92:
            k = int(rng.integers(0, P * M + 1))
            est, info = orc.peek(k)
            gst, ginfo = h.hicr_channel_peek(inst, ch, k)
            assert gst == est, step
            if est == om.OK:
                assert ginfo == info, step
                o, n, p, q = info
                assert (ring_bytes(h, inst, ch, p * R + o, n) == orc.payload(k)).all()
        else:
            assert h.hicr_channel_depth(inst, ch)[1:] == orc.depth(), step
    assert h.hicr_channel_push(inst, ch, P, s, 0, 8) == h.HICR_ERR_INVALID
    assert h.hicr_mpsc_nl_create(inst, 2, 3000, 8)[0] == h.HICR_ERR_INVALID
    assert h.hicr_mpsc_nl_create(inst, 2, 1024, 6)[0] == h.HICR_ERR_INVALID


def _check_mpsc_nl(w, run, res, sample=1.0, seed=0):
    rng = np.random.default_rng(seed)
    C = w.n_consumers
    logs = run.logs()
    for c in range(C):
        n = int(res[c].consumed)
        L = logs[c][:n]
        assert res[c].status == 0 and res[c].cas_failures == 0
        assert int(res[c].max_inflight_bytes) <= run.ring_bytes
        assert int(res[c].max_inflight_msgs) <= run.max_msgs
        probs = oc.check_mpsc_nl_log(w.sizes, C, c, list(zip(L["producer"], L["seq"], L["size"], L["offset"])),
                                     run.ring_bytes)
        assert probs == [], (c, probs[:5])
        assert int(res[c].bytes) == int(L["size"].astype(np.int64).sum())
        for j in np.nonzero(rng.random(n) < sample)[0]:
            p, q, sz = int(L["producer"][j]), int(L["seq"][j]), int(L["size"][j])
            assert int(L["digest"][j]) == od.byte_digest(splitmix.mpsc_payload_bytes(p, q, sz)), (c, j)


@pytest.mark.parametrize("P,C,M,ring,max_msgs,hi,group,ctas", [
    (64, 4, 64, 1 << 16, 8, 16 << 10, 4, 1),
    (48, 3, 40, 1 << 13, 4, 2 << 10, 1, 2),
    (33, 5, 17, 1 << 12, 2, 1 << 10, 8, 1),
    (700, 2, 6, 1 << 11, 8, 1 << 10, 2, 1),   # 350 rings per consumer: warps poll up to 22 rings
])
def test_nonlocking_stream_checker_and_payloads(h, inst, P, C, M, ring, max_msgs, hi, group, ctas):
    w = configs.mpsc(9, n_producers=P, n_consumers=C, msgs_per_producer=M, ring_bytes=ring, max_msgs=max_msgs,
                     hi=hi)
    run = bench.MpscRun(h, inst, w, group=group, nonlocking=True, consumer_ctas=ctas, ring_bytes=ring,
                        max_msgs=max_msgs)
    st, res = run.run(capture=True)
    assert st == 0
    _check_mpsc_nl(w, run, res)
    _check_capture(w, run, _oracle_deliveries(w, ring, max_msgs, True))
    # some rings wrapped (skip-to-start exercised) and all are empty again
    assert (((w.sizes + 15) // 16 * 16).sum(1) > ring).any()
    for ch in run.chans:
        assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    # a second run continues from the rings' counters; the positions then
    # start where the first run stopped, so only order, sizes and payloads
    # are checked
    st, res = run.run()
    assert st == 0 and sum(int(r.consumed) for r in res) == P * M
    run.free()


def test_nonlocking_stream_rejects_bad_shapes(h, inst):
    w = configs.mpsc(3, n_producers=8, n_consumers=2, msgs_per_producer=4, ring_bytes=1 << 12, max_msgs=4, hi=512)
    run = bench.MpscRun(h, inst, w, nonlocking=True, ring_bytes=1 << 12, max_msgs=4)
    P, M = w.sizes.shape
    args = (run.d_sizes.data_ptr(), run.d_offs.data_ptr(), run.staging)
    # the locking-mode stream does not take non-locking channels and vice versa
    assert h.hicr_mpsc_stream(inst, run.chans, P, M, *args, 1, 1, run.d_log.data_ptr(), run.stride)[0] == \
        h.HICR_ERR_INVALID
    lock = [h.hicr_mpsc_create(inst, 4, 1 << 12, 4)[1] for _ in range(2)]
    assert h.hicr_mpsc_nl_stream(inst, lock, P, M, *args, 1, 1, run.d_log.data_ptr(), run.stride)[0] == \
        h.HICR_ERR_INVALID
    # zero CTAs per consumer, a group above 8, a log stride too small
    assert h.hicr_mpsc_nl_stream(inst, run.chans, P, M, *args, 1, 0, run.d_log.data_ptr(), run.stride)[0] == \
        h.HICR_ERR_INVALID
    assert h.hicr_mpsc_nl_stream(inst, run.chans, P, M, *args, 9, 1, run.d_log.data_ptr(), run.stride)[0] == \
        h.HICR_ERR_INVALID
    assert h.hicr_mpsc_nl_stream(inst, run.chans, P, M, *args, 1, 1, run.d_log.data_ptr(), run.stride - 1)[0] == \
        h.HICR_ERR_INVALID
    # a message above half a ring is TOO_LARGE before anything is launched
    small = [h.hicr_mpsc_nl_create(inst, 4, 256, 4)[1] for _ in range(2)]
    assert h.hicr_mpsc_nl_stream(inst, small, P, M, *args, 1, 1, run.d_log.data_ptr(), run.stride)[0] == \
        h.HICR_ERR_TOO_LARGE
    for c in lock + small:
        assert h.hicr_channel_destroy(inst, c) == 0
    st, res = run.run()
    assert st == 0
    _check_mpsc_nl(w, run, res)
    run.free()
