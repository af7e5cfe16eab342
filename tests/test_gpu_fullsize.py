"""Full-size configurations in the launch configuration bench.py times.

Batched memcpy (256 slots, 16 GiB, 100,000 ops, all fence epochs, autotuned
configuration, one CUDA graph per step): the digest of every 1 MiB block of
every slot equals the oracle's digest of that block (the oracle applies the
whole table to the seeded slot contents on the host), a seeded 1 % of the
blocks are compared byte by byte, and the counters are exact. MPSC streams
(1,024 producers, 16 consumers, 26 GB): every consumer's log passes the
interleaving-agnostic checker and every message's payload digest equals the
oracle's."""
import numpy as np
import pytest
import torch

import bench
from oracle import memcpy as om
from workloads import configs
from tests import fullsize_oracle as fo
from tests.gpu_util import device_bytes, h, inst  # noqa: F401

pytestmark = pytest.mark.gpu

BLOCK = fo.BLOCK
_MPSC_DIGESTS = {}  # oracle expectations shared by the parametrized cases of one process


@pytest.mark.parametrize("maker", ["batched", "batched_large"])
def test_full_size_every_block(h, inst, maker):
    seed = 0
    w = getattr(configs, maker)(seed)
    ids = bench.setup_slots(h, inst, w, seed)
    dops = bench.device_ops(bench.remap(w.ops, ids))
    torch.cuda.synchronize()
    bench.autotune(h, inst, dops, w.epochs)
    g = bench.capture_epochs(h, inst, dops, w.epochs)
    # the autotuner ran real batches: compare counter increments from here
    st, s0, r0 = h.hicr_slot_counters_range(inst, ids[0], len(ids))
    st, t0 = h.hicr_tag_counter(inst, 0)
    steps = 2
    for _ in range(steps):
        assert h.hicr_graph_launch(inst, g) == 0
        assert h.hicr_fence(inst, 0, bench.FENCE_TIMEOUT) == 0
    # a seeded 1 % of all blocks are compared byte by byte
    nblocks = [(int(sz) + BLOCK - 1) // BLOCK for sz in w.slot_sizes]
    every = [(s, b) for s in range(len(ids)) for b in range(nblocks[s])]
    rng = np.random.default_rng(321)
    full = {}
    for i in rng.choice(len(every), size=max(1, len(every) // 100), replace=False):
        s, b = every[int(i)]
        full.setdefault(s, []).append(b)
    exp = fo.batched_expectations(maker, seed, full)
    bad = []
    for s, sid in enumerate(ids):
        size = int(w.slot_sizes[s])
        dig, blocks = exp[s]
        for b in range(nblocks[s]):
            st, d = h.hicr_util_digest(inst, sid, b * BLOCK, min(BLOCK, size - b * BLOCK))
            assert st == 0
            if d != int(dig[b]):
                bad.append((s, b))
        st, ptr, _, _, _ = h.hicr_slot_info(inst, sid)
        for b, data in blocks.items():
            got = device_bytes(ptr + b * BLOCK, len(data)).cpu().numpy()
            diff = np.nonzero(got != data)[0]
            assert len(diff) == 0, f"slot {s} block {b}: {len(diff)} bytes differ, first at {diff[0]}"
    assert bad == [], f"{len(bad)} of {len(every)} block digests differ, first {bad[:5]}"
    assert len(every) == sum(nblocks) > 16000
    sent, recv = om.counters_from_ops(w.ops, len(ids))
    st, gs, gr = h.hicr_slot_counters_range(inst, ids[0], len(ids))
    assert st == 0
    assert (gs - s0 == steps * sent).all() and (gr - r0 == steps * recv).all()
    assert h.hicr_tag_counter(inst, 0) == (0, t0 + steps * len(w.ops))
    assert h.hicr_graph_destroy(inst, g) == 0


@pytest.mark.parametrize("batch", [256, 1024, 2048])
def test_spsc_full_size(h, inst, batch):
    """64 channels x capacity 4,096 x 64 B, 10^7 tokens per channel, at the
    hand-off batch sizes the bench chooses from: exact counts, capacity
    respected, and the whole-stream digest of every channel against the
    oracle's (the consumers also count words that differ from the payload
    rule: none may)."""
    w = configs.SpscWorkload()
    chans = [h.hicr_spsc_create(inst, w.token_bytes, w.capacity)[1] for _ in range(w.n_channels)]
    st, res = h.hicr_spsc_stream(inst, chans, w.tokens_per_channel, batch)
    assert st == 0
    for r in res:
        assert (r.pushed, r.popped, r.mismatches, r.status) == (w.tokens_per_channel,) * 2 + (0, 0)
        assert r.max_occupancy <= w.capacity
    if "spsc" not in _MPSC_DIGESTS:
        _MPSC_DIGESTS["spsc"] = fo.spsc_expectations(w.n_channels, w.tokens_per_channel)
    assert [r.digest for r in res] == _MPSC_DIGESTS["spsc"]


def _mpsc_oracle_digests(w):
    """[P, M] oracle digests of every message of the full-size workload
    (computed once per process)."""
    if "full" not in _MPSC_DIGESTS:
        _MPSC_DIGESTS["full"] = fo.mpsc_expectations(w.sizes)
    return _MPSC_DIGESTS["full"]


def _every_digest(w, logs, res):
    exp = _mpsc_oracle_digests(w)
    for c in range(w.n_consumers):
        n = int(res[c].consumed)
        L = logs[c][:n]
        p, q = L["producer"].astype(np.int64), L["seq"].astype(np.int64)
        bad = np.nonzero(L["digest"] != exp[p, q])[0]
        assert len(bad) == 0, f"consumer {c}: {len(bad)} of {n} payload digests differ, first entry {bad[0]}"


@pytest.mark.parametrize("ctas,group", [(1, 4), (4, 4), (5, 4), (5, 8)])
def test_mpsc_full_size(h, inst, ctas, group):
    """1,024 producers -> 16 consumers, 1,024 messages each (log-uniform
    8 B - 256 KiB), 1 GiB rings, 1 to 5 CTAs per consumer (the bench's
    launch shapes): every consumer's log passes the checker and every
    message's payload digest equals the oracle's."""
    from tests.test_gpu_channels import _check_mpsc
    w = configs.mpsc(0)
    run = bench.MpscRun(h, inst, w, group=group, consumer_ctas=ctas)
    st, res = run.run()
    assert st == 0
    assert sum(int(r.consumed) for r in res) == w.sizes.size
    logs = run.logs()
    _check_mpsc(w, logs, res, w.ring_bytes, sample=0.0)
    _every_digest(w, logs, res)
    run.free()


@pytest.mark.parametrize("ctas,group", [(1, 4), (4, 4), (5, 4), (5, 8)])
def test_mpsc_nonlocking_full_size(h, inst, ctas, group):
    """The same messages over 64 rings of 16 MiB per consumer (non-locking
    mode at the locking mode's memory), 1 to 5 CTAs per consumer: checker and
    every message's digest."""
    from tests.test_gpu_channels import _check_mpsc_nl
    w = configs.mpsc(0)
    run = bench.MpscRun(h, inst, w, group=group, nonlocking=True, consumer_ctas=ctas)
    st, res = run.run()
    assert st == 0
    assert sum(int(r.consumed) for r in res) == w.sizes.size
    _check_mpsc_nl(w, run, res, sample=0.0)
    _every_digest(w, run.logs(), res)
    run.free()


def test_serving_full_run_sampled(h, inst):
    """The serving configuration at full length: Poisson 20,000 req/s for
    60 s (about 1.2 M requests) on the bench's engine (64 GiB budget, 16
    channels), with the regions of a seeded sample of memcpy requests kept
    for checking (requests of 64 seeded templates of at most 32 MiB, drawn
    with the probability that keeps about 3 GiB spread over the whole run;
    at most 4 GiB). After the run: every burst request's digest (all of
    them) and every sampled memcpy request's digest equal the oracle's."""
    seed = 0
    src_w = configs.batched(seed)
    tmpl = configs.serve_templates(seed, src_w)
    ss = bench.ServeSetup(h, inst, src_w, tmpl, seed=seed)
    reqs = ss.requests(configs.serve_trace(seed, rate=20000.0, duration_s=60.0))
    rng = np.random.default_rng(55)
    small = np.nonzero(tmpl.region_bytes <= 32 << 20)[0]
    chosen = set(rng.choice(small, size=min(64, len(small)), replace=False).tolist())
    keep = np.zeros(len(reqs), dtype=np.uint8)
    kept_bytes = 0
    mine = (reqs["kind"] == 0) & np.isin(reqs["tmpl"], sorted(chosen))
    p = min(0.05, 3 * 2**30 / float(tmpl.region_bytes[reqs["tmpl"][mine]].sum()))
    draw = rng.random(len(reqs))
    for i in np.nonzero(mine & (draw < p))[0]:
        t = int(reqs["tmpl"][i])
        if t in chosen and kept_bytes + int(tmpl.region_bytes[t]) <= 4 << 30:
            keep[i] = 1
            kept_bytes += int(tmpl.region_bytes[t])
    assert keep.sum() > 100
    st, res, stats = h.hicr_serve_run_ex(inst, ss.srv, reqs, 0, int(180e9), keep=keep)
    assert st == 0 and stats.completed == len(reqs), (st, stats.as_dict(), h.hicr_last_error_string(inst))
    assert h.hicr_serve_digests(inst, ss.srv, reqs, res) == 0
    bexp = fo.burst_expectations(tmpl)
    burst = np.nonzero(reqs["kind"] == 1)[0]
    got = res["digest"][burst]
    want = np.array([bexp[int(t)] for t in reqs["tmpl"][burst]], dtype=np.uint64)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{len(bad)} of {len(burst)} burst digests differ, first request {burst[bad[0]]}"
    mexp = {}
    sampled = np.nonzero(keep)[0]
    for i in sampled:
        t = int(reqs["tmpl"][i])
        if t not in mexp:
            mexp[t] = fo.memcpy_template_digest(seed, tmpl, t)
        assert int(res["digest"][i]) == mexp[t], (i, t)
    print(f"serving 60 s: {len(reqs)} requests, {len(burst)} burst digests and {len(sampled)} sampled memcpy "
          f"regions ({kept_bytes / 2**30:.2f} GiB, {len(mexp)} templates) equal the oracle", flush=True)
    ss.free()