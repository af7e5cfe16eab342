#!/usr/bin/env python3
"""Benchmark of the GB300 HiCR communication path.

Headline (one JSON line on stdout): batched memcpy between memory slots --
256 HBM slots totalling 16 GiB (log-uniform 1-256 MiB, seeded bytes),
100,000 ops per batch, sizes log-uniform 16 B - 4 MiB, 10% unaligned
offsets, destinations disjoint within each of the fence epochs; one step =
one CUDA-graph replay of every epoch's batch (validate + plan + persistent
copy kernel) followed by fence(tag 0). value = algorithmic bytes (2n per op:
n read + n written) / device time, GB/s.

Side results in the same line: the large-segment case (1-4 MiB aligned ops),
the per-op cudaMemcpyAsync plain form, the end-to-end API call with host op
tables, SPSC/MPSC channel rates, and the CPU oracle baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import configs, splitmix  # noqa: E402

METRIC = "HiCR memcpy GB/s vs HBM peak; channel msgs/s; p99 latency vs per-op plain"
GiB = 1 << 30
MiB = 1 << 20
FENCE_TIMEOUT = 120_000_000_000


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-side", action="store_true", help="headline only (no plain/large/e2e/channels/CPU)")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU work for the oracle baseline")
    p.add_argument("--serve-seconds", type=float, default=60.0, help="length of the serving trace (0 = skip)")
    p.add_argument("--plain-serve-seconds", type=float, default=0.25,
                   help="prefix of the serving trace replayed through the per-op plain form")
    p.add_argument("--scale", type=float, default=1.0,
                   help="fraction of the batched workload (slots, bytes, ops); 1.0 = 16 GiB / 100,000 ops")
    p.add_argument("--profile-case", choices=["mpsc_small", "copy_small", "side_small", "control_small"], default=None,
                   help="run one small side case for a profiler capture, print its timings and exit")
    p.add_argument("--copy-scale", type=float, default=0.125,
                   help="copy_small: fraction of the batched workload to run (1.0 = the full 16 GiB / 100,000 ops)")
    p.add_argument("--batch-config", default=None,
                   help="JSON object of batch configuration fields: fixes the copy kernel's configuration "
                        "instead of autotuning (headline) or of the library default (copy_small)")
    return p.parse_args(argv)


def kernel_source_sha(sources):
    """sha256 over the text a kernel is compiled from: for each entry its file,
    or the part of it from the line starting with `begin` up to the line
    starting with `end` (exclusive)."""
    import hashlib
    hs = hashlib.sha256()
    for e in sources:
        text = open(os.path.join(ROOT, e["path"])).read()
        if e.get("begin"):
            lines = text.splitlines(keepends=True)
            a = next(i for i, l in enumerate(lines) if l.startswith(e["begin"]))
            b = next(i for i, l in enumerate(lines) if i > a and l.startswith(e["end"]))
            text = "".join(lines[a:b])
        hs.update(text.encode())
    return hs.hexdigest()


def copy_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch of the copy kernel: the DRAM-to-algorithmic ratio
    of its committed ncu capture (taken on the full-size workload, whose
    launches are the ones timed here) times the algorithmic bytes of a
    launch; None when there is no capture or the kernel's source changed
    since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    try:
        if kernel_source_sha(d["sources"]) != d["source_sha256"]:
            return None
    except (OSError, StopIteration, KeyError):
        return None
    return d["traffic_over_algorithmic"] * alg_bytes_per_launch


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# Workload set-up on the device (through the C ABI).
# ---------------------------------------------------------------------------
def remap(ops, ids):
    o = ops.copy()
    m = np.asarray(ids, dtype=np.uint32)
    o["dst"] = m[ops["dst"]]
    o["src"] = m[ops["src"]]
    return o


def scaled_batched(seed, scale=1.0, large=False):
    """The batched-memcpy workload, or a fraction of it (slots, bytes and ops
    scaled together; the size distributions are unchanged)."""
    if scale == 1.0:
        return configs.batched_large(seed) if large else configs.batched(seed)
    kw = dict(n_slots=max(8, int(round(256 * scale))), total_bytes=int(16 * GiB * scale) // 4096 * 4096,
              n_ops=max(100, int(100_000 * scale)))
    return configs.batched_large(seed, **kw) if large else configs.batched(seed, **kw)


def setup_slots(h, inst, w, seed):
    ids = []
    for s, sz in enumerate(w.slot_sizes):
        sid = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, int(sz), 0), "hicr_mem_alloc")
        h.check(h.hicr_util_fill(inst, sid, 0, int(sz), splitmix.fill_key_base(seed, s)), "fill")
        ids.append(sid)
    return ids


def device_ops(ops):
    import torch
    return torch.from_numpy(ops.view(np.uint8).copy()).cuda()


def capture_epochs(h, inst, dops, epochs):
    """One CUDA graph holding every epoch's device-validated batch in order."""
    h.check(h.hicr_batch_reserve(inst, max(b - a for a, b in epochs)), "reserve")
    h.check(h.hicr_graph_begin(inst), "graph_begin")
    for a, b in epochs:
        h.check(h.hicr_memcpy_batch_device(inst, dops.data_ptr() + 32 * a, b - a), "batch_device")
    return h.check(h.hicr_graph_end(inst), "graph_end")


def autotune(h, inst, dops, epochs, reps=3):
    a, b = max(epochs, key=lambda e: e[1] - e[0])
    st, cfg, ms = h.hicr_batch_autotune(inst, dops.data_ptr() + 32 * a, b - a, reps)
    h.check(st, "autotune")
    return cfg.as_dict(), ms


def time_graph(h, inst, stream, g, steps, warmup, prof=False, dist=None):
    """Device time of `steps` graph replays, each followed by fence(0)."""
    import torch
    for _ in range(warmup):
        h.check(h.hicr_graph_launch(inst, g), "graph_launch")
        h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
    copy_ms, launches = 0.0, 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0.record(stream)
    for _ in range(steps):
        h.check(h.hicr_graph_launch(inst, g), "graph_launch")
        h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
        if prof:
            ms, n = h.check(h.hicr_profile_read(inst), "profile_read")
            copy_ms += ms
            launches += n
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return e0.elapsed_time(e1), copy_ms, launches


# ---------------------------------------------------------------------------
# Channels.
# ---------------------------------------------------------------------------
class MpscRun:
    """Device set-up of an MPSC streaming run: staging slot with every
    message's seeded payload (16-byte aligned and packed, or `stage_gap`
    bytes apart), device size / offset tables, one channel per consumer and a
    device log."""

    def __init__(self, h, inst, w, group=4, nonlocking=False, consumer_ctas=1, ring_bytes=None, max_msgs=None,
                 stage_gap=None):
        import torch
        self.h, self.inst, self.w, self.group = h, inst, w, group
        self.nonlocking, self.consumer_ctas = nonlocking, consumer_ctas
        P, M = w.sizes.shape
        C = w.n_consumers
        sizes = w.sizes.reshape(-1).astype(np.uint64)
        if stage_gap is None:  # packed, each payload 16-byte aligned
            padded = ((sizes + np.uint64(15)) // np.uint64(16)) * np.uint64(16)
        else:  # `stage_gap` bytes between payloads: arbitrary alignments
            padded = sizes + np.uint64(stage_gap)
        offs = np.zeros(len(sizes), dtype=np.uint64)
        offs[1:] = np.cumsum(padded)[:-1]
        self.staging_bytes = max(int(padded.sum()), 16)
        self.offs = offs
        self.staging = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, self.staging_bytes), "staging")
        self.capture = None
        p = np.repeat(np.arange(P, dtype=np.uint64), M)
        q = np.tile(np.arange(M, dtype=np.uint64), P)
        keys = (np.uint64(1) << np.uint64(63)) | (p << np.uint64(40)) | (q << np.uint64(16))
        seg = np.stack([offs, sizes, keys], 1).astype(np.uint64)
        d_seg = torch.from_numpy(seg.view(np.int64).copy()).cuda()
        h.check(h.hicr_util_fill_segments(inst, self.staging, d_seg.data_ptr(), len(sizes)), "fill_segments")
        self.d_sizes = torch.from_numpy(sizes.view(np.int64).copy()).cuda()
        self.d_offs = torch.from_numpy(offs.view(np.int64).copy()).cuda()
        per = -(-P // C)
        self.stride = per * M
        self.d_log = torch.empty(C * self.stride * 32, dtype=torch.uint8, device="cuda")
        self.chans = []
        self.set_mode(nonlocking, consumer_ctas, ring_bytes, max_msgs)
        torch.cuda.synchronize()
        del d_seg

    def set_mode(self, nonlocking, consumer_ctas=1, ring_bytes=None, max_msgs=None):
        """(Re)create the channels: locking mode with one shared ring per
        consumer, or non-locking mode with one ring per producer (by default
        the locking ring and metadata capacity split evenly, so both modes
        hold the same memory)."""
        h, w = self.h, self.w
        per = -(-w.sizes.shape[0] // w.n_consumers)
        for c in self.chans:
            h.check(h.hicr_channel_destroy(self.inst, c), "channel_destroy")
        self.nonlocking, self.consumer_ctas = nonlocking, consumer_ctas
        self.ring_bytes = ring_bytes or (w.ring_bytes // per if nonlocking else w.ring_bytes)
        self.max_msgs = max_msgs or (max(w.max_msgs // per, 1) if nonlocking else w.max_msgs)
        create = h.hicr_mpsc_nl_create if nonlocking else h.hicr_mpsc_create
        self.chans = [h.check(create(self.inst, per, self.ring_bytes, self.max_msgs), "mpsc_create")
                      for _ in range(w.n_consumers)]

    def run(self, timeout_ns=60_000_000_000, capture=False):
        """One streaming run. With capture=True the consumers also copy every
        message they consumed into ``self.capture`` (zeroed first), message
        (p, s) at the same offset as its staged payload."""
        import torch
        P, M = self.w.sizes.shape
        kw = {}
        if capture:
            self.capture = torch.zeros(self.staging_bytes, dtype=torch.uint8, device="cuda")
            kw = dict(d_capture=self.capture.data_ptr(), d_cap_off=self.d_offs.data_ptr())
        if self.nonlocking:
            return self.h.hicr_mpsc_nl_stream(self.inst, self.chans, P, M, self.d_sizes.data_ptr(),
                                              self.d_offs.data_ptr(), self.staging, self.group, self.consumer_ctas,
                                              self.d_log.data_ptr(), self.stride, timeout_ns, **kw)
        return self.h.hicr_mpsc_stream(self.inst, self.chans, P, M, self.d_sizes.data_ptr(), self.d_offs.data_ptr(),
                                       self.staging, self.group, self.consumer_ctas, self.d_log.data_ptr(),
                                       self.stride, timeout_ns, **kw)

    def logs(self):
        a = self.d_log.cpu().numpy().view(self.h.MPSC_LOG_DTYPE)
        return a.reshape(self.w.n_consumers, self.stride)

    def free(self):
        for c in self.chans:
            self.h.check(self.h.hicr_channel_destroy(self.inst, c), "channel_destroy")
        self.h.check(self.h.hicr_mem_free(self.inst, self.staging), "mem_free")
        self.chans = []
        self.capture = None


def bench_spsc(h, inst, reps=3):
    """64 SPSC channels x 4,096 tokens of 64 B, 10^7 tokens per channel."""
    w = configs.SpscWorkload()
    chans = [h.check(h.hicr_spsc_create(inst, w.token_bytes, w.capacity), "spsc_create") for _ in range(w.n_channels)]
    # tokens per head/tail update: pick the fastest on a tenth of the stream
    tune = {}
    for b in (256, 512, 1024, 2048):
        t0 = time.perf_counter()
        h.check(h.hicr_spsc_stream(inst, chans, w.tokens_per_channel // 10, b)[0], "spsc tune")
        tune[b] = time.perf_counter() - t0
    batch = min(tune, key=tune.get)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        st, res = h.hicr_spsc_stream(inst, chans, w.tokens_per_channel, batch)
        times.append(time.perf_counter() - t0)
        h.check(st, "spsc_stream")
        assert all(r.mismatches == 0 and r.popped == w.tokens_per_channel for r in res)
    t = statistics.median(times)
    tokens = w.n_channels * w.tokens_per_channel
    # the same payload rule with consumers that only digest (no per-word
    # check): the channel's rate without the checker's arithmetic; the run's
    # digests must equal those of the checked run, channel by channel
    dtune = {}
    for b in (256, 512, 1024, 2048):
        t0 = time.perf_counter()
        h.check(h.hicr_spsc_stream_ex(inst, chans, w.tokens_per_channel // 10, b, flags=h.HICR_SPSC_DIGEST_ONLY)[0],
                "spsc digest-only tune")
        dtune[b] = time.perf_counter() - t0
    dbatch = min(dtune, key=dtune.get)
    dtimes = []
    for _ in range(reps):
        t0 = time.perf_counter()
        st, dres = h.hicr_spsc_stream_ex(inst, chans, w.tokens_per_channel, dbatch, flags=h.HICR_SPSC_DIGEST_ONLY)
        dtimes.append(time.perf_counter() - t0)
        h.check(st, "spsc_stream digest-only")
        assert all(x.popped == w.tokens_per_channel for x in dres)
    same = all(x.digest == y.digest for x, y in zip(dres, res))
    td = statistics.median(dtimes)
    # the channel as the paper defines a push (a copy from a memory slot into
    # the consumer's ring): producers copy staged tokens (4,096 per channel,
    # 16 MiB in all), consumers only digest
    staged = w.capacity
    stg = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, w.n_channels * staged * w.token_bytes), "staging")
    h.check(h.hicr_util_fill(inst, stg, 0, w.n_channels * staged * w.token_bytes, splitmix.fill_key_base(0, 77)),
            "fill staging")
    # tokens per head/tail update for this form, tuned the same way
    ctune = {}
    for b in (256, 512, 1024, 2048):
        t0 = time.perf_counter()
        h.check(h.hicr_spsc_stream_ex(inst, chans, w.tokens_per_channel // 10, b, src=stg, src_tokens=staged)[0],
                "spsc copy tune")
        ctune[b] = time.perf_counter() - t0
    cbatch = min(ctune, key=ctune.get)
    ctimes = []
    for r in range(reps + 1):
        t0 = time.perf_counter()
        st, res = h.hicr_spsc_stream_ex(inst, chans, w.tokens_per_channel, cbatch, src=stg, src_tokens=staged)
        if r:
            ctimes.append(time.perf_counter() - t0)
        h.check(st, "spsc_stream copy")
        assert all(x.popped == w.tokens_per_channel for x in res)
    for c in chans:
        h.check(h.hicr_channel_destroy(inst, c), "channel_destroy")
    tc = statistics.median(ctimes)
    # the L2 bound: this library's copy-loop probe over a 16 MiB working set
    # (8 MiB copied into 8 MiB, passes repeated), best of 2, 4 and 8 CTAs per
    # SM; and the same probe on as many SMs as the channels' producers hold
    # (one CTA each), the rate the producer side can reach
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    l2 = 0.0
    for per in (2, 4, 8):
        ns = h.check(h.hicr_util_copy_loop(inst, stg, 8 * MiB, stg, 0, 8 * MiB, 2000, per * sms), "copy loop")
        l2 = max(l2, 2 * 8 * MiB * 2000 / ns)
    ns = h.check(h.hicr_util_copy_loop(inst, stg, 8 * MiB, stg, 0, 8 * MiB, 500, w.n_channels), "copy loop")
    l2_prod = 2 * 8 * MiB * 500 / ns
    h.check(h.hicr_mem_free(inst, stg), "free staging")
    return {"workload": "64 channels x capacity 4,096 x 64 B tokens, 10^7 tokens/channel, "
                        "1 producer + 1 consumer CTA per channel (cooperative grid)", "batch_tokens": batch,
            "msgs_per_s": tokens / t, "GB_per_s": tokens * 128 / t / 1e9, "s_per_run": t,
            "frac_of_hbm_peak": tokens * 128 / t / 1e9 / peaks()[0],
            "bound": "the consumers' SplitMix64 verification of every word (rings total 16 MiB, L2-resident: "
                     "the HBM fraction is context only)",
            "digest_only": {"msgs_per_s": tokens / td, "s_per_run": td, "batch_tokens": dbatch,
                            "digests_equal_checked_run": same,
                            "note": "payload-rule producers, consumers that digest without checking each word"},
            "copy_producers": {
                "workload": "the same channels; producers copy staged tokens (token s of a channel = staged token "
                            "s mod 4,096; 16 MiB staged in all) into the ring, consumers digest only",
                "msgs_per_s": tokens / tc, "s_per_run": tc, "batch_tokens": cbatch,
                "l2_GB_per_s": tokens * 192 / tc / 1e9,
                "l2_bytes_per_token": 192,
                "l2_copy_bound_GB_per_s": l2,
                "frac_of_l2_copy_bound": tokens * 192 / tc / 1e9 / l2,
                "producer_l2_GB_per_s": tokens * 128 / tc / 1e9,
                "l2_copy_bound_on_producer_sms_GB_per_s": l2_prod,
                "producer_frac_of_that_bound": tokens * 128 / tc / 1e9 / l2_prod,
                "note": "L2 traffic per token: staged read 64 B + ring write 64 B (producer SM) + ring read 64 B "
                        "(consumer SM); bounds = hicr_util_copy_loop's read+write rate over an L2-resident 16 MiB "
                        f"working set on the whole GPU ({sms} SMs x 2-8 CTAs) and on {w.n_channels} CTAs, one SM "
                        "each, as many as the producers hold"}}


def bench_pingpong(h, inst):
    """Test Case 1 on one GPU: goodput G(s) and one-way time over two opposing
    single-message SPSC channels, 1 B - 2 GiB, 10 timed round trips each."""
    top = 2 << 30
    sid = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, top), "alloc")
    h.check(h.hicr_util_fill(inst, sid, 0, top, splitmix.fill_key_base(0, 999)), "fill")
    rows = []
    for nbytes in [1 << e for e in range(0, 31, 3)] + [top]:
        best = None
        reps = 1000 if nbytes <= (1 << 20) else 10  # enough timed round trips for microsecond trips
        for ctas in (1, 4, 16, 38, 76, 152):  # a quarter, half, one, two CTAs per SM per agent at the top
            st, r = h.hicr_pingpong(inst, sid, 0, nbytes, reps, 2, ctas)
            if st == h.HICR_ERR_INVALID:  # both agents would not be co-resident
                continue
            h.check(st, "pingpong")
            if best is None or r.half_rtt_ns < best[1].half_rtt_ns:
                best = (ctas, r)
        ctas, r = best
        rows.append({"bytes": nbytes, "ctas_per_side": ctas, "reps": reps, "one_way_us": r.half_rtt_ns / 1e3,
                     "goodput_GB_per_s": r.goodput_gbs})
    h.check(h.hicr_mem_free(inst, sid), "free")
    return {"workload": "ping-pong over two opposing capacity-1 SPSC channels (paper Test Case 1), "
                        "1,000 timed round trips up to 1 MiB and 10 above (the paper's count), after 2 warm-up; "
                        "per size the fastest agent width of 1, 4, 16, 38, 76, 152 CTAs", "curve": rows}


# NVIDIA's nominal NVLink-C2C bandwidth between Grace and the GPU: 900 GB/s in
# both directions together, 450 GB/s each way (context for the host space;
# the measured probes are the practical bound).
NOMINAL_C2C_GBS = 450.0


def bench_host_space(h, inst, nbytes=4 * GiB, op_bytes=4 * MiB, reps=5):
    """Copies between HBM and page-locked Grace memory (the host memory
    space) through the copy kernels over NVLink-C2C: 4 GiB per direction in
    4 MiB ops, one device-resident batch + fence per repetition; beside it
    the copy engine (torch copy_ of a pinned tensor, cudaMemcpyAsync) on the
    same bytes."""
    import torch
    h.check(h.hicr_set_host_copies(inst, 1), "host copies on")
    d = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, nbytes), "alloc hbm")
    hs = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HOST, nbytes), "alloc host")
    h.check(h.hicr_util_fill(inst, d, 0, nbytes, splitmix.fill_key_base(0, 1)), "fill")
    h.check(h.hicr_util_fill(inst, hs, 0, nbytes, splitmix.fill_key_base(0, 2)), "fill")
    k = nbytes // op_bytes
    offs = np.arange(k, dtype=np.uint64) * np.uint64(op_bytes)
    out = {"workload": f"{nbytes >> 30} GiB per direction in {op_bytes >> 20} MiB ops, batch + fence"}
    for name, dst, src in (("hbm_to_host", hs, d), ("host_to_hbm", d, hs)):
        ops = configs.make_ops([dst] * k, [src] * k, offs, offs, [op_bytes] * k)
        t = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        times = []
        for r in range(reps + 1):
            t0 = time.perf_counter()
            h.check(h.hicr_memcpy_batch_device(inst, t.data_ptr(), k), "batch")
            h.check(h.hicr_fence(inst, 0), "fence")
            if r:
                times.append(time.perf_counter() - t0)
        out[name + "_GB_per_s"] = nbytes / statistics.median(times) / 1e9
    # the link's practical one-way rates: this library's streaming probes
    # reading, then writing, the host slot from every SM (best of 2, 4, 8 CTAs
    # per SM), and its copy loop between the two spaces
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    probes = {}
    for name, write in (("read_host", 0), ("write_host", 1)):
        best = 0.0
        for per in (2, 4, 8):
            ns = h.check(h.hicr_util_stream(inst, hs, 0, nbytes, write, 1, per * sms), "stream probe")
            best = max(best, nbytes / ns)
        probes[name + "_GB_per_s"] = best
    for name, dst, src in (("copy_loop_hbm_to_host", hs, d), ("copy_loop_host_to_hbm", d, hs)):
        best = 0.0
        for per in (2, 4, 8):
            ns = h.check(h.hicr_util_copy_loop(inst, dst, 0, src, 0, nbytes, 1, per * sms), "copy loop")
            best = max(best, nbytes / ns)
        probes[name + "_GB_per_s"] = best
    # both directions at once: a copy inside the host slot reads and writes
    # the link together (the bytes crossing it, both ways, per second)
    best = 0.0
    for per in (2, 4, 8):
        ns = h.check(h.hicr_util_copy_loop(inst, hs, nbytes // 2, hs, 0, nbytes // 2, 1, per * sms), "copy loop")
        best = max(best, nbytes / ns)
    probes["copy_loop_host_to_host_both_ways_GB_per_s"] = best
    out["link_probes"] = probes
    out["nominal_c2c_GB_per_s_per_direction"] = NOMINAL_C2C_GBS
    out["frac_of_probe"] = {"hbm_to_host": out["hbm_to_host_GB_per_s"] / probes["write_host_GB_per_s"],
                            "host_to_hbm": out["host_to_hbm_GB_per_s"] / probes["read_host_GB_per_s"]}
    out["frac_of_nominal"] = {"hbm_to_host": out["hbm_to_host_GB_per_s"] / NOMINAL_C2C_GBS,
                              "host_to_hbm": out["host_to_hbm_GB_per_s"] / NOMINAL_C2C_GBS}
    h.check(h.hicr_set_host_copies(inst, 0), "host copies off")
    h.check(h.hicr_mem_free(inst, hs), "free")
    h.check(h.hicr_mem_free(inst, d), "free")
    ph = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    dv = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    for name, a, b in (("copy_engine_hbm_to_host_GB_per_s", ph, dv), ("copy_engine_host_to_hbm_GB_per_s", dv, ph)):
        times = []
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a.copy_(b, non_blocking=True)
            torch.cuda.synchronize()
            if r:
                times.append(time.perf_counter() - t0)
        out[name] = nbytes / statistics.median(times) / 1e9
    del ph, dv
    return out


def bench_latencies(h, inst, reps=2000):
    """Host-observed latency (median and p99 over `reps` calls, microseconds)
    of the small synchronous operations: a 16-byte memcpy + fence (also in
    latency mode, where a persistent server kernel takes the copy), an
    execution-unit launch + await (the built-in fill on 16 bytes), a Data
    Object get (16 bytes) + fence, and a 1-token SPSC host push + pop (also in
    latency mode, where the server takes the channel calls). Python's
    garbage collector is off while the calls are timed."""
    import ctypes as C

    def stats(f):
        for _ in range(50):
            f()
        ts = []
        gc_was = gc.isenabled()
        gc.disable()  # as timeit does: a collection inside a call is not the library's latency
        try:
            for _ in range(reps):
                t0 = time.perf_counter()
                f()
                ts.append(time.perf_counter() - t0)
        finally:
            if gc_was:
                gc.enable()
        ts = np.asarray(ts) * 1e6
        return {"p50_us": float(np.percentile(ts, 50)), "p99_us": float(np.percentile(ts, 99))}

    a = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 1 << 20), "alloc")
    b = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 1 << 20), "alloc")
    out = {}

    def memcpy_fence():
        h.check(h.hicr_memcpy(inst, b, 0, a, 0, 16), "memcpy")
        h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
    out["memcpy_16B_plus_fence"] = stats(memcpy_fence)
    h.check(h.hicr_set_latency_mode(inst, 2000), "latency mode on")
    out["memcpy_16B_plus_fence_latency_mode"] = stats(memcpy_fence)
    h.check(h.hicr_set_latency_mode(inst, 0), "latency mode off")

    unit = h.check(h.hicr_exec_unit_builtin("fill_seeded"), "exec_unit")
    ptr = h.check(h.hicr_slot_info(inst, a), "slot_info")[0]
    pu = h.check(h.hicr_pu_create(inst), "pu")
    args = [C.c_void_p(ptr), C.c_uint64(0), C.c_uint64(16), C.c_uint64(1)]

    def launch_await():
        e = h.check(h.hicr_exec_launch(inst, pu, unit, args), "exec_launch")
        h.check(h.hicr_exec_await(inst, e, FENCE_TIMEOUT), "exec_await")
    out["exec_launch_plus_await"] = stats(launch_await)
    h.check(h.hicr_pu_destroy(inst, pu), "pu_destroy")

    oid = h.check(h.hicr_dobj_publish(inst, a, 64, 16), "publish")
    hd = h.check(h.hicr_dobj_get_handle(inst, oid), "get_handle")

    def dobj_get():
        h.check(h.hicr_dobj_get(inst, hd, b, 128), "dobj_get")
        h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
    out["dobj_get_16B_plus_fence"] = stats(dobj_get)
    h.check(h.hicr_dobj_release(inst, oid), "release")

    ch = h.check(h.hicr_spsc_create(inst, 64, 4096), "spsc_create")

    def push_pop():
        h.check(h.hicr_channel_push(inst, ch, 0, a, 0, 1), "push")
        h.check(h.hicr_channel_pop(inst, ch, 1), "pop")
    out["spsc_host_push_plus_pop"] = stats(push_pop)
    h.check(h.hicr_set_latency_mode(inst, 2000), "latency mode on")
    out["spsc_host_push_plus_pop_latency_mode"] = stats(push_pop)
    h.check(h.hicr_set_latency_mode(inst, 0), "latency mode off")
    h.check(h.hicr_channel_destroy(inst, ch), "destroy")
    for sid in (a, b):
        h.check(h.hicr_mem_free(inst, sid), "free")
    out["reps"] = reps
    out["from_c"] = latency_from_c(reps)
    return out


def latency_from_c(reps=2000):
    """The same small operations timed from C through the C ABI only
    (paper_2509_01425_gb300/hicr_latency): no interpreter on the path."""
    from paper_2509_01425_gb300 import build
    exe = build.LATENCY_BIN
    if not os.path.exists(exe):
        build.build_latency_tool()
    r = subprocess.run([exe, str(torch_device_index()), str(reps)], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"hicr_latency failed: {r.stderr.strip()}")
    d = json.loads(r.stdout)
    d["reps"] = reps
    return d


def torch_device_index():
    import torch
    return torch.cuda.current_device()


def _time_mpsc(h, run, reps):
    h.check(run.run()[0], "mpsc warm-up")
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        st, res = run.run()
        times.append(time.perf_counter() - t0)
        h.check(st, "mpsc_stream")
    cap_ok = all(int(r.max_inflight_bytes) <= run.ring_bytes and int(r.max_inflight_msgs) <= run.max_msgs
                 for r in res)
    t = statistics.median(times)
    return {"msgs_per_s": run.w.sizes.size / t, "payload_GB_per_s": run.w.total_bytes / t / 1e9,
            "algorithmic_GB_per_s": 3 * run.w.total_bytes / t / 1e9, "s_per_run": t, "capacity_respected": cap_ok}


def bench_mpsc(h, inst, reps=3, groups=(4, 8)):
    """1,024 producers -> 16 consumers, log-uniform 8 B - 256 KiB: locking
    mode over one 1 GiB ring per consumer against non-locking mode over 64
    rings of 16 MiB per consumer (the same memory), both with 1 to 5 CTAs per
    consumer (the producer warps spread over the SMs left free) and
    reservation groups of 4 or 8 messages; the fastest shape is reported."""
    w = configs.mpsc(0)
    run = MpscRun(h, inst, w)

    def sweep(nonlocking):
        res = {}
        for g in (1, 2, 3, 4, 5):
            for grp in groups:
                run.group = grp
                run.set_mode(nonlocking, g)
                if run.run()[0] == h.HICR_ERR_INVALID:  # grid not co-resident on this GPU
                    continue
                res[(g, grp)] = _time_mpsc(h, run, reps)
        best = max(res, key=lambda k: res[k]["msgs_per_s"])
        return {**res[best], "consumer_ctas": best[0], "group": best[1],
                "msgs_per_s_by_consumer_ctas_and_group": {f"{g}x{grp}": r["msgs_per_s"] for (g, grp), r in res.items()}}

    out = {"workload": "1,024 producers -> 16 consumers, 1,024 msgs each, log-uniform 8 B-256 KiB, 1 GiB rings",
           **sweep(False)}
    nl = sweep(True)
    out["nonlocking"] = {"rings": f"64 x {run.ring_bytes >> 20} MiB per consumer, {run.max_msgs} msgs each", **nl}
    run.free()
    return out


# ---------------------------------------------------------------------------
# Serving.
# ---------------------------------------------------------------------------
class ServeSetup:
    """Source slots of a batched workload (its source half only), request
    templates, the burst staging slot and a serving engine."""

    def __init__(self, h, inst, src_w, tmpl, seed=0, budget=64 * GiB, n_channels=16, ring_bytes=1 * GiB,
                 max_msgs=65536, chunk_bytes=128 << 10, op_cost_bytes=4096, verify=False):
        import torch
        self.h, self.inst, self.tmpl = h, inst, tmpl
        self.slot_of = {}
        for s in np.asarray(src_w.src_slots):
            sz = int(src_w.slot_sizes[s])
            sid = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, sz, 0), "alloc source")
            h.check(h.hicr_util_fill(inst, sid, 0, sz, splitmix.fill_key_base(seed, int(s))), "fill source")
            self.slot_of[int(s)] = sid
        cfg = dict(budget_bytes=budget, n_channels=n_channels, max_msgs=max_msgs, ring_bytes=ring_bytes,
                   chunk_bytes=chunk_bytes, op_cost_bytes=op_cost_bytes, verify=1 if verify else 0)
        self.srv = h.check(h.hicr_serve_create(inst, cfg), "serve_create")
        # memcpy templates
        m = np.vectorize(self.slot_of.get, otypes=[np.uint32])
        for t in range(len(tmpl.region_bytes)):
            a, b = int(tmpl.op_start[t]), int(tmpl.op_start[t + 1])
            ops = tmpl.ops[a:b].copy()
            ops["src"] = m(ops["src"])
            h.check(h.hicr_serve_add_memcpy_template(inst, self.srv, ops, int(tmpl.region_bytes[t])), "memcpy tmpl")
        # burst staging: message m of template t = MPSC payload (producer t, seq m)
        sizes = tmpl.msg_sizes.astype(np.uint64)
        padded = ((sizes + np.uint64(15)) // np.uint64(16)) * np.uint64(16)
        offs = np.zeros(len(sizes), dtype=np.uint64)
        offs[1:] = np.cumsum(padded)[:-1]
        self.staging_bytes = max(int(padded.sum()), 16)
        self.offs = offs
        self.staging = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, self.staging_bytes), "staging")
        self.capture = None
        nt = len(tmpl.msg_start) - 1
        tt = np.repeat(np.arange(nt, dtype=np.uint64), np.diff(tmpl.msg_start))
        mm = np.concatenate([np.arange(c, dtype=np.uint64) for c in np.diff(tmpl.msg_start)])
        keys = (np.uint64(1) << np.uint64(63)) | (tt << np.uint64(40)) | (mm << np.uint64(16))
        seg = np.stack([offs, sizes, keys], 1).astype(np.uint64)
        d_seg = torch.from_numpy(seg.view(np.int64).copy()).cuda()
        h.check(h.hicr_util_fill_segments(inst, self.staging, d_seg.data_ptr(), len(sizes)), "fill staging")
        for t in range(nt):
            a, b = int(tmpl.msg_start[t]), int(tmpl.msg_start[t + 1])
            h.check(h.hicr_serve_add_burst_template(inst, self.srv, sizes[a:b], offs[a:b], self.staging), "burst tmpl")
        torch.cuda.synchronize()
        del d_seg

    def requests(self, trace):
        r = np.zeros(len(trace.arrival_ns), dtype=self.h.SERVE_REQ_DTYPE)
        r["arrival_ns"] = trace.arrival_ns
        r["kind"] = trace.kind
        r["tmpl"] = trace.template
        return r

    def free(self):
        h, inst = self.h, self.inst
        h.check(h.hicr_serve_destroy(inst, self.srv), "serve_destroy")
        h.check(h.hicr_mem_free(inst, self.staging), "free staging")
        for sid in self.slot_of.values():
            h.check(h.hicr_mem_free(inst, sid), "free source")


def latency_summary(res, mask=None):
    lat = res["latency_ns"] if mask is None else res["latency_ns"][mask]
    if len(lat) == 0:
        return {}
    return {"p50_us": float(np.percentile(lat, 50)) / 1e3, "p99_us": float(np.percentile(lat, 99)) / 1e3,
            "mean_us": float(lat.mean()) / 1e3, "max_us": float(lat.max()) / 1e3}


def stall_summary(res, stats, watch=None):
    """Where the longest pause of a serving run happened: the host's longest
    interval between two passes of its admission/completion loop, the longest
    interval between two consecutive completions on the device clock, and
    (`watch`, a HostPauseWatch) the pauses that a second host thread, which
    only sleeps 1 ms at a time, saw meanwhile. A pause seen by both host
    threads at once was the whole host process not running."""
    dev = np.sort(res["device_done_ns"][res["device_done_ns"] > 0].astype(np.int64))
    gap = np.diff(dev)
    out = {"host_max_poll_gap_ms": stats.max_poll_gap_ns / 1e6,
           "host_max_poll_gap_at_s": stats.max_poll_gap_at_ns / 1e9,
           "device_max_completion_gap_ms": float(gap.max()) / 1e6 if len(gap) else None,
           "device_max_completion_gap_at_s": float(dev[int(np.argmax(gap)) + 1] - dev[0]) / 1e9 if len(gap) else None}
    if watch is not None:
        out.update(watch.summary())
    return out


class HostPauseWatch:
    """A thread that sleeps 1 ms at a time and records every wake-up later
    than `over_ms`, with the guest kernel's steal time over the same span."""

    def __init__(self, over_ms=10.0):
        import threading
        self.over = over_ms / 1e3
        self.pauses = []
        self._stop = threading.Event()
        self._t0 = time.monotonic()
        self._steal0 = _steal_ticks()
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()

    def _run(self):
        last = time.monotonic()
        while not self._stop.is_set():
            time.sleep(0.001)
            t = time.monotonic()
            if t - last > self.over:
                self.pauses.append((round(last - self._t0, 3), round((t - last) * 1e3, 1)))
            last = t

    def summary(self):
        self._stop.set()
        self._th.join(timeout=1.0)
        steal = _steal_ticks()
        tck = os.sysconf("SC_CLK_TCK")
        return {"second_thread_pause_threshold_ms": self.over * 1e3,
                "second_thread_pauses_s_ms": self.pauses[:20],
                "guest_steal_ms": (steal - self._steal0) * 1e3 / tck
                if steal is not None and self._steal0 is not None else None}


def _steal_ticks():
    """The guest kernel's steal time over all CPUs (/proc/stat), in ticks."""
    try:
        with open("/proc/stat") as f:
            parts = f.readline().split()
        return int(parts[8]) if parts[0] == "cpu" and len(parts) > 8 else None
    except (OSError, ValueError):
        return None


def bench_serve(h, inst, seconds=60.0, plain_seconds=1.0, seed=0):
    """Config 5: Poisson 20,000 req/s, 70% memcpy batches of log-uniform 1-4,096
    ops (16 B-4 MiB) over config 2's source slots, 30% MPSC bursts of
    log-uniform 1-512 messages (8 B-256 KiB), 64 GiB budget (16 x 1 GiB rings +
    48 GiB destination arena)."""
    src_w = configs.batched(seed)
    tmpl = configs.serve_templates(seed, src_w)
    ss = ServeSetup(h, inst, src_w, tmpl, seed=seed)
    tr = configs.serve_trace(seed, rate=20000.0, duration_s=seconds)
    reqs = ss.requests(tr)
    watch = HostPauseWatch()
    st, res, stats = h.hicr_serve_run(inst, ss.srv, reqs, 0, int((seconds + 120) * 1e9))
    h.check(st, "serve_run")
    out = {"workload": f"Poisson 20,000 req/s for {seconds:g} s ({len(reqs):,} requests): 70% memcpy batches of "
                       "log-uniform 1-4,096 ops (16 B-4 MiB), 30% MPSC bursts of log-uniform 1-512 msgs "
                       "(8 B-256 KiB); 64 GiB budget = 16 x 1 GiB rings + 48 GiB arena",
           "requests": int(stats.completed), "wall_s": stats.wall_ns / 1e9,
           "GB_per_s_moved": stats.bytes_moved / (stats.wall_ns / 1e9) / 1e9,
           "algorithmic_GB_per_s": (2 * (stats.bytes_moved - stats.burst_bytes) + 3 * stats.burst_bytes)
           / (stats.wall_ns / 1e9) / 1e9,
           "req_per_s": stats.completed / (stats.wall_ns / 1e9),
           "max_inflight": int(stats.max_inflight), "arena_high_water_GB": stats.max_region_bytes / 1e9,
           "latency_all": latency_summary(res), "latency_memcpy": latency_summary(res, reqs["kind"] == 0),
           "latency_burst": latency_summary(res, reqs["kind"] == 1),
           "stalls": stall_summary(res, stats, watch)}
    # the plain form on the first plain_seconds of the same trace
    hz = int(plain_seconds * 1e9)
    st, pres, pst = h.hicr_serve_run_plain(inst, ss.srv, reqs, hz, int((plain_seconds + 600) * 1e9))
    h.check(st, "serve_run_plain")
    m = reqs["arrival_ns"] <= hz
    out["plain_form"] = {"horizon_s": plain_seconds, "requests": int(pst.completed),
                         "wall_s": pst.wall_ns / 1e9, "GB_per_s_moved": pst.bytes_moved / (pst.wall_ns / 1e9) / 1e9,
                         "latency_all": latency_summary(pres[: int(m.sum())]),
                         "engine_latency_same_requests": latency_summary(res[: int(m.sum())])}
    out["rate_sweep"] = serve_rate_sweep(h, inst, ss, seed)
    ss.free()
    return out


SERVE_P99_BOUND_MS = 50.0


def serve_rate_sweep(h, inst, ss, seed=0, engine_rates=(15000, 20000, 25000, 30000, 40000), engine_s=3.0,
                     plain_rates=(100, 200, 400, 800), plain_s=2.0):
    """Each form's highest sustainable arrival rate: the highest swept Poisson
    rate (same request mix) whose p99 latency stays within
    SERVE_P99_BOUND_MS over a short trace."""
    def sweep(rates, seconds, plain):
        rows = []
        for r in rates:
            reqs = ss.requests(configs.serve_trace(seed + 1, rate=float(r), duration_s=seconds))
            if plain:
                st, res, stats = h.hicr_serve_run_plain(inst, ss.srv, reqs, int(seconds * 1e9),
                                                        int((seconds + 600) * 1e9))
            else:
                st, res, stats = h.hicr_serve_run(inst, ss.srv, reqs, 0, int((seconds + 120) * 1e9))
            h.check(st, "serve sweep")
            n = int((reqs["arrival_ns"] <= int(seconds * 1e9)).sum())
            lat = latency_summary(res[:n])
            wall = stats.wall_ns / 1e9
            alg = 2 * (stats.bytes_moved - stats.burst_bytes) + 3 * stats.burst_bytes
            rows.append({"rate": r, "requests": n, "p50_us": lat.get("p50_us"), "p99_us": lat.get("p99_us"),
                         "GB_per_s_moved": stats.bytes_moved / wall / 1e9,
                         "algorithmic_GB_per_s": alg / wall / 1e9,
                         "frac_of_hbm_peak": alg / wall / 1e9 / peaks()[0],
                         "sustainable": bool(n and lat["p99_us"] <= SERVE_P99_BOUND_MS * 1e3)})
        ok = [x["rate"] for x in rows if x["sustainable"]]
        return rows, (max(ok) if ok else None)

    eng, eng_max = sweep(engine_rates, engine_s, False)
    pl, pl_max = sweep(plain_rates, plain_s, True)
    return {"p99_bound_ms": SERVE_P99_BOUND_MS, "engine_seconds_per_rate": engine_s,
            "plain_seconds_per_rate": plain_s, "engine": eng, "engine_max_sustainable_req_per_s": eng_max,
            "plain": pl, "plain_max_sustainable_req_per_s": pl_max,
            "note": "null = not sustainable at the lowest swept rate"}


# ---------------------------------------------------------------------------
# CPU oracle baseline: the oracle as it stands on a bounded sample.
# ---------------------------------------------------------------------------
CPU_SAMPLE = dict(n_slots=32, total_bytes=2 * GiB, slot_lo=1 << 20, slot_hi=256 << 20, n_ops=12_500)
CPU_SAMPLE_TEXT = ("config-2 distribution at 1/8 scale: 32 slots, 2 GiB, 12,500 ops log-uniform 16 B-4 MiB, "
                   "10% unaligned, all epochs; slot bytes set to a constant (the copy cost does not depend on values)")


def oracle_sample(seed):
    from oracle import memcpy as om
    w = configs.batched(seed, **CPU_SAMPLE, name="cpu_sample")
    cm = om.CommManager()
    for sz in w.slot_sizes:
        cm.register(om.SPACE_HBM, np.ones(int(sz), dtype=np.uint8))
    return cm, w


def oracle_pass(cm, w):
    from oracle import memcpy as om
    for a, b in w.epochs:
        st, _ = cm.memcpy_batch(w.ops[a:b])
        assert st == om.OK
        cm.fence(0)
    return 2 * w.total_bytes


def cpu_baseline(seed, target_s):
    cm, w = oracle_sample(seed)
    oracle_pass(cm, w)  # first touch of every page
    t0 = time.perf_counter()
    nbytes, passes = 0, 0
    while True:
        nbytes += oracle_pass(cm, w)
        passes += 1
        el = time.perf_counter() - t0
        if el >= target_s or passes >= 200:
            break
    out = {"value": nbytes / el / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"{CPU_SAMPLE_TEXT}; {passes} passes in {el:.1f} s", "host": host_info()}
    # the same sample as plain memcpy on every host core (oracle/memcpy_threads.c)
    try:
        from oracle.native import ThreadedMemcpy
        cores = os.cpu_count() or 1
        tm = ThreadedMemcpy([cm.slots[i].data for i in sorted(cm.slots)], w.ops, w.epochs)
        tm.run(cores)
        t0 = time.perf_counter()
        passes = 0
        while True:
            tm.run(cores)
            passes += 1
            el = time.perf_counter() - t0
            if el >= min(target_s, 3.0) or passes >= 200:
                break
        out["all_cores"] = {"value": passes * 2 * w.total_bytes / el / 1e9, "unit": "GB/s", "cores": cores,
                            "kind": "memcpy on all host cores", "sample": f"same sample; {passes} passes in {el:.1f} s"}
    except (OSError, subprocess.CalledProcessError) as e:
        out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return out


def nominal_hbm(h, inst):
    """Datasheet-style HBM bandwidth (GB/s): the memory clock x bus width the
    driver reports (the library's topology query), else the GB300 HBM3e
    figure of about 7.9 TB/s."""
    st, t = h.hicr_topology_query(inst)
    if st == 0 and t.spaces[0].peak_mbps:
        return t.spaces[0].peak_mbps / 1e3, "memory clock x bus width reported by the driver"
    return 7900.0, "GB300 HBM3e datasheet figure (about 7.9 TB/s)"


def cpu_channels_baseline(seed, target_s=2.0):
    """The oracles as they stand on bounded samples of configs 1, 3 and 4
    (one core): SPSC push/pop of 64-B tokens in batches of 2,048 through a
    4,096-token ring; MPSC push/pop of config 4's first consumer's messages
    (64 producers round-robin, payloads generated beforehand) through its
    1 GiB ring in windows of 64; config 1's memcpy table."""
    from oracle import channels as oc
    w3 = configs.SpscWorkload()
    ch = oc.SpscOracle(w3.token_bytes, w3.capacity)
    batch = 2048
    data = splitmix.spsc_token_words(0, 0, batch, w3.token_bytes // 8).view(np.uint8)
    t0 = time.perf_counter()
    tokens = 0
    while time.perf_counter() - t0 < target_s:
        assert ch.push(data) == 0 and ch.pop(batch) == 0
        tokens += batch
    spsc = tokens / (time.perf_counter() - t0)
    w4 = configs.mpsc(seed)
    prods = list(range(0, w4.n_producers, w4.n_consumers))
    msgs = [(p, q, splitmix.mpsc_payload_bytes(p, q, int(w4.sizes[p, q]))) for q in range(2) for p in prods]
    mc = oc.MpscOracle(len(prods), w4.ring_bytes, w4.max_msgs)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < target_s:
        for i in range(0, len(msgs), 64):
            for p, q, payload in msgs[i:i + 64]:
                assert mc.push(p // w4.n_consumers, payload) == 0
            assert mc.pop(len(msgs[i:i + 64])) == 0
            n += len(msgs[i:i + 64])
    mpsc = n / (time.perf_counter() - t0)
    # config 1 (2 x 64 MiB slots, 1,024 ops): the memcpy oracle on the whole table
    from oracle import memcpy as om
    w1 = configs.tiny(seed)
    cm = om.CommManager()
    for sz in w1.slot_sizes:
        cm.register(om.SPACE_HBM, np.ones(int(sz), dtype=np.uint8))
    t0 = time.perf_counter()
    passes = 0
    while time.perf_counter() - t0 < target_s:
        assert cm.memcpy_batch(w1.ops) == (om.OK, None)
        passes += 1
    tiny_gbs = passes * 2 * int(w1.ops["n"].astype(np.int64).sum()) / (time.perf_counter() - t0) / 1e9
    return {"spsc_tokens_per_s": spsc, "mpsc_msgs_per_s": mpsc, "config1_memcpy_GB_per_s": tiny_gbs,
            "cores": 1, "kind": "oracle",
            "sample": f"SPSC: 64-B tokens, batches of {batch}, capacity {w3.capacity}; MPSC: {len(msgs)} messages "
                      f"of config 4's consumer 0 (64 producers), 1 GiB ring, windows of 64; config 1: the whole "
                      f"1,024-op table; about {target_s:g} s each"}


def host_info():
    """Core count and CPU model of the machine that timed the CPU lines."""
    model = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def run_reference(args):
    """--impl reference: the oracle (the parity authority) timed on the host
    cores on the same metric, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cm, w = oracle_sample(args.seed)
    for _ in range(args.warmup):
        oracle_pass(cm, w)
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(args.steps):
        nbytes += oracle_pass(cm, w)
    el = time.perf_counter() - t0
    v = nbytes / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": "batched memcpy (CPU oracle sample)",
                                            "sample": CPU_SAMPLE_TEXT},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": CPU_SAMPLE_TEXT},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our arm.
# ---------------------------------------------------------------------------
def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, bytes_per_step, steps, job_ms):
    """Whole-job GB/s: every rank (replica) moves bytes_per_step per step on
    its own copy of the workload; the job takes job_ms (max over ranks)."""
    return world * bytes_per_step * steps / (job_ms * 1e-3) / 1e9


def run_ours(args):
    import torch
    from paper_2509_01425_gb300 import build
    build.build()
    from paper_2509_01425_gb300 import hicr as h

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    inst = h.check(h.hicr_init(dev), "hicr_init")
    stream_ptr = h.check(h.hicr_pu_stream(inst, 0), "pu_stream")
    stream = torch.cuda.ExternalStream(stream_ptr)
    peak, peak_src = peaks()
    nominal, nominal_src = nominal_hbm(h, inst)

    w = scaled_batched(args.seed, args.scale)
    ids = setup_slots(h, inst, w, args.seed)
    lops = remap(w.ops, ids)
    dops = device_ops(lops)
    torch.cuda.synchronize()
    if args.batch_config:  # a fixed configuration (e.g. for a profiler's launch list): no autotuning
        c = h.check(h.hicr_batch_get_config(inst), "get_config")
        for k, v in json.loads(args.batch_config).items():
            setattr(c, k, int(v))
        h.check(h.hicr_batch_set_config(inst, c), "set_config")
        tuned, tuned_ms = c.as_dict(), None
    else:
        tuned, tuned_ms = autotune(h, inst, dops, w.epochs)
    h.check(h.hicr_profile_enable(inst, 1), "profile")
    g = capture_epochs(h, inst, dops, w.epochs)
    bytes_step = 2 * w.total_bytes

    clocks = Clocks(dev)
    clocks.start()
    ms, copy_ms, launches = time_graph(h, inst, stream, g, args.steps, args.warmup, prof=True, dist=dist)
    clk = clocks.stop()
    h.check(h.hicr_profile_enable(inst, 0), "profile")
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_value(world, bytes_step, args.steps, ms)
    achieved = bytes_step * args.steps / (copy_ms * 1e-3) / 1e9 if copy_ms > 0 else None
    n_epochs = len(w.epochs)

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"batched memcpy: {len(ids)} HBM slots totalling "
                               f"{int(w.slot_sizes.sum()) / GiB:g} GiB (log-uniform 1-256 MiB), "
                               f"{len(w.ops):,} ops log-uniform 16 B-4 MiB, 10% unaligned, "
                               f"{n_epochs} fence epochs, one CUDA graph per step + fence(0)",
                   "scale": args.scale,
                   "ops_per_step": int(len(w.ops)), "bytes_moved_per_step": int(w.total_bytes),
                   "algorithmic_bytes_per_step": int(bytes_step), "epochs": n_epochs,
                   "l2": "no flush: 16 GiB of slots >> 126 MB L2", "batch_config": tuned,
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "nominal_peak": nominal, "nominal_source": nominal_src,
                     "frac_of_nominal": (achieved / nominal) if achieved else None,
                     "traffic": copy_traffic("k_copy_tma" if tuned.get("engine") == 1 else "k_copy",
                                             bytes_step / n_epochs),
                     "algorithmic_bytes_per_launch": bytes_step / n_epochs,
                     "kernel": "k_copy_tma" if tuned.get("engine") == 1 else "k_copy",
                     "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                     "launches_timed": launches},
        "gpu_launches": args.steps * 2 * n_epochs,
        "clocks": clk,
    }

    if not args.no_side:
        side = {}
        # large-segment case (1-4 MiB aligned): the >= 80% of peak gate
        wl = scaled_batched(args.seed, args.scale, large=True)
        assert (wl.slot_sizes == w.slot_sizes).all()
        dl = device_ops(remap(wl.ops, ids))
        lsteps = max(3, args.steps // 2)
        lb = 2 * wl.total_bytes

        def large_run():
            h.check(h.hicr_profile_enable(inst, 1), "profile")
            h.check(h.hicr_profile_reset(inst), "profile")
            gl = capture_epochs(h, inst, dl, wl.epochs)
            lms, lcopy, _ = time_graph(h, inst, stream, gl, lsteps, 2, prof=True)
            h.check(h.hicr_profile_enable(inst, 0), "profile")
            h.check(h.hicr_graph_destroy(inst, gl), "graph_destroy")
            return {"GB_per_s": lb * lsteps / (lms * 1e-3) / 1e9,
                    "copy_kernel_GB_per_s": lb * lsteps / (lcopy * 1e-3) / 1e9,
                    "frac_of_peak": lb * lsteps / (lms * 1e-3) / 1e9 / peak}

        headline_cfg = h.check(h.hicr_batch_get_config(inst), "get_config")
        side["large_segments"] = {"workload": "1-4 MiB aligned ops, same slots", "ops": int(len(wl.ops)),
                                  "config": tuned, **large_run()}
        # the TMA engine (bulk copies through shared memory) on the same ops
        tma = h.check(h.hicr_batch_get_config(inst), "get_config")
        tma.engine, tma.tma_min_bytes, tma.threads, tma.blocks_per_sm = 1, 256 << 10, 384, 1
        tma.chunk_bytes, tma.op_cost_bytes = 1 << 20, 4096
        if h.hicr_batch_set_config(inst, tma) == 0:
            side["large_segments"]["tma_engine"] = {"config": tma.as_dict(), **large_run()}
        # what the autotuner picks for this workload (both engines are candidates)
        ltuned, _ = autotune(h, inst, dl, wl.epochs)
        side["large_segments"]["autotuned"] = {"config": ltuned, **large_run()}
        h.check(h.hicr_batch_set_config(inst, headline_cfg), "set_config")
        del dl

        # plain form: one cudaMemcpyAsync per op, same op table, same epochs + fences
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in w.epochs:
            h.check(h.hicr_memcpy_batch_plain(inst, lops[a:b]), "plain")
            h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
        pl = time.perf_counter() - t0
        side["plain_form"] = {"GB_per_s": bytes_step / pl / 1e9, "ms_per_step": pl * 1e3,
                              "speedup_of_batched": (bytes_step / pl / 1e9) and value / world / (bytes_step / pl / 1e9)}

        # end to end through the public API with host op tables
        esteps = max(3, args.steps // 4)
        for _ in range(2):
            for a, b in w.epochs:
                h.check(h.hicr_memcpy_batch(inst, lops[a:b]), "batch")
                h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(esteps):
            for a, b in w.epochs:
                h.check(h.hicr_memcpy_batch(inst, lops[a:b]), "batch")
                h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
            h.check(h.hicr_slot_counters_range(inst, ids[0], len(ids)), "counters")
        el = time.perf_counter() - t0
        line["e2e"] = {"value": bytes_step * esteps / el / 1e9, "unit": "GB/s",
                       "h2d_bytes_per_step": int(32 * len(w.ops)), "d2h_bytes_per_step": int(16 * len(ids)),
                       "steps": esteps, "call": "hicr_memcpy_batch (host ops) + hicr_fence per epoch, "
                                                "hicr_slot_counters_range per step"}
        side["spsc"] = bench_spsc(h, inst)
        side["pingpong"] = bench_pingpong(h, inst)
        side["host_space"] = bench_host_space(h, inst)
        side["latency"] = bench_latencies(h, inst)
        side["mpsc"] = bench_mpsc(h, inst)
        if args.serve_seconds > 0:
            h.check(h.hicr_graph_destroy(inst, g), "graph_destroy")
            g = None
            for sid in ids:  # the serving run allocates its own copy of the source slots
                h.check(h.hicr_mem_free(inst, sid), "free")
            ids = []
            side["serving"] = bench_serve(h, inst, seconds=args.serve_seconds,
                                          plain_seconds=args.plain_serve_seconds, seed=args.seed)
        line["side"] = side
        if world == 1 and rank == 0:
            line["cpu_baseline"] = cpu_baseline(args.seed, args.cpu_seconds)
            line["cpu_baseline"]["channels"] = cpu_channels_baseline(args.seed)

    if g is not None:
        h.check(h.hicr_graph_destroy(inst, g), "graph_destroy")
    h.check(h.hicr_finalize(inst), "finalize")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    if args.profile_case == "copy_small":
        return run_copy_small(args)
    if args.profile_case == "side_small":
        return run_side_small(args)
    if args.profile_case == "control_small":
        return run_control_small(args)
    return run_mpsc_small(args)


def run_control_small(args):
    """control_small, for a one-pass capture (duration and DRAM bytes) of the
    control-path kernels: slot registration (k_set_slot); host-side channel
    calls, 16 rounds each of push, peek and pop on an SPSC channel (64 B
    tokens), a locking MPSC and a non-locking MPSC channel (messages of
    100 B-64 KiB) (k_*_push_host, k_*_ctl); the seeded staging fill and the
    pre-checks of both MPSC streams on a 64 -> 4 producer x 16 message table
    (k_fill_segments, k_mpsc_check, k_nl_check, the streams' set-up and
    wrap-up kernels, and the two stream kernels); two allocation-free batches
    of 10,000 ops (k_plan, k_scan, k_copy); four single memcpys, each
    followed by a fence (k_copy_small); the same four in latency mode with a
    100 us idle window, 1 ms apart (four k_lat_server launches); four SPSC
    push + pop pairs in latency mode, 1 ms apart (four more k_lat_server
    launches, each taking a push and a pop); and a 1 ms bounded device wait
    (k_wait_test)."""
    import torch
    from paper_2509_01425_gb300 import build
    build.build()
    from paper_2509_01425_gb300 import hicr as h
    torch.cuda.set_device(0)
    inst = h.check(h.hicr_init(0), "hicr_init")
    size = 64 * MiB
    a = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size), "alloc")
    h.check(h.hicr_util_fill(inst, a, 0, size, splitmix.fill_key_base(args.seed, 1)), "fill")
    t = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(4):
        r = h.check(h.hicr_slot_register(inst, h.HICR_SPACE_HBM, t.data_ptr(), t.numel()), "register")
        h.check(h.hicr_slot_deregister(inst, r), "deregister")
    spsc = h.check(h.hicr_spsc_create(inst, 64, 4096), "spsc_create")
    lock = h.check(h.hicr_mpsc_create(inst, 4, 1 << 20, 64), "mpsc_create")
    nl = h.check(h.hicr_mpsc_nl_create(inst, 4, 1 << 20, 64), "nl_create")
    for i in range(16):
        h.check(h.hicr_channel_push(inst, spsc, 0, a, 4096 * i, 16), "spsc push")
        h.check(h.hicr_channel_peek(inst, spsc, 0)[0], "spsc peek")
        h.check(h.hicr_channel_pop(inst, spsc, 16), "spsc pop")
        n = (100, 4096, 65536)[i % 3]
        for ch in (lock, nl):
            h.check(h.hicr_channel_push(inst, ch, i % 4, a, 65536 * i, n), "mpsc push")
            h.check(h.hicr_channel_peek(inst, ch, 0)[0], "mpsc peek")
            h.check(h.hicr_channel_pop(inst, ch, 1), "mpsc pop")
    for ch in (spsc, lock, nl):
        h.check(h.hicr_channel_destroy(inst, ch), "destroy")
    w = configs.mpsc(args.seed, n_producers=64, n_consumers=4, msgs_per_producer=16, ring_bytes=1 << 20,
                     max_msgs=256, hi=16 << 10)
    run = MpscRun(h, inst, w, group=4, consumer_ctas=2)
    h.check(run.run()[0], "mpsc stream")
    run.set_mode(True, 2, 1 << 16, 16)
    h.check(run.run()[0], "nl stream")
    run.free()
    n_ops = 10_000
    rng = np.random.default_rng(args.seed)
    n = rng.integers(16, 2048, n_ops).astype(np.uint64)
    dst = np.arange(n_ops, dtype=np.uint64) * np.uint64(2048)
    src = np.uint64(32 * MiB) + dst
    b = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size), "alloc")
    ops = configs.make_ops([b] * n_ops, [a] * n_ops, dst, src, n)
    d_ops = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    h.check(h.hicr_batch_reserve(inst, n_ops), "reserve")
    for _ in range(2):
        h.check(h.hicr_memcpy_batch_noalloc(inst, d_ops.data_ptr(), n_ops), "noalloc")
        h.check(h.hicr_fence(inst, 0, 10_000_000_000), "fence")
    for i in range(4):  # single memcpys before a fence: the small-batch kernel
        h.check(h.hicr_memcpy(inst, b, 40 * MiB + 64 * i, a, 64 * i, 16 << i), "memcpy")
        h.check(h.hicr_fence(inst, 0, 10_000_000_000), "fence")
    # the same in latency mode: each server takes its copy, idles 100 us and ends
    h.check(h.hicr_set_latency_mode(inst, 100), "latency mode")
    for i in range(4):
        h.check(h.hicr_memcpy(inst, b, 41 * MiB + 64 * i, a, 64 * i, 16 << i), "memcpy")
        h.check(h.hicr_fence(inst, 0, 10_000_000_000), "fence")
        time.sleep(0.001)
    # channel calls in latency mode: one server takes a push and its pop
    spsc = h.check(h.hicr_spsc_create(inst, 64, 4096), "spsc_create")
    for i in range(4):
        h.check(h.hicr_channel_push(inst, spsc, 0, a, 4096 * i, 16), "spsc push")
        h.check(h.hicr_channel_pop(inst, spsc, 16), "spsc pop")
        time.sleep(0.001)
    h.check(h.hicr_channel_destroy(inst, spsc), "destroy")
    h.check(h.hicr_set_latency_mode(inst, 0), "latency mode off")
    st, wst, waited = h.hicr_util_wait_test(inst, 1_000_000)
    h.check(st, "wait_test")
    h.check(h.hicr_finalize(inst), "finalize")
    print(json.dumps({"case": "control_small", "wait_status": wst, "waited_ns": waited}), flush=True)
    return 0


def run_side_small(args):
    """side_small, for a one-pass capture (DRAM bytes and duration) of the
    kernels that are not profiled elsewhere: an SPSC stream (64 channels x
    10^6 tokens of 64 B, batches of 2,048), generating and then copying
    staged tokens, a ping-pong of 256 MiB with agents
    of 152 CTAs and one of 1 GiB with agents of 76 CTAs (the bulk-copy form;
    10 round trips each), a 0.5 s serving trace at 20,000 req/s on
    the bench's engine set-up, and the word digest of a 4 GiB slot. Prints
    the algorithmic bytes of each so the capture can be read against them."""
    import torch
    from paper_2509_01425_gb300 import build
    build.build()
    from paper_2509_01425_gb300 import hicr as h
    torch.cuda.set_device(0)
    inst = h.check(h.hicr_init(0), "hicr_init")
    out = {"case": "side_small"}
    w = configs.SpscWorkload()
    chans = [h.check(h.hicr_spsc_create(inst, w.token_bytes, w.capacity), "spsc") for _ in range(w.n_channels)]
    h.check(h.hicr_spsc_stream(inst, chans, 1_000_000, 2048)[0], "spsc_stream")
    out["spsc_tokens"] = w.n_channels * 1_000_000
    out["spsc_algorithmic_bytes"] = w.n_channels * 1_000_000 * 128
    # copying producers (4,096 staged tokens per channel)
    stg_bytes = w.n_channels * w.capacity * w.token_bytes
    stg = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, stg_bytes), "staging")
    h.check(h.hicr_util_fill(inst, stg, 0, stg_bytes, splitmix.fill_key_base(0, 77)), "fill staging")
    h.check(h.hicr_spsc_stream_ex(inst, chans, 1_000_000, 2048, src=stg, src_tokens=w.capacity)[0], "spsc copy")
    out["spsc_copy_l2_bytes"] = w.n_channels * 1_000_000 * 192
    h.check(h.hicr_mem_free(inst, stg), "free")
    for c in chans:
        h.check(h.hicr_channel_destroy(inst, c), "destroy")
    size = 256 << 20
    sid = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size), "alloc")
    h.check(h.hicr_util_fill(inst, sid, 0, size, splitmix.fill_key_base(0, 5)), "fill")
    st, r = h.hicr_pingpong(inst, sid, 0, size, 10, 2, 152)
    h.check(st, "pingpong")
    out["pingpong_algorithmic_bytes"] = 12 * 2 * 2 * size  # 12 round trips x 2 one-way copies x (read + write)
    h.check(h.hicr_mem_free(inst, sid), "free")
    size = 1 << 30  # the bulk-copy form: agents of 76 CTAs, one per SM
    sid = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size), "alloc")
    h.check(h.hicr_util_fill(inst, sid, 0, size, splitmix.fill_key_base(0, 7)), "fill")
    st, r = h.hicr_pingpong(inst, sid, 0, size, 10, 2, 76)
    h.check(st, "pingpong bulk")
    out["pingpong_bulk_algorithmic_bytes"] = 12 * 2 * 2 * size
    h.check(h.hicr_mem_free(inst, sid), "free")
    big = 4 << 30
    sid = h.check(h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, big), "alloc")
    h.check(h.hicr_util_fill(inst, sid, 0, big, splitmix.fill_key_base(0, 6)), "fill")
    h.check(h.hicr_util_digest(inst, sid, 0, big), "digest")
    out["digest_algorithmic_bytes"] = big
    out["fill_algorithmic_bytes"] = big
    h.check(h.hicr_mem_free(inst, sid), "free")
    src_w = configs.batched(args.seed)
    tmpl = configs.serve_templates(args.seed, src_w)
    ss = ServeSetup(h, inst, src_w, tmpl, seed=args.seed)
    reqs = ss.requests(configs.serve_trace(args.seed, rate=20000.0, duration_s=0.5))
    st, res, stats = h.hicr_serve_run(inst, ss.srv, reqs, 0, 120_000_000_000)
    h.check(st, "serve_run")
    out["serve_requests"] = int(stats.completed)
    out["serve_bytes_moved"] = int(stats.bytes_moved)
    out["serve_wall_s"] = stats.wall_ns / 1e9
    ss.free()
    h.check(h.hicr_finalize(inst), "finalize")
    print(json.dumps(out), flush=True)
    return 0


def run_copy_small(args):
    """copy_small: the batched workload at --copy-scale (default 1/8: 32
    slots, 2 GiB, 12,500 ops; 1.0 is the full workload) under the
    configuration --batch-config, each epoch one device batch + fence; two
    passes, so the copy kernel launches once per epoch in each (the second
    pass is the one to capture)."""
    import torch
    from paper_2509_01425_gb300 import build
    build.build()
    from paper_2509_01425_gb300 import hicr as h
    torch.cuda.set_device(0)
    inst = h.check(h.hicr_init(0), "hicr_init")
    if args.batch_config:
        c = h.check(h.hicr_batch_get_config(inst), "get_config")
        for k, v in json.loads(args.batch_config).items():
            setattr(c, k, int(v))
        h.check(h.hicr_batch_set_config(inst, c), "set_config")
    scale = args.copy_scale
    w = scaled_batched(args.seed, scale)
    ids = setup_slots(h, inst, w, args.seed)
    dops = device_ops(remap(w.ops, ids))
    out = {"case": "copy_small", "scale": scale, "ops": int(len(w.ops)), "epochs": len(w.epochs),
           "config": h.check(h.hicr_batch_get_config(inst), "get_config").as_dict()}
    for rep in range(2):
        t0 = time.perf_counter()
        for a, b in w.epochs:
            h.check(h.hicr_memcpy_batch_device(inst, dops.data_ptr() + 32 * a, b - a), "batch")
            h.check(h.hicr_fence(inst, 0, FENCE_TIMEOUT), "fence")
        out[f"pass{rep}_s"] = time.perf_counter() - t0
    out["algorithmic_bytes_per_pass"] = int(2 * w.total_bytes)
    for sid in ids:
        h.check(h.hicr_mem_free(inst, sid), "free")
    h.check(h.hicr_finalize(inst), "finalize")
    print(json.dumps(out), flush=True)
    return 0


def run_mpsc_small(args):
    """mpsc_small: config 4's producers and consumers with 32 messages each
    (0.83 GB of payload) over 16 x 128 MiB locking rings, then over 64 x 2 MiB
    non-locking rings per consumer, 5 CTAs per consumer; each mode runs once
    untimed and once timed, so the stream kernels launch in the order
    locking, non-locking, locking, non-locking (about 3 GB on the device)."""
    import torch
    from paper_2509_01425_gb300 import build
    build.build()
    from paper_2509_01425_gb300 import hicr as h
    torch.cuda.set_device(0)
    inst = h.check(h.hicr_init(0), "hicr_init")
    w = configs.mpsc(args.seed, msgs_per_producer=32, ring_bytes=128 * MiB)
    run = MpscRun(h, inst, w, group=4, consumer_ctas=5)
    out = {"case": "mpsc_small", "msgs": int(w.sizes.size), "payload_bytes": int(w.total_bytes)}
    timings = {}
    for rep in range(2):
        for mode in ("locking", "nonlocking"):
            run.set_mode(mode == "nonlocking", 5)
            t0 = time.perf_counter()
            h.check(run.run()[0], mode)
            if rep:
                timings[mode + "_s"] = time.perf_counter() - t0
    run.free()
    out.update(timings)
    h.check(h.hicr_finalize(inst), "finalize")
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
