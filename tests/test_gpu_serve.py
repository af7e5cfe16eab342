"""Serving loop: every request's result is the same alone and in the mix.

A request is a memcpy batch into its own destination region or an MPSC burst
drained by a channel consumer. Its result digest (memcpy: ordered combination
of the word digests of its ops' destination bytes; burst: ordered combination
of the consumed messages' digests) must be bit-identical when the requests
run one at a time and when they arrive together and overlap on the device,
and both must equal the digest the oracle computes from the seeded sources.
"""
import numpy as np
import pytest

import bench
from oracle import digest as od
from workloads import configs, splitmix
from tests.gpu_util import h, inst  # noqa: F401

pytestmark = pytest.mark.gpu

SEED = 3
T = 30_000_000_000


def small_setup(h, inst, verify=True, budget=512 << 20):
    src_w = configs.batched(SEED, n_slots=8, total_bytes=64 << 20, slot_lo=1 << 20, slot_hi=16 << 20, n_ops=50,
                            n_hi=64 << 10)
    tmpl = configs.serve_templates(SEED, src_w, n_templates=16, max_ops=48, max_msgs=24, n_hi=256 << 10,
                                   msg_hi=16 << 10)
    assert tmpl.region_bytes.max() <= 16 << 20
    ss = bench.ServeSetup(h, inst, src_w, tmpl, seed=SEED, budget=budget, n_channels=4, ring_bytes=8 << 20,
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
    st, pres, pstats = h.hicr_serve_run_plain(inst, ss.srv, reqs, int(1e12), T)
    assert st == 0 and pstats.completed == len(reqs)
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
