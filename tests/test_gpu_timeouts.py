"""Failure detection without a GPU fault: every device-side wait of the
channel kernels is bounded by the run's deadline. With a deadline of 1 us the
streams and the ping-pong cannot finish: their waits give up, raise the
shared abort flag, every CTA leaves, and the call returns HICR_ERR_TIMEOUT.
The context stays usable: a normal run right after succeeds and is exact."""
import numpy as np
import pytest

import bench
from oracle import channels as oc
from oracle import digest as od
from workloads import configs, splitmix
from tests.gpu_util import h, inst  # noqa: F401
from tests.test_gpu_channels import _check_mpsc, _check_mpsc_nl, _spsc_expected_digest

pytestmark = pytest.mark.gpu

TINY = 1_000  # 1 us


def test_spsc_stream_gives_up_and_recovers(h, inst):
    chans = [h.hicr_spsc_create(inst, 64, 16)[1] for _ in range(4)]
    st, res = h.hicr_spsc_stream(inst, chans, 10_000_000, 16, TINY)
    assert st == h.HICR_ERR_TIMEOUT
    assert any(r.status == h.HICR_ERR_TIMEOUT for r in res)
    assert all(r.pushed < 10_000_000 for r in res)
    for c in chans:
        assert h.hicr_channel_destroy(inst, c) == 0
    chans = [h.hicr_spsc_create(inst, 64, 64)[1] for _ in range(2)]
    st, res = h.hicr_spsc_stream(inst, chans, 5000, 16)
    assert st == 0
    for i, r in enumerate(res):
        assert (r.popped, r.mismatches, r.status) == (5000, 0, 0)
        assert r.digest == _spsc_expected_digest(i, 5000)


@pytest.mark.parametrize("nonlocking", [False, True])
def test_mpsc_stream_gives_up_and_recovers(h, inst, nonlocking):
    # rings far smaller than the traffic: producers must wait for the
    # consumers, long after the 1 us deadline has passed
    w = configs.mpsc(11, n_producers=64, n_consumers=4, msgs_per_producer=64, ring_bytes=1 << 16, max_msgs=64,
                     hi=8 << 10)
    run = bench.MpscRun(h, inst, w, group=2, nonlocking=nonlocking, consumer_ctas=2, ring_bytes=1 << 16,
                        max_msgs=64 if not nonlocking else 8)
    st, res = run.run(timeout_ns=TINY)
    assert st == h.HICR_ERR_TIMEOUT
    assert sum(int(r.consumed) for r in res) < w.sizes.size
    # fresh channels (the old ones hold reservations that were never published)
    run.set_mode(nonlocking, 2, 1 << 16, 64 if not nonlocking else 8)
    st, res = run.run()
    assert st == 0
    if nonlocking:
        _check_mpsc_nl(w, run, res)
    else:
        _check_mpsc(w, run.logs(), res, 1 << 16)
    run.free()


@pytest.mark.parametrize("size,ctas", [(1 << 20, 1), (128 << 20, 64)])  # vector form, bulk-copy form
def test_pingpong_gives_up_and_recovers(h, inst, size, ctas):
    st, s = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, size)
    assert h.hicr_util_fill(inst, s, 0, size, splitmix.fill_key_base(8, 1)) == 0
    st, r = h.hicr_pingpong(inst, s, 0, size, 1000, 0, ctas, TINY)
    assert st == h.HICR_ERR_TIMEOUT
    st, r = h.hicr_pingpong(inst, s, 0, size, 4, 1, max(ctas, 4))
    assert st == 0 and r.status == 0
    exp = od.byte_digest(splitmix.fill_bytes(8, 1, 0, size))
    assert r.digest_a == exp and r.digest_b == exp
    assert h.hicr_mem_free(inst, s) == 0
