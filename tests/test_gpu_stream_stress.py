"""Stress parity of the MPSC streams: random shapes, both modes.

Each seed draws a producer and consumer count, messages per producer, a
log-uniform size range, ring and metadata capacities (powers of two; every
message fits half a ring), a reservation group size, consumer CTAs, whether
the staged payloads are packed 16-byte aligned or `gap` bytes apart (so the
producers' bulk copies meet every alignment and fall back where they must),
and which messages are empty. The streams' logs must pass the oracle's
interleaving-agnostic checker, every message the consumers received (the
capture form) must equal the oracle's delivery byte by byte, and every
payload digest must equal the oracle's; a second run continues from the
channels' counters."""
import numpy as np
import pytest

import bench
from workloads import configs
from tests.gpu_util import h, inst  # noqa: F401
from tests.test_gpu_channels import _check_capture, _check_mpsc, _check_mpsc_nl, _oracle_deliveries

pytestmark = pytest.mark.gpu


def _shape(seed, nonlocking):
    rng = np.random.default_rng(7000 + 2 * seed + int(nonlocking))
    C = int(rng.integers(1, 9))
    P = int(rng.integers(C, 257))
    M = int(rng.integers(1, 65))
    hi = int(rng.choice([64, 1 << 10, 8 << 10, 64 << 10]))
    lo = int(rng.choice([1, 8, 16]))
    ring = int(rng.choice([1 << 15, 1 << 17, 1 << 20]))
    ring = max(ring, 4 * hi)  # every message fits half a ring with room to spare
    max_msgs = int(rng.choice([4, 16, 64, 256]))
    group = int(rng.integers(1, 9))
    ctas = int(rng.integers(1, 6))
    gap = None if rng.random() < 0.5 else int(rng.choice([1, 3, 7, 16, 33]))
    w = configs.mpsc(seed, n_producers=P, n_consumers=C, msgs_per_producer=M, ring_bytes=ring, max_msgs=max_msgs,
                     lo=lo, hi=hi)
    empty_every = int(rng.choice([0, 3, 7]))
    if empty_every:
        w.sizes[:, ::empty_every] = 0
    return w, ring, max_msgs, group, ctas, gap


@pytest.mark.parametrize("nonlocking", [False, True])
@pytest.mark.parametrize("seed", range(32))
def test_random_stream_shapes(h, inst, seed, nonlocking):
    w, ring, max_msgs, group, ctas, gap = _shape(seed, nonlocking)
    run = bench.MpscRun(h, inst, w, group=group, nonlocking=nonlocking, consumer_ctas=ctas, ring_bytes=ring,
                        max_msgs=max_msgs, stage_gap=gap)
    for rnd in range(2):
        st, res = run.run(capture=True)
        assert st == 0, (seed, rnd)
        assert sum(int(r.consumed) for r in res) == w.sizes.size
        if rnd == 0:  # positions replay from the first ticket only on the first run
            if nonlocking:
                _check_mpsc_nl(w, run, res)
            else:
                _check_mpsc(w, run.logs(), res, ring)
            deliveries = _oracle_deliveries(w, ring, max_msgs, nonlocking)
        _check_capture(w, run, deliveries)
    for ch in run.chans:
        assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    run.free()
