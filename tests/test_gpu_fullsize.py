"""Full-size batched memcpy (256 slots, 16 GiB, 100,000 ops, all fence epochs)
in the launch configuration bench.py times (autotuned config, one CUDA graph
per step): sampled bytes one by one against the oracle, counters exactly."""
import numpy as np
import pytest
import torch

import bench
from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, h, inst  # noqa: F401

pytestmark = pytest.mark.gpu


def _positions(w, slot, rng, n_random=4096):
    size = int(w.slot_sizes[slot])
    m = w.ops["dst"] == slot
    d = w.ops["dst_off"][m].astype(np.int64)
    n = w.ops["n"][m].astype(np.int64)
    edges = np.concatenate([d - 1, d, d + n - 1, d + n, d + n // 2])
    pos = np.concatenate([edges, rng.integers(0, size, n_random)])
    return np.unique(pos[(pos >= 0) & (pos < size)])


@pytest.mark.parametrize("maker", [configs.batched, configs.batched_large])
def test_full_size_sampled_parity(h, inst, maker):
    seed = 0
    w = maker(seed)
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
    rng = np.random.default_rng(123)
    init = lambda s, p: splitmix.fill_byte_at(seed, s, p)  # noqa: E731
    checked = 0
    for s in range(len(ids)):
        st, ptr, size, _, _ = h.hicr_slot_info(inst, ids[s])
        view = device_bytes(ptr, size)
        pos = _positions(w, s, rng) if s in set(w.dst_slots.tolist()) else rng.integers(0, size, 2048)
        got = view[torch.from_numpy(np.asarray(pos, dtype=np.int64)).cuda()].cpu().numpy()
        exp = om.expected_bytes_at(w.ops, w.epochs, s, pos, init)
        bad = np.nonzero(got != exp)[0]
        assert len(bad) == 0, f"slot {s}: {len(bad)} of {len(pos)} sampled bytes differ, first at {pos[bad[0]]}"
        checked += len(pos)
    assert checked > 500_000
    sent, recv = om.counters_from_ops(w.ops, len(ids))
    st, gs, gr = h.hicr_slot_counters_range(inst, ids[0], len(ids))
    assert st == 0
    assert (gs - s0 == steps * sent).all() and (gr - r0 == steps * recv).all()
    assert h.hicr_tag_counter(inst, 0) == (0, t0 + steps * len(w.ops))
    assert h.hicr_graph_destroy(inst, g) == 0


@pytest.mark.parametrize("batch", [256, 1024, 2048])
def test_spsc_full_size(h, inst, batch):
    """64 channels x capacity 4,096 x 64 B, 10^7 tokens per channel, at the
    hand-off batch sizes the bench chooses from: every word checked on the
    device against the payload rule, exact counts, capacity respected, and
    the whole-stream digest of two channels against the oracle."""
    from tests.test_gpu_channels import _spsc_expected_digest
    w = configs.SpscWorkload()
    chans = [h.hicr_spsc_create(inst, w.token_bytes, w.capacity)[1] for _ in range(w.n_channels)]
    st, res = h.hicr_spsc_stream(inst, chans, w.tokens_per_channel, batch)
    assert st == 0
    for r in res:
        assert (r.pushed, r.popped, r.mismatches, r.status) == (w.tokens_per_channel,) * 2 + (0, 0)
        assert r.max_occupancy <= w.capacity
    for i in (0, w.n_channels - 1):
        assert res[i].digest == _spsc_expected_digest(i, w.tokens_per_channel)


@pytest.mark.parametrize("ctas,group", [(1, 4), (4, 4), (5, 4), (5, 8)])
def test_mpsc_full_size(h, inst, ctas, group):
    """1,024 producers -> 16 consumers, 1,024 messages each (log-uniform
    8 B - 256 KiB), 1 GiB rings, 1 or 4 CTAs per consumer (the bench's
    launch shapes): every consumer's log passes the checker; a sample of
    payload digests matches the oracle."""
    from tests.test_gpu_channels import _check_mpsc
    w = configs.mpsc(0)
    run = bench.MpscRun(h, inst, w, group=group, consumer_ctas=ctas)
    st, res = run.run()
    assert st == 0
    assert sum(int(r.consumed) for r in res) == w.sizes.size
    _check_mpsc(w, run.logs(), res, w.ring_bytes, sample=0.003)
    run.free()


@pytest.mark.parametrize("ctas,group", [(1, 4), (4, 4), (5, 4), (5, 8)])
def test_mpsc_nonlocking_full_size(h, inst, ctas, group):
    """The same messages over 64 rings of 16 MiB per consumer (non-locking
    mode at the locking mode's memory), 1 or 4 CTAs per consumer."""
    from tests.test_gpu_channels import _check_mpsc_nl
    w = configs.mpsc(0)
    run = bench.MpscRun(h, inst, w, group=group, nonlocking=True, consumer_ctas=ctas)
    st, res = run.run()
    assert st == 0
    assert sum(int(r.consumed) for r in res) == w.sizes.size
    _check_mpsc_nl(w, run, res, sample=0.003)
    run.free()
