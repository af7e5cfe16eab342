"""The seeded input generators: published SplitMix64 outputs and the
structural promises of each configuration."""
import numpy as np

from workloads import configs, splitmix


def test_splitmix64_published_first_outputs():
    # SplitMix64 started from state 0 (Steele, Lea & Flood 2014; Vigna's
    # public-domain splitmix64.c): the first three outputs.
    out = splitmix.sequence(0, 3)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert splitmix.H_int(0) == 0xE220A8397B1DCDAF
    assert splitmix.H_int(int(splitmix.GAMMA)) == 0x6E789E6AA1B965F4


def test_H_is_injective_on_a_window():
    k = np.arange(1 << 16, dtype=np.uint64) * np.uint64(0x10001)
    assert len(np.unique(splitmix.H(k))) == len(k)


def test_fill_bytes_windows_agree():
    whole = splitmix.fill_bytes(0, 3, 0, 4096)
    for a, n in [(0, 1), (1, 7), (7, 9), (13, 100), (4000, 96)]:
        assert (splitmix.fill_bytes(0, 3, a, n) == whole[a:a + n]).all()
    pos = np.array([0, 1, 7, 8, 4095])
    assert (splitmix.fill_byte_at(0, 3, pos) == whole[pos]).all()
    w = splitmix.fill_words(0, 3, 0, 1)[0]
    assert int(w) == splitmix.H_int(3 << 40)
    assert int.from_bytes(bytes(whole[:8]), "little") == int(w)


def test_tiny_config_shape():
    w = configs.tiny(0)
    o = w.ops
    assert len(o) == 1024 and (o["src"] == 0).all() and (o["dst"] == 1).all()
    n = o["n"].astype(np.int64)
    assert n.min() >= 1 and n.max() <= 65536
    assert ((o["src_off"].astype(np.int64) + n) <= (64 << 20)).all()
    s = o["dst_off"].astype(np.int64)
    idx = np.argsort(s)
    assert (s[idx][1:] >= (s + n)[idx][:-1]).all()
    assert ((s + n) <= (64 << 20)).all()
    assert (configs.tiny(0).ops == o).all()


def _epoch_nonoverlap(w):
    for a, b in w.epochs:
        e = w.ops[a:b]
        for s in np.unique(e["dst"]):
            m = e[e["dst"] == s]
            st = m["dst_off"].astype(np.int64)
            en = st + m["n"].astype(np.int64)
            idx = np.argsort(st)
            assert (st[idx][1:] >= en[idx][:-1]).all()
            assert en.max() <= int(w.slot_sizes[s])
    assert not np.isin(w.ops["dst"], w.src_slots).any()


def test_batched_small_shape():
    w = configs.batched_small(0)
    assert int(w.slot_sizes.sum()) == 256 << 20
    assert len(w.epochs) >= 2 and w.epochs[0][0] == 0 and w.epochs[-1][1] == len(w.ops)
    _epoch_nonoverlap(w)
    o = w.ops
    mis = (o["src_off"] % 16) != 0
    assert ((o["dst_off"] % 16 != 0) == mis).all()
    assert 0.05 < mis.mean() < 0.15
    n = o["n"].astype(np.int64)
    assert n.min() >= 16 and n.max() <= 1 << 20
    assert ((o["src_off"].astype(np.int64) + n) <= w.slot_sizes[o["src"]].astype(np.int64)).all()


def test_slot_sizes_rule():
    s = configs.slot_sizes_log_uniform(0, 256, 16 << 30, 1 << 20, 256 << 20)
    assert int(s.sum()) == 16 << 30
    assert s.min() >= 1 << 20 and s.max() <= 256 << 20 and (s % 4096 == 0).all()


def test_mpsc_sizes_and_mapping():
    w = configs.mpsc(0, n_producers=64, msgs_per_producer=32)
    assert w.sizes.shape == (64, 32) and w.sizes.min() >= 8 and w.sizes.max() <= 256 << 10
    assert w.consumer_of(17) == 1


def test_serve_trace_is_poisson_like():
    tr = configs.serve_trace(0, rate=20000.0, duration_s=2.0)
    n = len(tr.arrival_ns)
    assert abs(n - 40000) < 4 * np.sqrt(40000)
    assert (np.diff(tr.arrival_ns) >= 0).all()
    assert abs(tr.kind.mean() - 0.3) < 0.02
