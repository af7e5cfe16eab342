"""Copies between the GPU's HBM and page-locked Grace host memory (the host
memory space, HiCR paper Sec. 3.1.2-3.1.4): rejected by default (reading r6),
byte-exact against the oracle once the pair is enabled."""
import numpy as np
import pytest
import torch

from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, fill_key, h, inst  # noqa: F401

pytestmark = pytest.mark.gpu

T = 30_000_000_000
ALL_PAIRS = ((om.SPACE_HBM, om.SPACE_HBM), (om.SPACE_HBM, om.SPACE_HOST), (om.SPACE_HOST, om.SPACE_HBM),
             (om.SPACE_HOST, om.SPACE_HOST))


def slot_view(h, inst, sid):
    st, ptr, size, space, _ = h.hicr_slot_info(inst, sid)
    torch.cuda.synchronize()
    if space == h.HICR_SPACE_HOST:
        return h.host_bytes(ptr, size).copy()
    return device_bytes(ptr, size).cpu().numpy()


def test_host_pairs_rejected_by_default(h, inst):
    st, a = h.hicr_mem_alloc(inst, h.HICR_SPACE_HBM, 4096)
    st, hs = h.hicr_mem_alloc(inst, h.HICR_SPACE_HOST, 4096)
    assert h.hicr_memcpy(inst, hs, 0, a, 0, 16) == h.HICR_ERR_UNSUPPORTED
    assert h.hicr_memcpy(inst, a, 0, hs, 0, 16) == h.HICR_ERR_UNSUPPORTED
    assert h.hicr_set_host_copies(inst, 1) == 0
    assert h.hicr_memcpy(inst, hs, 0, a, 0, 16) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    assert h.hicr_set_host_copies(inst, 0) == 0
    assert h.hicr_memcpy(inst, hs, 0, a, 0, 16) == h.HICR_ERR_UNSUPPORTED


@pytest.mark.parametrize("path,engine", [("batch", 0), ("device", 0), ("device", 1)])
def test_hbm_host_copies_match_oracle(h, inst, path, engine):
    """engine 1: the TMA engine, which must leave pieces with a host end to the
    vector copy (its bulk copies are for HBM pairs only)."""
    if engine == 1:
        st, c = h.hicr_batch_get_config(inst)
        c.engine, c.tma_min_bytes, c.threads, c.blocks_per_sm = 1, 1024, 256, 1
        assert h.hicr_batch_set_config(inst, c) == 0
    size = 4 << 20
    spaces = [h.HICR_SPACE_HBM, h.HICR_SPACE_HOST, h.HICR_SPACE_HBM, h.HICR_SPACE_HOST]
    ids = []
    for s, sp in enumerate(spaces):
        st, sid = h.hicr_mem_alloc(inst, sp, size)
        assert st == 0
        assert h.hicr_util_fill(inst, sid, 0, size, fill_key(9, s)) == 0
        ids.append(sid)
    assert h.hicr_set_host_copies(inst, 1) == 0
    cm = om.CommManager(supported_pairs=ALL_PAIRS)
    oids = [cm.register(sp, splitmix.fill_bytes(9, s, 0, size)) for s, sp in enumerate(spaces)]
    # three epochs (a fence between them): HBM -> host, host -> HBM, host -> host;
    # sizes 1 B - 256 KiB, arbitrary (also misaligned) offsets, destinations
    # disjoint within each slot and never read in the same epoch
    rng = np.random.default_rng(2)
    cursor = [0] * 4
    epochs = []
    for pairs in ([(1, 0), (3, 2), (1, 2)], [(0, 1), (2, 3), (0, 3)], [(1, 3)]):
        dst, src, doff, soff, n = [], [], [], [], []
        for k in range(150):
            d, s_ = pairs[k % len(pairs)]
            nn = int(np.exp(rng.uniform(0, np.log(256 << 10))))
            do = cursor[d] + int(rng.integers(0, 64))
            if do + nn > size:
                continue
            cursor[d] = do + nn
            dst.append(d), src.append(s_), doff.append(do), soff.append(int(rng.integers(0, size - nn))), n.append(nn)
        e = configs.make_ops(dst, src, doff, soff, n)
        assert len(e) > 20 and om.first_hazard(e) is None
        epochs.append(e)
    for e in epochs:
        assert cm.memcpy_batch(e) == (om.OK, None)
        lops = e.copy()
        lops["dst"] = np.asarray(ids, dtype=np.uint32)[e["dst"]]
        lops["src"] = np.asarray(ids, dtype=np.uint32)[e["src"]]
        if path == "batch":
            assert h.hicr_memcpy_batch(inst, lops) == (0, 0)
        else:
            t = torch.from_numpy(lops.view(np.uint8).copy()).cuda()
            assert h.hicr_memcpy_batch_device(inst, t.data_ptr(), len(lops)) == 0
        assert h.hicr_fence(inst, 0, T) == 0
    for k in range(4):
        assert (slot_view(h, inst, ids[k]) == cm.slots[oids[k]].data).all(), k
        assert h.hicr_slot_counters(inst, ids[k])[1:] == cm.counters(oids[k])


def test_registered_pinned_tensor_as_host_slot(h, inst):
    host = torch.arange(1 << 16, dtype=torch.int32).view(torch.uint8).pin_memory()
    dev = torch.zeros(1 << 18, dtype=torch.uint8, device="cuda")
    st, hs = h.hicr_slot_register(inst, h.HICR_SPACE_HOST, host.data_ptr(), host.numel())
    st2, ds = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, dev.data_ptr(), dev.numel())
    assert st == 0 and st2 == 0
    assert h.hicr_set_host_copies(inst, 1) == 0
    assert h.hicr_memcpy(inst, ds, 3, hs, 5, 100_000) == 0
    assert h.hicr_fence(inst, 0, T) == 0
    exp = np.zeros(1 << 18, dtype=np.uint8)
    exp[3:100_003] = host.numpy()[5:100_005]
    assert (dev.cpu().numpy() == exp).all()
