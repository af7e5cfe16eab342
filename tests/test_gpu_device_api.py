"""Device-side channel calls (include/hicr_device.cuh) against the oracle.

A small kernel library (tests/device_api_kernels.cu) is compiled with nvcc
for sm_103a and calls the header's warp-collective functions:
  * SPSC: a producer warp and a consumer warp in one cooperative grid carry
    tokens through a small ring (many wrap-arounds); the consumer's output is
    the exact token stream;
  * MPSC: producer warps push their messages while one consumer warp pops
    them; the consumption log passes the interleaving-agnostic checker
    (per-producer order, sizes, offsets replayed from the placement rule)
    and every payload equals the oracle's;
  * the state is shared with the host calls: tokens pushed by the host are
    popped on the device and the reverse, matching the oracle's FIFO.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

from oracle import channels as oc
from oracle import memcpy as om
from workloads import configs, splitmix
from tests.gpu_util import device_bytes, h, inst  # noqa: F401

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T = 10_000_000_000


class MsgInfo(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_uint64), ("size", ctypes.c_uint64), ("producer", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("seq", ctypes.c_uint64)]


@pytest.fixture(scope="module")
def dev():
    out = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "libdevapi.so")
    src = os.path.join(ROOT, "tests", "device_api_kernels.cu")
    deps = [src, os.path.join(ROOT, "include", "hicr_device.cuh"), os.path.join(ROOT, "include", "hicr_channels.h")]
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(d) for d in deps):
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-shared",
                        "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"), src, "-o", so + ".tmp"],
                       check=True)
        os.replace(so + ".tmp", so)
    lib = ctypes.CDLL(so)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.devapi_spsc.argtypes = [vp, vp, vp, u32, u32, u64, i32, vp]
    lib.devapi_mpsc.argtypes = [vp, vp, vp, vp, u32, u32, i32, vp, u64, vp, u64, vp]
    lib.devapi_mpsc_pop.argtypes = [vp, u64, vp, u64, vp, u64, vp]
    lib.devapi_nl.argtypes = [vp, vp, vp, vp, u32, u32, i32, vp, u64, vp, u64, vp]
    return lib


def _view(h, inst, ch):
    st, v = h.hicr_channel_device_view(inst, ch)
    assert st == 0
    return v


def _status():
    return torch.zeros(2, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("ts,cap,n,batch", [(64, 16, 5000, 4), (16, 7, 999, 3), (24, 64, 4096, 64), (1, 5, 300, 2)])
def test_device_spsc_roundtrip(h, inst, dev, ts, cap, n, batch):
    st, ch = h.hicr_spsc_create(inst, ts, cap)
    assert st == 0
    v = _view(h, inst, ch)
    data = np.random.default_rng(ts + cap).integers(0, 256, n * ts, dtype=np.uint8)
    src = torch.from_numpy(data).cuda()
    dst = torch.zeros(n * ts, dtype=torch.uint8, device="cuda")
    status = _status()
    assert dev.devapi_spsc(ctypes.byref(v), src.data_ptr(), dst.data_ptr(), n, batch, T, 0, status.data_ptr()) == 0
    assert status.cpu().tolist() == [0, 0]
    assert (dst.cpu().numpy() == data).all()
    assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    assert h.hicr_channel_destroy(inst, ch) == 0


def test_device_spsc_shares_state_with_the_host(h, inst, dev):
    ts, cap = 32, 8
    st, ch = h.hicr_spsc_create(inst, ts, cap)
    v = _view(h, inst, ch)
    orc = oc.SpscOracle(ts, cap)
    pool = np.random.default_rng(1).integers(0, 256, 64 * ts, dtype=np.uint8)
    pt = torch.from_numpy(pool).cuda()
    st, s = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, pt.data_ptr(), pt.numel())
    status = _status()
    # host pushes 5, the device pops 3
    assert h.hicr_channel_push(inst, ch, 0, s, 0, 5) == orc.push(pool[:5 * ts]) == om.OK
    out = torch.zeros(3 * ts, dtype=torch.uint8, device="cuda")
    assert dev.devapi_spsc(ctypes.byref(v), 0, out.data_ptr(), 3, 3, T, 2, status.data_ptr()) == 0
    assert (out.cpu().numpy() == np.concatenate([orc.token(k) for k in range(3)])).all()
    assert orc.pop(3) == om.OK
    # the device pushes 6 (wrapping), the host peeks and pops
    assert dev.devapi_spsc(ctypes.byref(v), pt.data_ptr() + 10 * ts, 0, 6, 2, T, 1, status.data_ptr()) == 0
    assert orc.push(pool[10 * ts:16 * ts]) == om.OK
    assert status.cpu().tolist() == [0, 0]
    assert h.hicr_channel_depth(inst, ch)[1:] == orc.depth() == (8, 8 * ts)
    for k in range(8):
        est, info = orc.peek(k)
        gst, ginfo = h.hicr_channel_peek(inst, ch, k)
        assert gst == est == om.OK and ginfo == info
    # full: a device push of one more token gives up after its timeout
    assert dev.devapi_spsc(ctypes.byref(v), pt.data_ptr(), 0, 1, 1, 2_000_000, 1, status.data_ptr()) == 0
    assert status.cpu().tolist()[0] == h.HICR_ERR_TIMEOUT
    assert h.hicr_channel_pop(inst, ch, 8) == orc.pop(8) == om.OK
    assert h.hicr_slot_deregister(inst, s) == 0
    assert h.hicr_channel_destroy(inst, ch) == 0


def _mpsc_inputs(P, M, hi, seed):
    w = configs.mpsc(seed, n_producers=P, n_consumers=1, msgs_per_producer=M, ring_bytes=1 << 20, max_msgs=64,
                     hi=hi)
    sizes = w.sizes.reshape(-1).astype(np.uint64)
    offs = np.zeros(len(sizes), dtype=np.uint64)
    offs[1:] = np.cumsum((sizes + np.uint64(15)) // np.uint64(16) * np.uint64(16))[:-1]
    staging = np.zeros(int(offs[-1] + sizes[-1]) + 16, dtype=np.uint8)
    for p in range(P):
        for q in range(M):
            i = p * M + q
            staging[int(offs[i]):int(offs[i]) + int(sizes[i])] = splitmix.mpsc_payload_bytes(p, q, int(sizes[i]))
    return w, sizes, offs, staging


@pytest.mark.parametrize("P,M,ring,max_msgs,hi", [(8, 40, 1 << 14, 16, 3000), (3, 100, 1 << 12, 4, 2000),
                                                  (16, 8, 1 << 16, 64, 16 << 10)])
def test_device_mpsc_producers_and_consumer(h, inst, dev, P, M, ring, max_msgs, hi):
    w, sizes, offs, staging = _mpsc_inputs(P, M, hi, P)
    st, ch = h.hicr_mpsc_create(inst, P, ring, max_msgs)
    assert st == 0
    v = _view(h, inst, ch)
    d_st = torch.from_numpy(staging).cuda()
    d_off = torch.from_numpy(offs.view(np.int64).copy()).cuda()
    d_sz = torch.from_numpy(sizes.view(np.int64).copy()).cuda()
    stride = int(((sizes.max() + 15) // 16) * 16)
    out = torch.zeros(P * M * stride, dtype=torch.uint8, device="cuda")
    infos = torch.zeros(P * M * ctypes.sizeof(MsgInfo), dtype=torch.uint8, device="cuda")
    status = _status()
    assert dev.devapi_mpsc(ctypes.byref(v), d_st.data_ptr(), d_off.data_ptr(), d_sz.data_ptr(), P, M, 1,
                           out.data_ptr(), stride, infos.data_ptr(), T, status.data_ptr()) == 0
    assert status.cpu().tolist() == [0, 0]
    info = np.frombuffer(infos.cpu().numpy().tobytes(), dtype=np.dtype([("offset", "<u8"), ("size", "<u8"),
                                                                       ("producer", "<u4"), ("reserved", "<u4"),
                                                                       ("seq", "<u8")]))
    log = list(zip(info["producer"], info["seq"], info["size"], info["offset"]))
    assert oc.check_mpsc_log(w.sizes, 1, 0, log, ring) == []
    o = out.cpu().numpy().reshape(P * M, stride)
    for j, (p, q, n, _) in enumerate(log):
        assert (o[j, :int(n)] == splitmix.mpsc_payload_bytes(int(p), int(q), int(n))).all(), j
    assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    assert h.hicr_channel_destroy(inst, ch) == 0


def test_device_mpsc_interoperates_with_host_calls(h, inst, dev):
    """Device producers fill the ring (no consumer), the host peeks and pops
    it in ticket order; then host pushes are popped by a device consumer.
    Both halves against the locking-mode oracle's FIFO."""
    P, M, ring = 4, 6, 1 << 16
    w, sizes, offs, staging = _mpsc_inputs(P, M, 1500, 21)
    st, ch = h.hicr_mpsc_create(inst, P, ring, 64)
    v = _view(h, inst, ch)
    d_st = torch.from_numpy(staging).cuda()
    d_off = torch.from_numpy(offs.view(np.int64).copy()).cuda()
    d_sz = torch.from_numpy(sizes.view(np.int64).copy()).cuda()
    status = _status()
    assert dev.devapi_mpsc(ctypes.byref(v), d_st.data_ptr(), d_off.data_ptr(), d_sz.data_ptr(), P, M, 0, 0, 16, 0,
                           T, status.data_ptr()) == 0
    assert status.cpu().tolist() == [0, 0]
    assert h.hicr_channel_depth(inst, ch)[1] == P * M
    log = []
    for k in range(P * M):
        gst, (off, n, p, q) = h.hicr_channel_peek(inst, ch, k)
        assert gst == 0
        log.append((p, q, n, off))
    assert oc.check_mpsc_log(w.sizes, 1, 0, log, ring) == []
    assert h.hicr_channel_pop(inst, ch, P * M) == 0
    # host pushes, device consumer: FIFO in push order
    st, s = h.hicr_slot_register(inst, h.HICR_SPACE_HBM, d_st.data_ptr(), d_st.numel())
    pushed = []
    for i in range(10):
        p, q = i % P, i // P
        n = int(sizes[p * M + q])
        assert h.hicr_channel_push(inst, ch, p, s, int(offs[p * M + q]), n) == 0
        pushed.append((p, n, staging[int(offs[p * M + q]):int(offs[p * M + q]) + n]))
    stride = 1504
    out = torch.zeros(10 * stride, dtype=torch.uint8, device="cuda")
    infos = torch.zeros(10 * ctypes.sizeof(MsgInfo), dtype=torch.uint8, device="cuda")
    assert dev.devapi_mpsc_pop(ctypes.byref(v), 10, out.data_ptr(), stride, infos.data_ptr(), T,
                               status.data_ptr()) == 0
    assert status.cpu().tolist() == [0, 0]
    o = out.cpu().numpy().reshape(10, stride)
    info = np.frombuffer(infos.cpu().numpy().tobytes(), dtype=np.dtype([("offset", "<u8"), ("size", "<u8"),
                                                                       ("producer", "<u4"), ("reserved", "<u4"),
                                                                       ("seq", "<u8")]))
    for j, (p, n, payload) in enumerate(pushed):
        assert int(info["producer"][j]) == p and int(info["size"][j]) == n
        assert (o[j, :n] == payload).all()
    assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    assert h.hicr_slot_deregister(inst, s) == 0
    assert h.hicr_channel_destroy(inst, ch) == 0


INFO_DTYPE = np.dtype([("offset", "<u8"), ("size", "<u8"), ("producer", "<u4"), ("reserved", "<u4"), ("seq", "<u8")])


@pytest.mark.parametrize("P,M,ring,max_msgs,hi", [(6, 30, 1 << 12, 8, 1500), (40, 5, 1 << 13, 4, 3000)])
def test_device_nonlocking_producers_and_consumer(h, inst, dev, P, M, ring, max_msgs, hi):
    """Producer warps push into their own rings (waiting for room as the
    rings wrap) while one consumer warp pops with pop_any: every message once,
    per-producer order, offsets replayed per ring, payloads exact."""
    w, sizes, offs, staging = _mpsc_inputs(P, M, hi, 40 + P)
    st, ch = h.hicr_mpsc_nl_create(inst, P, ring, max_msgs)
    assert st == 0
    v = _view(h, inst, ch)
    assert (v.kind, v.capacity, v.ring_bytes, v.max_msgs) == (2, P, ring, max_msgs)
    d_st = torch.from_numpy(staging).cuda()
    d_off = torch.from_numpy(offs.view(np.int64).copy()).cuda()
    d_sz = torch.from_numpy(sizes.view(np.int64).copy()).cuda()
    stride = int(((sizes.max() + 15) // 16) * 16)
    out = torch.zeros(P * M * stride, dtype=torch.uint8, device="cuda")
    infos = torch.zeros(P * M * INFO_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    status = _status()
    assert dev.devapi_nl(ctypes.byref(v), d_st.data_ptr(), d_off.data_ptr(), d_sz.data_ptr(), P, M, 1,
                         out.data_ptr(), stride, infos.data_ptr(), T, status.data_ptr()) == 0
    assert status.cpu().tolist() == [0, 0]
    info = np.frombuffer(infos.cpu().numpy().tobytes(), dtype=INFO_DTYPE)
    log = list(zip(info["producer"], info["seq"], info["size"], info["offset"]))
    assert oc.check_mpsc_nl_log(w.sizes, 1, 0, log, ring) == []
    o = out.cpu().numpy().reshape(P * M, stride)
    for j, (p, q, n, _) in enumerate(log):
        assert (o[j, :int(n)] == splitmix.mpsc_payload_bytes(int(p), int(q), int(n))).all(), j
    assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    assert h.hicr_channel_destroy(inst, ch) == 0


def test_device_nonlocking_push_host_drain(h, inst, dev):
    """Device producers fill their rings (no consumer); the host's peek and
    pop see the non-locking oracle's order (producers in index order, each
    producer's messages oldest first) with its offsets and payloads."""
    P, M, ring = 5, 4, 1 << 14
    w, sizes, offs, staging = _mpsc_inputs(P, M, 2000, 77)
    st, ch = h.hicr_mpsc_nl_create(inst, P, ring, 8)
    v = _view(h, inst, ch)
    d_st = torch.from_numpy(staging).cuda()
    d_off = torch.from_numpy(offs.view(np.int64).copy()).cuda()
    d_sz = torch.from_numpy(sizes.view(np.int64).copy()).cuda()
    status = _status()
    assert dev.devapi_nl(ctypes.byref(v), d_st.data_ptr(), d_off.data_ptr(), d_sz.data_ptr(), P, M, 0, 0, 16, 0, T,
                         status.data_ptr()) == 0
    assert status.cpu().tolist() == [0, 0]
    orc = oc.MpscNonLockingOracle(P, ring, 8)
    for p in range(P):
        for q in range(M):
            i = p * M + q
            assert orc.push(p, staging[int(offs[i]):int(offs[i]) + int(sizes[i])]) == om.OK
    assert h.hicr_channel_depth(inst, ch)[1:] == orc.depth()
    st, rs = h.hicr_channel_ring(inst, ch)
    st, rptr, _, _, _ = h.hicr_slot_info(inst, rs)
    torch.cuda.synchronize()
    rings = device_bytes(rptr, P * ring).cpu().numpy()
    for k in range(P * M):
        est, einfo = orc.peek(k)
        gst, ginfo = h.hicr_channel_peek(inst, ch, k)
        assert gst == est == om.OK and ginfo == einfo, k
        o, n, p, q = ginfo
        assert (rings[p * ring + o:p * ring + o + n] == orc.payload(k)).all(), k
    assert h.hicr_channel_pop(inst, ch, P * M) == orc.pop(P * M) == om.OK
    assert h.hicr_channel_depth(inst, ch)[1:] == (0, 0)
    assert h.hicr_channel_destroy(inst, ch) == 0


def test_device_view_of_every_kind(h, inst):
    st, a = h.hicr_spsc_create(inst, 64, 16)
    st, b = h.hicr_mpsc_create(inst, 3, 1 << 12, 8)
    st, c = h.hicr_mpsc_nl_create(inst, 2, 1 << 12, 4)
    assert [h.hicr_channel_device_view(inst, x)[1].kind for x in (a, b, c)] == [0, 1, 2]
    assert h.hicr_channel_device_view(inst, 12345)[0] == h.HICR_ERR_INVALID
    for x in (a, b, c):
        assert h.hicr_channel_destroy(inst, x) == 0
