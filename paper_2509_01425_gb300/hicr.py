"""ctypes binding of libhicr_gb300.so: the C-ABI calls under the same names.

Argument marshalling only. Every function returns the hicr_status code first,
followed by its out-parameters, e.g. ``st, inst = hicr_init(0)``. ``check``
turns a non-zero status into ``HicrError``. Buffers may be passed as integers
(addresses), numpy arrays or objects exposing ``data_ptr()`` (torch tensors).

The library must have been built (``paper_2509_01425_gb300.build.build()``);
importing this module without it raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhicr_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2509_01425_gb300.build.build()")
lib = C.CDLL(LIB_PATH)

# ---------------------------------------------------------------------------
# Constants (values of include/hicr.h)
# ---------------------------------------------------------------------------
HICR_OK = 0
HICR_ERR_INVALID = -1
HICR_ERR_UNSUPPORTED = -2
HICR_ERR_BOUNDS = -3
HICR_ERR_OVERLAP = -4
HICR_ERR_HAZARD = -5
HICR_ERR_NOMEM = -6
HICR_ERR_FULL = -7
HICR_ERR_EMPTY = -8
HICR_ERR_TOO_LARGE = -9
HICR_ERR_TIMEOUT = -10
HICR_ERR_BUSY = -11
HICR_ERR_DEVICE = -12

HICR_NOALLOC_MAX_OPS = 32768
HICR_MAX_SLOTS = 65536
HICR_MAX_TAGS = 1024
HICR_MAX_SPACES = 4
HICR_MAX_RESOURCES = 4
HICR_SPACE_HBM = 0
HICR_SPACE_HOST = 1
HICR_RESOURCE_GPU = 0

u8, u32, u64, i32 = C.c_uint8, C.c_uint32, C.c_uint64, C.c_int32
vp = C.c_void_p


class hicr_op_t(C.Structure):
    _fields_ = [("dst", u32), ("src", u32), ("dst_off", u64), ("src_off", u64), ("n", u64)]


class hicr_memory_space_t(C.Structure):
    _fields_ = [("id", u32), ("kind", u32), ("device", i32), ("peak_mbps", u32),
                ("phys_size", u64), ("free_size", u64)]


class hicr_compute_resource_t(C.Structure):
    _fields_ = [("id", u32), ("kind", u32), ("device", i32), ("sm_count", u32),
                ("max_threads_per_sm", u32), ("cc_major", u32), ("cc_minor", u32), ("reserved", u32),
                ("l2_bytes", u64), ("smem_per_block_optin", u64)]


class hicr_topology_t(C.Structure):
    _fields_ = [("device", i32), ("n_spaces", u32), ("n_resources", u32), ("reserved", u32),
                ("name", C.c_char * 128), ("spaces", hicr_memory_space_t * HICR_MAX_SPACES),
                ("resources", hicr_compute_resource_t * HICR_MAX_RESOURCES)]


class hicr_batch_config_t(C.Structure):
    _fields_ = [("chunk_bytes", u32), ("op_cost_bytes", u32), ("blocks_per_sm", u32), ("threads", u32),
                ("engine", u32), ("tma_min_bytes", u32), ("tma_stage_bytes", u32), ("tma_stages", u32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class hicr_exec_unit_t(C.Structure):
    _fields_ = [("func", vp), ("grid", u32 * 3), ("block", u32 * 3), ("smem_bytes", u32), ("n_args", u32)]


class HicrError(RuntimeError):
    def __init__(self, status, what=""):
        super().__init__(f"{what}: {hicr_status_str(status)} ({status})")
        self.status = status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, C.Array) or isinstance(x, C.Structure):
        return C.addressof(x)
    raise TypeError(f"cannot take the address of {type(x)}")


def _decl(name, args, res=i32):
    f = getattr(lib, name)
    f.argtypes = args
    f.restype = res
    return f


H = vp  # hicr_instance_t

_status_str = _decl("hicr_status_str", [i32], C.c_char_p)
_init = _decl("hicr_init", [C.c_int, C.POINTER(vp)])
_finalize = _decl("hicr_finalize", [H])
_is_root = _decl("hicr_is_root", [H, C.POINTER(i32)])
_topology = _decl("hicr_topology_query", [H, C.POINTER(hicr_topology_t)])
_mem_alloc = _decl("hicr_mem_alloc", [H, u32, u64, u32, C.POINTER(u32)])
_mem_free = _decl("hicr_mem_free", [H, u32])
_slot_register = _decl("hicr_slot_register", [H, u32, vp, u64, u32, C.POINTER(u32)])
_slot_deregister = _decl("hicr_slot_deregister", [H, u32])
_slot_info = _decl("hicr_slot_info", [H, u32, C.POINTER(vp), C.POINTER(u64), C.POINTER(u32), C.POINTER(u32)])
_memcpy = _decl("hicr_memcpy", [H, u32, u64, u32, u64, u64])
_flush = _decl("hicr_flush", [H])
_memcpy_batch = _decl("hicr_memcpy_batch", [H, vp, u64, C.POINTER(u64)])
_memcpy_batch_device = _decl("hicr_memcpy_batch_device", [H, vp, u64])
_memcpy_batch_noalloc = _decl("hicr_memcpy_batch_noalloc", [H, vp, u64])
_batch_error = _decl("hicr_batch_error", [H, C.POINTER(i32), C.POINTER(u64)])
_batch_reserve = _decl("hicr_batch_reserve", [H, u64])
_set_checked = _decl("hicr_set_checked", [H, i32])
_set_host_copies = _decl("hicr_set_host_copies", [H, i32])
_set_latency_mode = _decl("hicr_set_latency_mode", [H, u32])
_fence = _decl("hicr_fence", [H, u32, u64])
_fence_slot = _decl("hicr_fence_slot", [H, u32, u64, u64, u64])
_slot_counters = _decl("hicr_slot_counters", [H, u32, C.POINTER(u64), C.POINTER(u64)])
_slot_counters_range = _decl("hicr_slot_counters_range", [H, u32, u32, vp, vp])
_tag_counter = _decl("hicr_tag_counter", [H, u32, C.POINTER(u64)])
_memcpy_batch_plain = _decl("hicr_memcpy_batch_plain", [H, vp, u64, C.POINTER(u64)])
_batch_get_config = _decl("hicr_batch_get_config", [H, C.POINTER(hicr_batch_config_t)])
_batch_set_config = _decl("hicr_batch_set_config", [H, C.POINTER(hicr_batch_config_t)])
_batch_autotune = _decl("hicr_batch_autotune", [H, vp, u64, u32, C.POINTER(hicr_batch_config_t),
                                                C.POINTER(C.c_float)])
_graph_begin = _decl("hicr_graph_begin", [H])
_graph_end = _decl("hicr_graph_end", [H, C.POINTER(u64)])
_graph_launch = _decl("hicr_graph_launch", [H, u64])
_graph_destroy = _decl("hicr_graph_destroy", [H, u64])
_profile_enable = _decl("hicr_profile_enable", [H, i32])
_profile_reset = _decl("hicr_profile_reset", [H])
_profile_read = _decl("hicr_profile_read", [H, C.POINTER(C.c_float), C.POINTER(u32)])
_pu_create = _decl("hicr_pu_create", [H, vp, C.POINTER(u32)])
_pu_destroy = _decl("hicr_pu_destroy", [H, u32])
_pu_stream = _decl("hicr_pu_stream", [H, u32, C.POINTER(vp)])
_comm_set_pu = _decl("hicr_comm_set_pu", [H, u32])
_exec_unit_builtin = _decl("hicr_exec_unit_builtin", [C.c_char_p, C.POINTER(hicr_exec_unit_t)])
_exec_launch = _decl("hicr_exec_launch", [H, u32, C.POINTER(hicr_exec_unit_t), C.POINTER(vp), C.POINTER(u64)])
_exec_query = _decl("hicr_exec_query", [H, u64, C.POINTER(i32)])
_exec_await = _decl("hicr_exec_await", [H, u64, u64])
_last_error_string = _decl("hicr_last_error_string", [H, C.c_char_p, u64])
_util_fill = _decl("hicr_util_fill", [H, u32, u64, u64, u64])
_util_fill_segments = _decl("hicr_util_fill_segments", [H, u32, vp, u64])
_util_wait_test = _decl("hicr_util_wait_test", [H, u64, C.POINTER(i32), C.POINTER(u64)])
_util_digest = _decl("hicr_util_digest", [H, u32, u64, u64, C.POINTER(u64)])
_util_copy_loop = _decl("hicr_util_copy_loop", [H, u32, u64, u32, u64, u64, u32, u32, C.POINTER(u64)])
_util_stream = _decl("hicr_util_stream", [H, u32, u64, u64, i32, u32, u32, C.POINTER(u64)])


def hicr_status_str(s: int) -> str:
    return _status_str(s).decode()


def check(st, what="hicr"):
    """Raise HicrError unless st (or st[0] of a tuple) is HICR_OK; return the outs."""
    if isinstance(st, tuple):
        if st[0] != HICR_OK:
            raise HicrError(st[0], what)
        return st[1] if len(st) == 2 else st[1:]
    if st != HICR_OK:
        raise HicrError(st, what)
    return None


def hicr_init(device: int = 0):
    h = vp()
    st = _init(device, C.byref(h))
    return st, h


def hicr_finalize(inst):
    return _finalize(inst)


def hicr_is_root(inst):
    v = i32()
    st = _is_root(inst, C.byref(v))
    return st, v.value


def hicr_topology_query(inst):
    t = hicr_topology_t()
    st = _topology(inst, C.byref(t))
    return st, t


def hicr_mem_alloc(inst, space, size, tag=0):
    s = u32()
    st = _mem_alloc(inst, space, size, tag, C.byref(s))
    return st, s.value


def hicr_mem_free(inst, slot):
    return _mem_free(inst, slot)


def hicr_slot_register(inst, space, ptr, size, tag=0):
    s = u32()
    st = _slot_register(inst, space, _ptr(ptr), size, tag, C.byref(s))
    return st, s.value


def hicr_slot_deregister(inst, slot):
    return _slot_deregister(inst, slot)


def hicr_slot_info(inst, slot):
    p, n, sp, tg = vp(), u64(), u32(), u32()
    st = _slot_info(inst, slot, C.byref(p), C.byref(n), C.byref(sp), C.byref(tg))
    return st, (p.value or 0), n.value, sp.value, tg.value


def hicr_memcpy(inst, dst, dst_off, src, src_off, n):
    return _memcpy(inst, dst, dst_off, src, src_off, n)


def hicr_flush(inst):
    return _flush(inst)


def _ops_ptr(ops):
    if isinstance(ops, np.ndarray):
        if ops.dtype.itemsize != 32 or not ops.flags.c_contiguous:
            raise TypeError("op table must be a C-contiguous array of 32-byte records")
        return ops.ctypes.data, len(ops)
    raise TypeError("op table must be a numpy structured array")


def hicr_memcpy_batch(inst, ops):
    p, n = _ops_ptr(ops)
    bad = u64(0)
    st = _memcpy_batch(inst, p, n, C.byref(bad))
    return st, bad.value


def hicr_memcpy_batch_device(inst, d_ops, count):
    return _memcpy_batch_device(inst, _ptr(d_ops), count)


def hicr_memcpy_batch_noalloc(inst, d_ops, count):
    return _memcpy_batch_noalloc(inst, _ptr(d_ops), count)


def hicr_batch_error(inst):
    s, b = i32(), u64()
    st = _batch_error(inst, C.byref(s), C.byref(b))
    return st, s.value, b.value


def hicr_batch_reserve(inst, max_ops):
    return _batch_reserve(inst, max_ops)


def hicr_set_checked(inst, on):
    return _set_checked(inst, 1 if on else 0)


def hicr_set_latency_mode(inst, idle_us):
    return _set_latency_mode(inst, idle_us)


def hicr_set_host_copies(inst, on):
    return _set_host_copies(inst, 1 if on else 0)


def host_bytes(ptr, nbytes):
    """numpy uint8 view of host memory [ptr, ptr+nbytes) (no copy)."""
    if nbytes == 0:
        return np.zeros(0, dtype=np.uint8)
    return np.ctypeslib.as_array((C.c_uint8 * nbytes).from_address(ptr))


def hicr_fence(inst, tag=0, timeout_ns=30_000_000_000):
    return _fence(inst, tag, timeout_ns)


def hicr_fence_slot(inst, slot, expect_sent, expect_recv, timeout_ns=30_000_000_000):
    return _fence_slot(inst, slot, expect_sent, expect_recv, timeout_ns)


def hicr_slot_counters(inst, slot):
    s, r = u64(), u64()
    st = _slot_counters(inst, slot, C.byref(s), C.byref(r))
    return st, s.value, r.value


def hicr_slot_counters_range(inst, first, count):
    sent = np.zeros(count, dtype=np.uint64)
    recv = np.zeros(count, dtype=np.uint64)
    st = _slot_counters_range(inst, first, count, sent.ctypes.data, recv.ctypes.data)
    return st, sent, recv


def hicr_tag_counter(inst, tag):
    v = u64()
    st = _tag_counter(inst, tag, C.byref(v))
    return st, v.value


def hicr_memcpy_batch_plain(inst, ops):
    p, n = _ops_ptr(ops)
    bad = u64(0)
    st = _memcpy_batch_plain(inst, p, n, C.byref(bad))
    return st, bad.value


def hicr_batch_get_config(inst):
    c = hicr_batch_config_t()
    st = _batch_get_config(inst, C.byref(c))
    return st, c


def hicr_batch_set_config(inst, cfg):
    if isinstance(cfg, dict):
        c = hicr_batch_config_t()
        for k, v in cfg.items():
            setattr(c, k, v)
        cfg = c
    return _batch_set_config(inst, C.byref(cfg))


def hicr_batch_autotune(inst, d_ops, count, reps=3):
    c = hicr_batch_config_t()
    ms = C.c_float()
    st = _batch_autotune(inst, _ptr(d_ops), count, reps, C.byref(c), C.byref(ms))
    return st, c, ms.value


def hicr_graph_begin(inst):
    return _graph_begin(inst)


def hicr_graph_end(inst):
    g = u64()
    st = _graph_end(inst, C.byref(g))
    return st, g.value


def hicr_graph_launch(inst, g):
    return _graph_launch(inst, g)


def hicr_graph_destroy(inst, g):
    return _graph_destroy(inst, g)


def hicr_profile_enable(inst, on):
    return _profile_enable(inst, 1 if on else 0)


def hicr_profile_reset(inst):
    return _profile_reset(inst)


def hicr_profile_read(inst):
    ms, n = C.c_float(), u32()
    st = _profile_read(inst, C.byref(ms), C.byref(n))
    return st, ms.value, n.value


def hicr_pu_create(inst, stream=None):
    p = u32()
    st = _pu_create(inst, _ptr(stream) if stream is not None else None, C.byref(p))
    return st, p.value


def hicr_pu_destroy(inst, pu):
    return _pu_destroy(inst, pu)


def hicr_pu_stream(inst, pu):
    s = vp()
    st = _pu_stream(inst, pu, C.byref(s))
    return st, (s.value or 0)


def hicr_comm_set_pu(inst, pu):
    return _comm_set_pu(inst, pu)


def hicr_exec_unit_builtin(name):
    u = hicr_exec_unit_t()
    st = _exec_unit_builtin(name.encode(), C.byref(u))
    return st, u


def hicr_exec_launch(inst, pu, unit, arg_values):
    """arg_values: list of ctypes scalars (c_void_p, c_uint64, ...) in kernel
    parameter order; their addresses are passed as cudaLaunchKernel expects."""
    arr = (vp * max(1, len(arg_values)))(*[C.cast(C.pointer(a), vp) for a in arg_values])
    e = u64()
    st = _exec_launch(inst, pu, C.byref(unit), arr, C.byref(e))
    return st, e.value


def hicr_exec_query(inst, e):
    d = i32()
    st = _exec_query(inst, e, C.byref(d))
    return st, d.value


def hicr_exec_await(inst, e, timeout_ns=30_000_000_000):
    return _exec_await(inst, e, timeout_ns)


def hicr_last_error_string(inst):
    buf = C.create_string_buffer(1024)
    st = _last_error_string(inst, buf, 1024)
    return st, buf.value.decode(errors="replace")


def hicr_util_fill(inst, slot, off, n, key_base):
    return _util_fill(inst, slot, off, n, key_base)


def hicr_util_fill_segments(inst, slot, d_seg, count):
    return _util_fill_segments(inst, slot, _ptr(d_seg), count)


def hicr_util_wait_test(inst, timeout_ns):
    st_, w = i32(), u64()
    st = _util_wait_test(inst, timeout_ns, C.byref(st_), C.byref(w))
    return st, st_.value, w.value


def hicr_util_copy_loop(inst, dst, dst_off, src, src_off, n, reps, ctas):
    v = u64()
    st = _util_copy_loop(inst, dst, dst_off, src, src_off, n, reps, ctas, C.byref(v))
    return st, v.value


def hicr_util_stream(inst, slot, off, n, write, reps, ctas):
    v = u64()
    st = _util_stream(inst, slot, off, n, 1 if write else 0, reps, ctas, C.byref(v))
    return st, v.value


def hicr_util_digest(inst, slot, off, n):
    v = u64()
    st = _util_digest(inst, slot, off, n, C.byref(v))
    return st, v.value


# ---------------------------------------------------------------------------
# Channels (include/hicr_channels.h)
# ---------------------------------------------------------------------------
class hicr_msg_info_t(C.Structure):
    _fields_ = [("offset", u64), ("size", u64), ("producer", u32), ("reserved", u32), ("seq", u64)]


class hicr_spsc_result_t(C.Structure):
    _fields_ = [("pushed", u64), ("popped", u64), ("mismatches", u64), ("digest", u64),
                ("max_occupancy", u64), ("status", i32), ("reserved", u32)]


class hicr_mpsc_log_t(C.Structure):
    _fields_ = [("producer", u32), ("seq", u32), ("size", u32), ("reserved", u32), ("offset", u64),
                ("digest", u64)]


MPSC_LOG_DTYPE = np.dtype([("producer", "<u4"), ("seq", "<u4"), ("size", "<u4"), ("reserved", "<u4"),
                           ("offset", "<u8"), ("digest", "<u8")])


class hicr_mpsc_result_t(C.Structure):
    _fields_ = [("consumed", u64), ("bytes", u64), ("max_inflight_bytes", u64), ("max_inflight_msgs", u64),
                ("windows", u64), ("room_waits", u64), ("cas_failures", u64), ("consumer_ns", u64 * 3),
                ("status", i32), ("reserved", u32)]


_spsc_create = _decl("hicr_spsc_create", [H, u32, u32, C.POINTER(u32)])
_mpsc_create = _decl("hicr_mpsc_create", [H, u32, u64, u32, C.POINTER(u32)])
_mpsc_nl_create = _decl("hicr_mpsc_nl_create", [H, u32, u64, u32, C.POINTER(u32)])
_channel_destroy = _decl("hicr_channel_destroy", [H, u32])
_channel_ring = _decl("hicr_channel_ring", [H, u32, C.POINTER(u32)])
_channel_push = _decl("hicr_channel_push", [H, u32, u32, u32, u64, u64])
_channel_peek = _decl("hicr_channel_peek", [H, u32, u64, C.POINTER(hicr_msg_info_t)])
_channel_pop = _decl("hicr_channel_pop", [H, u32, u64])
_channel_depth = _decl("hicr_channel_depth", [H, u32, C.POINTER(u64), C.POINTER(u64)])
_spsc_stream = _decl("hicr_spsc_stream", [H, vp, u32, u64, u32, u64, vp])
_mpsc_stream = _decl("hicr_mpsc_stream", [H, vp, u32, u32, u32, vp, vp, u32, u32, u32, u64, vp, u64, vp])
_mpsc_nl_stream = _decl("hicr_mpsc_nl_stream", [H, vp, u32, u32, u32, vp, vp, u32, u32, u32, u64, vp, u64, vp])
_mpsc_stream_capture = _decl("hicr_mpsc_stream_capture",
                             [H, vp, u32, u32, u32, vp, vp, u32, u32, u32, u64, vp, u64, vp, vp, vp])
_mpsc_nl_stream_capture = _decl("hicr_mpsc_nl_stream_capture",
                                [H, vp, u32, u32, u32, vp, vp, u32, u32, u32, u64, vp, u64, vp, vp, vp])


class hicr_spsc_stream_opts_t(C.Structure):
    _fields_ = [("src", u32), ("flags", u32), ("src_off", u64), ("src_tokens", u64), ("d_capture", vp),
                ("capture_stride", u64)]


HICR_SPSC_DIGEST_ONLY = 1


_spsc_stream_ex = _decl("hicr_spsc_stream_ex", [H, vp, u32, u64, u32, C.POINTER(hicr_spsc_stream_opts_t), u64, vp])


class hicr_pingpong_result_t(C.Structure):
    _fields_ = [("bytes", u64), ("reps", u32), ("ctas_per_side", u32), ("half_rtt_ns", C.c_double),
                ("goodput_gbs", C.c_double), ("digest_a", u64), ("digest_b", u64), ("status", i32),
                ("reserved", u32)]


_pingpong = _decl("hicr_pingpong", [H, u32, u64, u64, u32, u32, u32, u64, C.POINTER(hicr_pingpong_result_t)])
_pingpong_capture = _decl("hicr_pingpong_capture", [H, u32, u64, u64, u32, u32, u32, u64, vp, vp,
                                                    C.POINTER(hicr_pingpong_result_t)])


def hicr_pingpong(inst, src, src_off, nbytes, reps=10, warmup=2, ctas_per_side=1, timeout_ns=30_000_000_000):
    r = hicr_pingpong_result_t()
    st = _pingpong(inst, src, src_off, nbytes, reps, warmup, ctas_per_side, timeout_ns, C.byref(r))
    return st, r


def hicr_pingpong_capture(inst, src, src_off, nbytes, d_out_a, d_out_b, reps=10, warmup=2, ctas_per_side=1,
                          timeout_ns=30_000_000_000):
    r = hicr_pingpong_result_t()
    st = _pingpong_capture(inst, src, src_off, nbytes, reps, warmup, ctas_per_side, timeout_ns, _ptr(d_out_a),
                           _ptr(d_out_b), C.byref(r))
    return st, r


def hicr_spsc_create(inst, token_size, capacity):
    c = u32()
    st = _spsc_create(inst, token_size, capacity, C.byref(c))
    return st, c.value


def hicr_mpsc_create(inst, n_producers, ring_bytes, max_msgs):
    c = u32()
    st = _mpsc_create(inst, n_producers, ring_bytes, max_msgs, C.byref(c))
    return st, c.value


def hicr_mpsc_nl_create(inst, n_producers, ring_bytes, max_msgs):
    c = u32()
    st = _mpsc_nl_create(inst, n_producers, ring_bytes, max_msgs, C.byref(c))
    return st, c.value


class hicr_channel_view_t(C.Structure):
    _fields_ = [("kind", u32), ("token_size", u32), ("capacity", u32), ("max_msgs", u32), ("ring_bytes", u64),
                ("ring", vp), ("head", vp), ("tail", vp), ("freed", vp), ("meta", vp)]


_channel_device_view = _decl("hicr_channel_device_view", [H, u32, C.POINTER(hicr_channel_view_t)])


def hicr_channel_device_view(inst, ch):
    v = hicr_channel_view_t()
    st = _channel_device_view(inst, ch, C.byref(v))
    return st, v


def hicr_channel_destroy(inst, ch):
    return _channel_destroy(inst, ch)


def hicr_channel_ring(inst, ch):
    s = u32()
    st = _channel_ring(inst, ch, C.byref(s))
    return st, s.value


def hicr_channel_push(inst, ch, producer, src, off, n):
    return _channel_push(inst, ch, producer, src, off, n)


def hicr_channel_peek(inst, ch, k):
    m = hicr_msg_info_t()
    st = _channel_peek(inst, ch, k, C.byref(m))
    return st, (m.offset, m.size, m.producer, m.seq)


def hicr_channel_pop(inst, ch, count):
    return _channel_pop(inst, ch, count)


def hicr_channel_depth(inst, ch):
    a, b = u64(), u64()
    st = _channel_depth(inst, ch, C.byref(a), C.byref(b))
    return st, a.value, b.value


def hicr_spsc_stream(inst, chans, tokens, batch, timeout_ns=60_000_000_000):
    arr = (u32 * len(chans))(*chans)
    res = (hicr_spsc_result_t * len(chans))()
    st = _spsc_stream(inst, C.addressof(arr), len(chans), tokens, batch, timeout_ns, C.addressof(res))
    return st, list(res)


def hicr_spsc_stream_ex(inst, chans, tokens, batch, src=0, src_off=0, src_tokens=0, d_capture=None,
                        capture_stride=0, timeout_ns=60_000_000_000, flags=0):
    arr = (u32 * len(chans))(*chans)
    res = (hicr_spsc_result_t * len(chans))()
    o = hicr_spsc_stream_opts_t(src, flags, src_off, src_tokens, _ptr(d_capture), capture_stride)
    st = _spsc_stream_ex(inst, C.addressof(arr), len(chans), tokens, batch, C.byref(o), timeout_ns, C.addressof(res))
    return st, list(res)


def hicr_mpsc_stream(inst, chans, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                     consumer_ctas, d_log, log_stride, timeout_ns=120_000_000_000, d_capture=None, d_cap_off=None):
    """With d_capture / d_cap_off this calls hicr_mpsc_stream_capture."""
    arr = (u32 * len(chans))(*chans)
    res = (hicr_mpsc_result_t * len(chans))()
    args = (inst, C.addressof(arr), len(chans), n_producers, msgs_per_producer, _ptr(d_sizes), _ptr(d_src_off),
            staging, group, consumer_ctas, timeout_ns, _ptr(d_log), log_stride, C.addressof(res))
    if d_capture is None:
        st = _mpsc_stream(*args)
    else:
        st = _mpsc_stream_capture(*args, _ptr(d_capture), _ptr(d_cap_off))
    return st, list(res)


def hicr_mpsc_nl_stream(inst, chans, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                        consumer_ctas, d_log, log_stride, timeout_ns=120_000_000_000, d_capture=None,
                        d_cap_off=None):
    """With d_capture / d_cap_off this calls hicr_mpsc_nl_stream_capture."""
    arr = (u32 * len(chans))(*chans)
    res = (hicr_mpsc_result_t * len(chans))()
    args = (inst, C.addressof(arr), len(chans), n_producers, msgs_per_producer, _ptr(d_sizes), _ptr(d_src_off),
            staging, group, consumer_ctas, timeout_ns, _ptr(d_log), log_stride, C.addressof(res))
    if d_capture is None:
        st = _mpsc_nl_stream(*args)
    else:
        st = _mpsc_nl_stream_capture(*args, _ptr(d_capture), _ptr(d_cap_off))
    return st, list(res)


def hicr_mpsc_stream_capture(inst, chans, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                             consumer_ctas, d_log, log_stride, d_capture, d_cap_off, timeout_ns=120_000_000_000):
    return hicr_mpsc_stream(inst, chans, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                            consumer_ctas, d_log, log_stride, timeout_ns, d_capture=d_capture, d_cap_off=d_cap_off)


def hicr_mpsc_nl_stream_capture(inst, chans, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                                consumer_ctas, d_log, log_stride, d_capture, d_cap_off, timeout_ns=120_000_000_000):
    return hicr_mpsc_nl_stream(inst, chans, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                               consumer_ctas, d_log, log_stride, timeout_ns, d_capture=d_capture,
                               d_cap_off=d_cap_off)


# ---------------------------------------------------------------------------
# Serving (include/hicr_serve.h)
# ---------------------------------------------------------------------------
class hicr_serve_config_t(C.Structure):
    _fields_ = [("budget_bytes", u64), ("n_channels", u32), ("max_msgs", u32), ("ring_bytes", u64),
                ("chunk_bytes", u32), ("op_cost_bytes", u32), ("verify", u32), ("reserved", u32)]


class hicr_serve_stats_t(C.Structure):
    _fields_ = [("completed", u64), ("bytes_moved", u64), ("wall_ns", u64), ("max_inflight", u64),
                ("max_region_bytes", u64), ("admitted", u64), ("dev_units", u64), ("dev_claimed", u64),
                ("dev_requests", u64), ("dev_flags", u64), ("status", i32), ("reserved", u32),
                ("burst_bytes", u64), ("max_poll_gap_ns", u64), ("max_poll_gap_at_ns", u64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


SERVE_REQ_DTYPE = np.dtype([("arrival_ns", "<u8"), ("kind", "<u4"), ("tmpl", "<u4")])
SERVE_RES_DTYPE = np.dtype([("latency_ns", "<u8"), ("admit_ns", "<u8"), ("digest", "<u8"), ("dst_offset", "<u8"),
                            ("device_done_ns", "<u8")])

_serve_create = _decl("hicr_serve_create", [H, C.POINTER(hicr_serve_config_t), C.POINTER(u64)])
_serve_destroy = _decl("hicr_serve_destroy", [H, u64])
_serve_add_memcpy = _decl("hicr_serve_add_memcpy_template", [H, u64, vp, u64, u64, C.POINTER(u32)])
_serve_add_burst = _decl("hicr_serve_add_burst_template", [H, u64, vp, vp, u64, u32, C.POINTER(u32)])
_serve_run = _decl("hicr_serve_run", [H, u64, vp, u64, u32, u64, vp, C.POINTER(hicr_serve_stats_t)])
_serve_run_plain = _decl("hicr_serve_run_plain", [H, u64, vp, u64, u64, u64, vp, C.POINTER(hicr_serve_stats_t)])
_serve_digests = _decl("hicr_serve_digests", [H, u64, vp, u64, vp])
_serve_run_ex = _decl("hicr_serve_run_ex", [H, u64, vp, u64, u32, u64, vp, vp, vp, vp,
                                            C.POINTER(hicr_serve_stats_t)])
_serve_arena = _decl("hicr_serve_arena", [H, u64, C.POINTER(u32)])


def hicr_serve_create(inst, cfg):
    if isinstance(cfg, dict):
        c = hicr_serve_config_t()
        for k, v in cfg.items():
            setattr(c, k, v)
        cfg = c
    s = u64()
    st = _serve_create(inst, C.byref(cfg), C.byref(s))
    return st, s.value


def hicr_serve_destroy(inst, srv):
    return _serve_destroy(inst, srv)


def hicr_serve_add_memcpy_template(inst, srv, ops, region_bytes):
    p, n = _ops_ptr(ops)
    t = u32()
    st = _serve_add_memcpy(inst, srv, p, n, region_bytes, C.byref(t))
    return st, t.value


def hicr_serve_add_burst_template(inst, srv, sizes, staging_off, staging):
    sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
    offs = np.ascontiguousarray(staging_off, dtype=np.uint64)
    t = u32()
    st = _serve_add_burst(inst, srv, sizes.ctypes.data, offs.ctypes.data, len(sizes), staging, C.byref(t))
    return st, t.value


def hicr_serve_run(inst, srv, reqs, mode=0, timeout_ns=300_000_000_000):
    reqs = np.ascontiguousarray(reqs, dtype=SERVE_REQ_DTYPE)
    res = np.zeros(len(reqs), dtype=SERVE_RES_DTYPE)
    stats = hicr_serve_stats_t()
    st = _serve_run(inst, srv, reqs.ctypes.data, len(reqs), mode, timeout_ns, res.ctypes.data, C.byref(stats))
    return st, res, stats


def hicr_serve_run_ex(inst, srv, reqs, mode=0, timeout_ns=300_000_000_000, keep=None, d_capture=None,
                      d_cap_off=None):
    """keep: None or a uint8 array of len(reqs); d_capture / d_cap_off: device
    buffer and device u64 array (addresses or tensors)."""
    reqs = np.ascontiguousarray(reqs, dtype=SERVE_REQ_DTYPE)
    res = np.zeros(len(reqs), dtype=SERVE_RES_DTYPE)
    stats = hicr_serve_stats_t()
    k = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    st = _serve_run_ex(inst, srv, reqs.ctypes.data, len(reqs), mode, timeout_ns,
                       None if k is None else k.ctypes.data, _ptr(d_capture), _ptr(d_cap_off), res.ctypes.data,
                       C.byref(stats))
    return st, res, stats


def hicr_serve_arena(inst, srv):
    s = u32()
    st = _serve_arena(inst, srv, C.byref(s))
    return st, s.value


def hicr_serve_run_plain(inst, srv, reqs, horizon_ns, timeout_ns=300_000_000_000):
    reqs = np.ascontiguousarray(reqs, dtype=SERVE_REQ_DTYPE)
    res = np.zeros(len(reqs), dtype=SERVE_RES_DTYPE)
    stats = hicr_serve_stats_t()
    st = _serve_run_plain(inst, srv, reqs.ctypes.data, len(reqs), horizon_ns, timeout_ns, res.ctypes.data,
                          C.byref(stats))
    return st, res, stats


def hicr_serve_digests(inst, srv, reqs, results):
    reqs = np.ascontiguousarray(reqs, dtype=SERVE_REQ_DTYPE)
    st = _serve_digests(inst, srv, reqs.ctypes.data, len(reqs), results.ctypes.data)
    return st


# ---------------------------------------------------------------------------
# Data Object frontend (include/hicr_dataobject.h)
# ---------------------------------------------------------------------------
class hicr_dobj_handle_t(C.Structure):
    _fields_ = [("id", u64), ("size", u64), ("space", u32), ("instance", u32)]


_dobj_publish = _decl("hicr_dobj_publish", [H, u32, u64, u64, C.POINTER(u64)])
_dobj_get_handle = _decl("hicr_dobj_get_handle", [H, u64, C.POINTER(hicr_dobj_handle_t)])
_dobj_get = _decl("hicr_dobj_get", [H, C.POINTER(hicr_dobj_handle_t), u32, u64])
_dobj_release = _decl("hicr_dobj_release", [H, u64])


def hicr_dobj_publish(inst, slot, off, n):
    i = u64()
    st = _dobj_publish(inst, slot, off, n, C.byref(i))
    return st, i.value


def hicr_dobj_get_handle(inst, obj_id):
    hd = hicr_dobj_handle_t()
    st = _dobj_get_handle(inst, obj_id, C.byref(hd))
    return st, hd


def hicr_dobj_get(inst, handle, dst, dst_off):
    return _dobj_get(inst, C.byref(handle), dst, dst_off)


def hicr_dobj_release(inst, obj_id):
    return _dobj_release(inst, obj_id)
