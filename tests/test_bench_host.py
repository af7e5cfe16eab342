"""Host-side accounting of the serving bench (no GPU): where a run's longest
pause was, on the host loop's clock and on the device's completion clock,
and what a second host thread saw meanwhile."""
import time
import types

import numpy as np

import bench


def _results(done_ns):
    from paper_2509_01425_gb300 import build
    build.build()  # the binding (which holds the result layout) loads the library
    from paper_2509_01425_gb300 import hicr
    r = np.zeros(len(done_ns), dtype=hicr.SERVE_RES_DTYPE)
    r["device_done_ns"] = done_ns
    return r


def test_stall_summary_finds_the_longest_device_gap():
    # completions every 50 us on the device clock, then one 30 ms gap; the
    # results arrive out of completion order, and plain-form entries (0) are
    # ignored
    t = np.arange(1000, dtype=np.uint64) * 50_000 + 7_000_000_000
    t[600:] += 30_000_000
    done = np.concatenate([t[::-1], np.zeros(5, dtype=np.uint64)])
    stats = types.SimpleNamespace(max_poll_gap_ns=31_000_000, max_poll_gap_at_ns=12_500_000_000)
    s = bench.stall_summary(_results(done), stats)
    assert s["host_max_poll_gap_ms"] == 31.0
    assert s["host_max_poll_gap_at_s"] == 12.5
    assert abs(s["device_max_completion_gap_ms"] - 30.05) < 1e-9
    # the gap ends at completion 600, 600 x 50 us + 30 ms after the first
    assert abs(s["device_max_completion_gap_at_s"] - (600 * 50e-6 + 0.030)) < 1e-9


def test_stall_summary_without_device_times():
    stats = types.SimpleNamespace(max_poll_gap_ns=0, max_poll_gap_at_ns=0)
    s = bench.stall_summary(_results(np.zeros(3, dtype=np.uint64)), stats)
    assert s["device_max_completion_gap_ms"] is None and s["device_max_completion_gap_at_s"] is None


def test_host_pause_watch_records_a_late_wake_up():
    # Starve the watcher thread: with a long interpreter switch interval, a
    # pure-Python busy loop keeps the interpreter lock for its whole 80 ms, so
    # the watcher's 1 ms sleep ends about 80 ms late.
    import sys
    w = bench.HostPauseWatch(over_ms=10.0)
    time.sleep(0.02)
    old = sys.getswitchinterval()
    sys.setswitchinterval(1.0)
    try:
        t0 = time.monotonic()
        while time.monotonic() - t0 < 0.08:
            pass
    finally:
        sys.setswitchinterval(old)
    time.sleep(0.02)
    out = w.summary()
    assert out["second_thread_pause_threshold_ms"] == 10.0
    assert any(ms >= 40 for _, ms in out["second_thread_pauses_s_ms"]), out
    assert out["guest_steal_ms"] is None or out["guest_steal_ms"] >= 0
