"""CPU oracle for the HiCR communication path -- TEST INFRASTRUCTURE ONLY.

This package is the parity authority for the CUDA path: a plain, slow,
single-threaded restatement of what the HiCR model says the communication
manager and the channels frontend compute. It shares no code with the CUDA
library and never imports it; both sides only share the seeded input
generators in ``workloads``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py`` may import anything from here. The product
path (the C-ABI library and its Python binding) must never call into it.

Modules
  memcpy    -- memory slots, memcpy(dst, dOff, src, sOff, n), fence and the
               sent/received message counters (HiCR paper Sec. 3.1.3-3.1.4, Fig. 5).
  channels  -- SPSC and MPSC (locking and non-locking mode) circular-buffer
               channels and the interleaving-agnostic log checkers
               (HiCR paper Sec. 4.3, Channels frontend).
  dataobject -- the Data Object frontend: publish / getHandle / get
               (HiCR paper Sec. 4.3).
  digest    -- the position-weighted word digest the checkers compare.
  native    -- builds memcpy_threads.c, the all-cores CPU memcpy baseline.
"""
