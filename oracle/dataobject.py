"""Oracle for the Data Object frontend -- TEST INFRASTRUCTURE ONLY.

HiCR paper Sec. 4.3 (Data Object): publish makes a block of a local memory
slot accessible and returns a unique identifier; getHandle turns the
identifier into a handle; get starts a transfer of the object into a
destination, completed at the next fence. With one instance, get is the
communication manager's memcpy (oracle.memcpy) from the object's range.

Readings: identifiers are 1, 2, ... in publication order and are not reused;
a released or unknown identifier is INVALID; get validates exactly like
memcpy (bounds, space pair, same-slot overlap).
"""
from __future__ import annotations

from .memcpy import CommManager, OK, ERR_INVALID, ERR_BOUNDS, _range_ok


class DataObjects:
    def __init__(self, cm: CommManager):
        self.cm = cm
        self.next = 1
        self.objs: dict[int, tuple[int, int, int]] = {}

    def publish(self, slot: int, off: int, n: int):
        s = self.cm.slots.get(slot)
        if s is None or not s.live:
            return ERR_INVALID, None
        if not _range_ok(off, n, len(s.data)):
            return ERR_BOUNDS, None
        k = self.next
        self.next += 1
        self.objs[k] = (slot, off, n)
        return OK, k

    def get_handle(self, k: int):
        if k not in self.objs:
            return ERR_INVALID, None
        slot, off, n = self.objs[k]
        return OK, (k, n, self.cm.slots[slot].space)

    def get(self, k: int, dst: int, dst_off: int) -> int:
        if k not in self.objs:
            return ERR_INVALID
        slot, off, n = self.objs[k]
        return self.cm.memcpy(dst, dst_off, slot, off, n)

    def release(self, k: int) -> int:
        return OK if self.objs.pop(k, None) is not None else ERR_INVALID
