"""Helpers shared by the GPU tests: an instance fixture, device views of
slots, and oracle-side expectations (slot fill bytes)."""
import numpy as np
import pytest
import torch

from workloads import splitmix


class _CAI:
    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_bytes(ptr: int, nbytes: int) -> torch.Tensor:
    """A uint8 torch view of device memory [ptr, ptr+nbytes) (no copy)."""
    if nbytes == 0:
        return torch.zeros(0, dtype=torch.uint8, device="cuda")
    return torch.as_tensor(_CAI(ptr, nbytes), device="cuda")


def slot_bytes(h, inst, slot) -> np.ndarray:
    st, ptr, size, space, tag = h.hicr_slot_info(inst, slot)
    assert st == 0
    torch.cuda.synchronize()
    return device_bytes(ptr, size).cpu().numpy()


def fill_key(seed: int, slot_index: int) -> int:
    return splitmix.fill_key_base(seed, slot_index)


@pytest.fixture(scope="module")
def h():
    from paper_2509_01425_gb300 import build
    build.build()
    from paper_2509_01425_gb300 import hicr
    return hicr


@pytest.fixture()
def inst(h):
    st, i = h.hicr_init(0)
    assert st == 0, h.hicr_status_str(st)
    yield i
    st = h.hicr_finalize(i)
    assert st == 0, h.hicr_status_str(st)
