"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+char\s*\*|hicr_status)\s+(hicr_\w+)\s*\(", re.M)


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(DECL.findall(open(h).read()))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_01425_gb300 import build
    return build.build()


def test_headers_declare_the_boundary():
    names = declared()
    for must in ["hicr_init", "hicr_topology_query", "hicr_mem_alloc", "hicr_mem_free", "hicr_slot_register",
                 "hicr_slot_deregister", "hicr_memcpy", "hicr_fence", "hicr_exec_launch", "hicr_exec_await"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_status_strings(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared():
        getattr(lib, n)
    from paper_2509_01425_gb300 import hicr
    assert hicr.hicr_status_str(hicr.HICR_ERR_BOUNDS) == "HICR_ERR_BOUNDS"
    assert hicr.hicr_status_str(0) == "HICR_OK"
    assert ctypes.sizeof(hicr.hicr_op_t) == 32


def test_status_codes_match_the_oracle(libpath):
    from oracle import memcpy as om
    from paper_2509_01425_gb300 import hicr
    for name in ["OK", "ERR_INVALID", "ERR_UNSUPPORTED", "ERR_BOUNDS", "ERR_OVERLAP", "ERR_HAZARD", "ERR_NOMEM",
                 "ERR_FULL", "ERR_EMPTY", "ERR_TOO_LARGE", "ERR_TIMEOUT", "ERR_BUSY", "ERR_DEVICE"]:
        assert getattr(hicr, "HICR_" + name) == getattr(om, name)


def test_without_gpu_init_is_rejected_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_01425_gb300 import hicr
    st, _ = hicr.hicr_init(0)
    assert st == hicr.HICR_ERR_INVALID
