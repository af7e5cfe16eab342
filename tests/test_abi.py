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


def test_binding_has_every_declared_call(libpath):
    """The Python binding carries every call the headers declare, under the
    same name."""
    from paper_2509_01425_gb300 import hicr
    missing = [n for n in declared() if not callable(getattr(hicr, n, None))]
    assert not missing, missing


def _c_layout(tmp_path, types_fields):
    """sizeof and offsetof as the C compiler lays out the headers' structs:
    a small program built against include/*.h prints them."""
    lines = ["#include <stdio.h>", "#include <stddef.h>"]
    for h in ["hicr.h", "hicr_channels.h", "hicr_dataobject.h", "hicr_serve.h", "hicr_util.h"]:
        lines.append(f'#include "{h}"')
    lines.append("int main(void) {")
    for t, fields in types_fields.items():
        lines.append(f'  printf("{t} %zu\\n", sizeof({t}));')
        for f in fields:
            lines.append(f'  printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=gnu11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (l.split() for l in out.splitlines())}


def test_binding_struct_layouts_match_the_headers(libpath, tmp_path):
    """Every ctypes structure and numpy record type of the binding has the size
    and field offsets that the C compiler gives the header's struct of the
    same name: a field added on one side only would corrupt what the library
    reads or writes."""
    import numpy as np
    from paper_2509_01425_gb300 import hicr
    ctypes_structs = {n: c for n, c in vars(hicr).items()
                      if isinstance(c, type) and issubclass(c, ctypes.Structure) and n.startswith("hicr_")}
    dtypes = {"hicr_serve_request_t": hicr.SERVE_REQ_DTYPE, "hicr_serve_result_t": hicr.SERVE_RES_DTYPE,
              "hicr_mpsc_log_t": hicr.MPSC_LOG_DTYPE}
    want = {n: [f[0] for f in c._fields_] for n, c in ctypes_structs.items()}
    want.update({n: list(d.names) for n, d in dtypes.items()})
    assert len(ctypes_structs) >= 15, sorted(ctypes_structs)
    c = _c_layout(tmp_path, want)
    bad = []
    for n, cls in ctypes_structs.items():
        if ctypes.sizeof(cls) != c[n]:
            bad.append((n, "size", ctypes.sizeof(cls), c[n]))
        for f in want[n]:
            if getattr(cls, f).offset != c[f"{n}.{f}"]:
                bad.append((n, f, getattr(cls, f).offset, c[f"{n}.{f}"]))
    for n, d in dtypes.items():
        if d.itemsize != c[n]:
            bad.append((n, "size", d.itemsize, c[n]))
        for f in d.names:
            if d.fields[f][1] != c[f"{n}.{f}"]:
                bad.append((n, f, d.fields[f][1], c[f"{n}.{f}"]))
    assert not bad, bad
