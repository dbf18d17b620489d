"""The C ABI library builds for sm_103a and exports every entry point include/rcm.h declares.

No compute calls here (no GPU on this host); only pure host functions are called.
"""
import ctypes
import os
import re

import pytest

from paper_1610_08128_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rcm_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = build_mod.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("rcm_order", "rcm_order_batch", "rcm_stream_status", "rcm_bandwidth_profile"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_functions(lib):
    from paper_1610_08128_gb300 import rcm

    assert rcm.status_string(0) == "RCM_OK"
    assert rcm.status_string(6) == "RCM_ERR_TIMEOUT"
    ws = rcm.rcm_workspace_bytes(4096, 16128)
    assert ws >= 4 * (8 * 4096 + 16128)
    assert rcm.rcm_workspace_bytes(-1, 0) == 0
    # a server request holds the workspace plus what it stages
    both = rcm.rcm_request_bytes(4096, 16128, True, True)
    assert both > rcm.rcm_request_bytes(4096, 16128, False, False) + 4 * (2 * 4096 + 16128)
    # staging the output adds its 4n bytes (4 * 4096 is already a multiple of the 256-byte alignment)
    assert rcm.rcm_request_bytes(4096, 16128, False, True) == rcm.rcm_request_bytes(4096, 16128, False, False) + 4 * 4096
    assert rcm.rcm_request_bytes(-1, 0) == 0
    # sizes at the int32 limits: plain arithmetic, no overflow, monotone in n and nnz
    big = rcm.rcm_workspace_bytes(2**31 - 1, 2**31 - 2)
    assert big > 80 * (2**31 - 1) + 4 * (2**31 - 2) and big < 2**45
    assert rcm.rcm_workspace_bytes(2**31 - 1, 0) < big
    rb = rcm.rcm_request_bytes(2**31 - 1, 2**31 - 2, True, True)
    assert rb > big and rb < 2**46


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    from paper_1610_08128_gb300 import rcm

    monkeypatch.setattr(rcm, "_lib", None)
    monkeypatch.setattr(rcm, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        rcm.load()


def test_kernels_are_sm103a(lib):
    """The build targets exactly one architecture: compute_103a -> sm_103a."""
    assert build_mod.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_structures_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of its C declaration
    in include/rcm.h (compiled here with the host C compiler)."""
    import ctypes
    import shutil
    import subprocess

    from paper_1610_08128_gb300 import rcm

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    structs = [rcm.rcm_options, rcm.rcm_batch_options, rcm.rcm_server_options, rcm.rcm_stats, rcm.rcm_server_stats,
               rcm.rcm_validate_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rcm.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def test_option_checks_come_before_any_device_work(lib):
    """Invalid options and sizes are refused with RCM_ERR_INVALID_ARG before the call touches a
    device (so this runs on a host without one); n = 0 with valid options is a no-op."""
    from paper_1610_08128_gb300 import rcm

    bad = [("expand_mode", 4), ("expand_mode", -1), ("row_order", 2), ("async_sweeps", 2), ("async_sweeps", -2),
           ("bottom_up_divisor", -1), ("debug_async_slots", -1), ("executor", 3), ("cluster", 2),
           ("block_threads", 100), ("narrow_threshold", -2), ("grid_blocks", -1), ("spin_limit_ns", -1),
           ("fused_sweeps", 3), ("fused_sweeps", -2), ("l2_persist", 2), ("debug_order_bits", 64),
           ("debug_order_bits", -1), ("mid_cluster", 3), ("mid_cluster", 32), ("mid_threshold", -1),
           ("components_first", 2), ("components_first", -2)]
    for field, value in bad:
        o = rcm.rcm_options()
        setattr(o, field, value)
        assert rcm.rcm_order_ex(0, None, None, None, o, None) == rcm.RCM_ERR_INVALID_ARG, field
    assert rcm.rcm_order_ex(-1, None, None, None, None, None) == rcm.RCM_ERR_INVALID_ARG
    assert rcm.rcm_order_ex(0, None, None, None, rcm.rcm_options(), None) == rcm.RCM_OK
    rep = rcm.rcm_validate_report()
    assert rcm.rcm_validate(-1, None, None, rep) == rcm.RCM_ERR_INVALID_ARG
    assert rcm.rcm_validate(0, None, None, rep) == rcm.RCM_OK
    assert rep.first_bad_row == -1 and rep.duplicates == 0 and rep.asymmetric == 0
