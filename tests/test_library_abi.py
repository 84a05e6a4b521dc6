"""The C-ABI library loads without a GPU and exports every entry point that
include/wl.h declares; host-side argument checks work without a device."""
import os
import re
import subprocess

import pytest

import paper_1302_2320_gb300 as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:wl_status|size_t|const char\*)\s+(wl_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    wl.build()
    return wl.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["wl_create", "wl_set_option", "wl_run", "wl_get_lng", "wl_get_stats", "wl_destroy",
              "wl_last_error", "wl_assemble"]:
        assert n in names
    assert set(names) == set(wl.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", wl.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(wl_\w+)$", out, flags=re.M))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_host_side_validation_without_gpu(lib):
    h = wl.Handle("square", 64)
    assert h.N == 4096 and h.NB == 8192 and h.lines == 2049
    assert h.get_option("bins") == 2049 ** 2          # sum over l <= N/2 of (2l + 1)
    with pytest.raises(wl.WLError):
        h.set_option("mapping", 3)
    with pytest.raises(wl.WLError):
        h.set_option("no_such_option", 1)
    with pytest.raises(wl.WLError):
        wl.Handle("square", 2)                         # L < 3 has double bonds
    h.close()
    t = wl.Handle("triangular", 6)
    assert t.N == 36 and t.NB == 108
    c = wl.Handle("cubic", 4)
    assert c.N == 64 and c.NB == 192
    assert wl.wl_required_bytes(0, 64) > 4 * 2049 ** 2 * 8 // 4
