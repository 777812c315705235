"""CPU checks of the C ABI: the library builds, loads and exports every
symbol include/gbfd.h declares; host-side validation rejects bad
parameters without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1707_08900_gb300 import build as gb
from paper_1707_08900_gb300 import gbfd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return gbfd.load()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gbfd\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert "gbfd_rk3_step" in declared and "gbfd_init" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(gbfd.EXPORTS) <= declared


def test_workspace_bytes_rejects_bad_params(lib):
    assert gbfd.gbfd_workspace_bytes(gbfd.make_params((32, 32, 32))) > 0
    for shape in [(32, 32, 30), (4, 32, 32), (32, 7, 32)]:  # nx % 4, extents >= 8
        assert gbfd.gbfd_workspace_bytes(gbfd.make_params(shape)) == 0
    p = gbfd.make_params((16, 16, 16))
    p.nu = -1.0
    assert gbfd.gbfd_workspace_bytes(p) == 0
    p = gbfd.make_params((16, 16, 16))
    p.lx = float("nan")
    assert gbfd.gbfd_workspace_bytes(p) == 0
    p = gbfd.make_params((16, 16, 16))
    p.precision = 9
    assert gbfd.gbfd_workspace_bytes(p) == 0


def test_workspace_size_accounts_for_layout(lib):
    p64 = gbfd.make_params((64, 64, 64), precision="fp64")
    p32 = gbfd.make_params((64, 64, 64), precision="fp32")
    n = 64 ** 3
    # three padded state-sized buffers + staging, at least
    assert gbfd.gbfd_workspace_bytes(p64) >= 3 * 5 * n * 8 + 5 * n * 8
    assert gbfd.gbfd_workspace_bytes(p32) >= 3 * 5 * n * 4
    p19 = gbfd.make_params((64, 64, 64), precision="fp32", form="19p")
    assert gbfd.gbfd_workspace_bytes(p19) > gbfd.gbfd_workspace_bytes(p32)
    # walls in z: 3 ghost planes below and above, on both state buffers
    pw = gbfd.make_params((64, 64, 64), precision="fp32", bc_z="wall")
    plane = (64 + 8 + 24) * (64 + 6)  # padded row pitch (a multiple of 32 values) x rows
    assert gbfd.gbfd_workspace_bytes(pw) >= gbfd.gbfd_workspace_bytes(p32) + 2 * 5 * 6 * plane * 4
    bad = gbfd.make_params((64, 64, 64), precision="fp32")
    bad.bc_z = 3
    assert gbfd.gbfd_workspace_bytes(bad) == 0
    # exchanged halos (z-slabs of a decomposed box): 55-point form only
    assert gbfd.gbfd_workspace_bytes(gbfd.make_params((64, 64, 64), bc_z="exchange")) > 0
    assert gbfd.gbfd_workspace_bytes(gbfd.make_params((64, 64, 64), form="19p",
                                                      bc_z="exchange")) == 0
    assert gbfd.gbfd_workspace_bytes(gbfd.make_params((64, 64, 64), form="19p",
                                                      precision="fp32_accff")) == 0


def test_init_rejects_null_and_misaligned_workspace(lib):
    p = gbfd.make_params((16, 16, 16))
    ctx = ctypes.c_void_p()
    n = gbfd.gbfd_workspace_bytes(p)
    st = lib.gbfd_init(ctypes.byref(p), None, n, None, ctypes.byref(ctx))
    assert st == 2 and not ctx.value  # GBFD_ERR_WORKSPACE
    st = lib.gbfd_init(ctypes.byref(p), ctypes.c_void_p(0x1010), n, None, ctypes.byref(ctx))
    assert st == 2
    assert "aligned" in gbfd.gbfd_last_error(None)
    st = lib.gbfd_init(ctypes.byref(p), ctypes.c_void_p(0x100000), 16, None, ctypes.byref(ctx))
    assert st == 2 and "needed" in gbfd.gbfd_last_error(None)
    bad = gbfd.make_params((16, 16, 18))
    st = lib.gbfd_init(ctypes.byref(bad), ctypes.c_void_p(0x100000), n, None, ctypes.byref(ctx))
    assert st == 1


def test_status_strings(lib):
    for code, name in gbfd.STATUS.items():
        assert lib.gbfd_status_string(code).decode() == name


def test_calls_reject_null_context(lib):
    assert lib.gbfd_rk3_step(None, 0.1, 1) == 1
    assert lib.gbfd_sync(None) == 1
    assert lib.gbfd_destroy(None) == 0
