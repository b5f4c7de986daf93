"""The C-ABI library builds, loads and exports every entry point include/skconv.h
declares (no GPU needed: nothing here computes)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "skconv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sk_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sk_create", "sk_geometry_create", "sk_kernel_create", "sk_kernel_from_legendre",
                 "sk_convolve", "sk_convolve_adjoint", "sk_grad_table", "sk_convolve_jobs",
                 "sk_graph_capture", "sk_count_pairs", "sk_convolve_host"]:
        assert must in names


def test_library_loads_and_exports_every_symbol():
    import paper_1211_3556_b300 as sk
    L = sk.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", sk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sk_[a-z_0-9]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(L, name) is not None


def test_binding_declares_every_symbol():
    import paper_1211_3556_b300 as sk
    L = sk.lib()
    for name in declared_functions():
        assert getattr(L, name).argtypes is not None or name == "sk_last_error", name


def test_pure_host_entry_points():
    import paper_1211_3556_b300 as sk
    L = sk.lib()
    assert L.sk_npix(1) == 12 and L.sk_npix(2048) == 50331648 and L.sk_npix(8192) == 805306368
    assert L.sk_npix(3) == -1 and L.sk_npix(0) == -1 and L.sk_npix(16384) == -1
    # creating a context on a device that does not exist fails with an error code, no crash
    h = ctypes.c_void_p()
    assert L.sk_create(ctypes.byref(h), 999) != 0
    assert len(L.sk_last_error()) > 0
    assert L.sk_create(None, 0) == sk.SK_EINVAL


def test_null_handles_are_rejected():
    import paper_1211_3556_b300 as sk
    L = sk.lib()
    assert L.sk_convolve(None, None, None, None, 1, 12, None) == sk.SK_EINVAL
    assert L.sk_grad_table(None, None, None, None, 1, 12, None, None) == sk.SK_EINVAL
    assert L.sk_destroy(None) == 0 and L.sk_kernel_destroy(None) == 0
    assert L.sk_graph_launch(None, None) == sk.SK_EINVAL
    assert L.sk_set_workspace_limit(None, 0) == sk.SK_EINVAL
