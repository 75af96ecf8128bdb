"""The C-ABI library builds, loads and exports every entry point of include/hqmc.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hqmc.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"HQMC_API\s+[\w\s\*]+?\b(hqmc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2508_16298_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hqmc_make_config", "hqmc_apply_M", "hqmc_apply_MdagM", "hqmc_cg_solve", "hqmc_force",
                     "hqmc_leapfrog", "hqmc_trajectory"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header(lib_path):
    from paper_2508_16298_gb300 import hqmc
    assert sorted(hqmc.EXPORTS) == declared_functions()


def test_strerror_is_host_only(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.hqmc_strerror.restype = ctypes.c_char_p
    assert lib.hqmc_strerror(0) == b"success"
    assert b"converge" in lib.hqmc_strerror(2)
    lib.hqmc_free_config.argtypes = [ctypes.c_void_p]
    assert lib.hqmc_free_config(None) == 0


def test_params_struct_layout_matches_header(lib_path):
    from paper_2508_16298_gb300 import hqmc
    # int L, int Ntau, 4 doubles, int action, int reliable_interval, int autotune, int variant
    assert ctypes.sizeof(hqmc.Params) == 4 + 4 + 4 * 8 + 4 * 4
    assert ctypes.sizeof(hqmc.SolveInfo) == 4 * 4 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(hqmc.TrajInfo) == 4 * 4 + 5 * 8
