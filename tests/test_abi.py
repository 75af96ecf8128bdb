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


def test_host_only_setters_reject_null_handles(lib_path):
    """Setters and getters that touch no device state answer HQMC_EINVAL (1) for a
    NULL handle, on a machine without a GPU."""
    lib = ctypes.CDLL(lib_path)
    vp, i = ctypes.c_void_p, ctypes.c_int
    for name, args in [("hqmc_set_net_tensor_cores", [vp, i]), ("hqmc_set_net_interval", [vp, i]),
                       ("hqmc_set_guess_history", [vp, i]), ("hqmc_batch_set_solver", [vp, i]),
                       ("hqmc_set_multi_rhs", [vp, i]), ("hqmc_set_multi_ranges", [vp, i])]:
        f = getattr(lib, name)
        f.argtypes, f.restype = args, i
        assert f(None, 1) == 1, name
    f = lib.hqmc_batch_launch_shape
    f.argtypes, f.restype = [vp, vp, vp, vp, vp], i
    assert f(None, None, None, None, None) == 1
    f = lib.hqmc_multi_launch_shape
    f.argtypes, f.restype = [vp, i, vp, vp, vp], i
    assert f(None, 4, None, None, None) == 1


def test_params_struct_layout_matches_header(lib_path, tmp_path):
    """The binding's ctypes structs have the sizes and field offsets the C compiler
    gives the header's structs."""
    import shutil
    import subprocess
    from paper_2508_16298_gb300 import hqmc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"hqmc_params": hqmc.Params, "hqmc_solve_info": hqmc.SolveInfo, "hqmc_traj_info": hqmc.TrajInfo,
               "hqmc_checkpoint": hqmc.Checkpoint}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hqmc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)
