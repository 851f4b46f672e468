"""The C ABI from a plain C99 program: the header compiles as C, option defaults and
host-only calls (grid creation, level sizes, footprint, option validation) behave as
declared.  No device is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    import paper_1607_00648_gb300 as mg
    from paper_1607_00648_gb300 import build

    if not os.path.exists(mg._lib.LIB_PATH):
        build.build()
    libdir = os.path.dirname(mg._lib.LIB_PATH)
    exe = tmp_path / "abi_smoke"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_smoke.c"), "-L", libdir, "-lmg", f"-Wl,-rpath,{libdir}",
           "-o", str(exe)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0 and "cannot find -lmg" in res.stderr:
        # the library's file name is libmg.so; link it by path
        cmd = [c for c in cmd if c != "-lmg"] + [mg._lib.LIB_PATH]
        res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.split("\n")
    assert lines[0].split() == ["1", "1", "0", "2", "2", "0.600", "1", "1", "0", "0.0001", "0", "1", "0"]
    n_dofs, n_slots, B = (int(v) for v in lines[1].split())
    assert n_dofs == 26 * 26 and B == 27 and n_slots == 736
    assert lines[2] == "1 null"  # MG_ERR_INVALID_ARG, no handle
