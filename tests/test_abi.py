"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/flashsplat.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flashsplat.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2409_08270_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:
        if "nvcc not found" in str(e):
            pytest.skip("no CUDA toolkit")
        raise


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("fs_create", "fs_destroy", "fs_scene_create", "fs_scene_destroy", "fs_accumulate",
              "fs_assign", "fs_solve", "fs_synchronize", "fs_last_error", "fs_version"):
        assert f in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(fs_\w+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    from paper_2409_08270_gb300 import flashsplat
    assert sorted(flashsplat.EXPORTS) == declared_functions()


def test_library_loads_and_reports_version(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.fs_version.restype = ctypes.c_int32
    assert lib.fs_version() == 1
    lib.fs_last_error.restype = ctypes.c_char_p
    assert lib.fs_last_error() == b""


def test_argument_errors_without_gpu(lib_path):
    """Argument validation happens before any device work."""
    from paper_2409_08270_gb300 import flashsplat as fsb
    lib = fsb.load(lib_path)
    assert lib.fs_create(None, 0, None) == fsb.FS_INVALID_ARGUMENT
    assert b"NULL" in lib.fs_last_error()
    assert lib.fs_destroy(None) == fsb.FS_OK
    assert lib.fs_scene_destroy(None) == fsb.FS_OK
    assert lib.fs_scene_size(None) == 0
    assert lib.fs_assign(None, None, 0, 0, 2, 0.5, None, None, None, None) == fsb.FS_INVALID_ARGUMENT


def test_product_path_has_no_oracle_dependency():
    """The package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2409_08270_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "fs_oracle" not in text and "fso_" not in text, f


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes across the ABI has the header's size
    and field offsets (a C program compiled against include/flashsplat.h
    prints them; gcc only, no GPU)."""
    import shutil
    from paper_2409_08270_gb300 import flashsplat as fsb
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = [fsb.fs_options, fsb.fs_gaussians, fsb.fs_camera, fsb.fs_stats, fsb.fs_result,
               fsb.fs_server_options, fsb.fs_server_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "flashsplat.h"',
             "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, *_ in st._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    want = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for st in structs:
        name = st.__name__
        assert int(want[name]) == ctypes.sizeof(st), name
        for field, *_ in st._fields_:
            assert int(want[f"{name}.{field}"]) == getattr(st, field).offset, (name, field)
