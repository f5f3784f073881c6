"""The C ABI without a GPU: the library builds, loads and exports every
function include/hfcr.h declares, and the ctypes structures of the Python
binding have the C layout (sizes and offsets printed by a C program
compiled against the header)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hfcr.h")


@pytest.fixture(scope="module")
def built():
    from paper_1409_2081_gb300 import build
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hfcr_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_function(built):
    lib = ctypes.CDLL(built)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_1409_2081_gb300 import api
    assert sorted(api.EXPORTS) == names


def test_status_strings_without_gpu(built):
    from paper_1409_2081_gb300 import api
    assert api.status_string(0) == "HFCR_OK"
    assert api.status_string(8) == "HFCR_ERR_RANGE"
    lib = api.lib()
    # a NULL context pointer is an argument error, not a crash
    assert lib.hfcr_create(None, None) == api.HFCR_ERR_ARG
    assert lib.hfcr_destroy(None) == api.HFCR_OK
    assert lib.hfcr_last_error(None) == b""


def test_struct_layout_matches_header(tmp_path):
    from paper_1409_2081_gb300 import api
    probe = tmp_path / "probe.c"
    structs = {"hfcr_mesh": api.hfcr_mesh, "hfcr_pair": api.hfcr_pair,
               "hfcr_stencil": api.hfcr_stencil, "hfcr_options": api.hfcr_options,
               "hfcr_solve_info": api.hfcr_solve_info, "hfcr_detect_stats": api.hfcr_detect_stats,
               "hfcr_resolve_info": api.hfcr_resolve_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", str(probe), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
