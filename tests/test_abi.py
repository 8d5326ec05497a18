"""CPU-side checks of the C ABI: the library loads, exports every entry
point the header declares, and the ctypes mirror matches the header's
struct layouts (measured by compiling the header with gcc). No GPU needed."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bn():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_02926_gb300 as m
    return m


def test_library_exports_every_header_entry_point(bn):
    from paper_2310_02926_gb300 import _abi
    names = _abi.header_entry_points(_abi.INCLUDE)
    assert len(names) >= 19
    L = bn.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_abi.PROTOTYPES)
    out = subprocess.run(["nm", "-D", "--defined-only", bn.LIB_PATH], capture_output=True, text=True)
    exported = {line.split()[-1] for line in out.stdout.splitlines() if " T " in line}
    assert exported == set(names)


def test_struct_layouts_match_header(bn, tmp_path):
    from paper_2310_02926_gb300 import _abi
    src = tmp_path / "sz.c"
    structs = ["bn_buffer", "bn_grid", "bn_result", "bn_block", "bn_grid_spec", "bn_options",
               "bn_server_options", "bn_server_stats", "bn_request_timing"]
    body = "\n".join(f'printf("%zu\\n", sizeof({s}));' for s in structs)
    offs = [("bn_buffer", "stream"), ("bn_buffer", "deleter"), ("bn_block", "grid"),
            ("bn_grid_spec", "grid"),
            ("bn_block", "out"), ("bn_result", "bounds"), ("bn_grid", "res")]
    body += "\n" + "\n".join(f'printf("%zu\\n", offsetof({s}, {f}));' for s, f in offs)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "binning.h"\n'
                   f"int main(void) {{ {body} return 0; }}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    want = [ctypes.sizeof(getattr(_abi, s)) for s in structs]
    want += [getattr(getattr(_abi, s), f).offset for s, f in offs]
    assert vals == want


def test_header_compiles_as_c_and_cxx(tmp_path):
    for comp, ext in (("gcc", "c"), ("g++", "cpp")):
        f = tmp_path / f"h.{ext}"
        f.write_text('#include "binning.h"\nint main(void){ return BN_OK; }\n')
        subprocess.run([comp, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(f),
                        "-o", str(tmp_path / f"h_{ext}")], check=True)


def test_constants_match_header(bn):
    import re
    from paper_2310_02926_gb300 import _abi
    hdr = open(_abi.HEADER).read()
    for name in ("BN_OP_COUNT", "BN_OP_AVG", "BN_OP_ACCUMULATE", "BN_SUM_F32", "BN_SUM_F64",
                 "BN_STRATEGY_PRIVATE", "BN_STRATEGY_GLOBAL", "BN_STRATEGY_SORT",
                 "BN_STRATEGY_HYBRID"):
        m = re.search(name + r"\s*=\s*(\d+)u?\s*<<\s*(\d+)", hdr)
        assert m, name
        assert getattr(_abi, name[3:]) == int(m.group(1)) << int(m.group(2)), name
    for name, val in (("BN_MAX_MULTI_COLS", _abi.MAX_MULTI_COLS), ("BN_MAX_MULTI_SPECS", _abi.MAX_MULTI_SPECS),
                      ("BN_MAX_ATTR", _abi.MAX_ATTR)):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", hdr)
        assert m and int(m.group(1)) == val, name
    for name, val in (("BN_ERR_DEGENERATE", _abi.ERR_DEGENERATE), ("BN_ERR_BUDGET", _abi.ERR_BUDGET),
                      ("BN_ERR_TIMEOUT", _abi.ERR_TIMEOUT), ("BN_NOT_READY", _abi.NOT_READY)):
        m = re.search(name + r"\s*=\s*(-?\d+)", hdr)
        assert int(m.group(1)) == val, name


def test_context_create_without_gpu_fails_cleanly(bn):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = bn.lib().bn_context_create(0, None, ctypes.byref(h))
    assert st < 0 and not h.value
    assert bn.lib().bn_last_error()


def test_package_fails_loudly_without_the_library(tmp_path):
    # a copy of the package with no built library must raise, not fall back
    code = ("import sys, types, importlib.util, os\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "import paper_2310_02926_gb300 as m\n"
            f"m.LIB_PATH = {str(tmp_path / 'missing.so')!r}\n"
            "m._lib = None\n"
            "try:\n    m.lib()\nexcept RuntimeError as e:\n    print('raised', 'no CPU fallback' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert "raised True" in out.stdout, out.stderr
