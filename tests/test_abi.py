"""CPU checks of the C-ABI library: it builds, loads, exports every entry point that
include/*.h declares, and rejects invalid arguments before touching the GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_10058_gb300 import build, curldiv
    if not os.path.exists(curldiv.LIB_PATH):
        build.build()
    return curldiv.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"CD_API\s+[\w\s\*]+?\b(cd_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_host_side_argument_checks(lib):
    from paper_1805_10058_gb300 import curldiv as c
    assert c.cd_dofs(2, 2, 16) == 2 * 16 ** 2
    assert c.cd_dofs(3, 3, 64) == 3 * 65 ** 3
    assert c.cd_dofs(4, 2, 16) == 0 and c.cd_dofs(2, 0, 16) == 0
    h = ctypes.c_void_p()
    for args in [(4, 2, 16, 1.0, 1.0), (2, 0, 16, 1.0, 1.0), (2, 2, 0, 1.0, 1.0), (2, 1, 2, 1.0, 1.0),
                 (2, 2, 16, -1.0, 1.0), (2, 2, 16, 1.0, 0.0), (2, 2, 16, float("nan"), 1.0),
                 (2, 2, 16, 1.0, float("inf"))]:
        assert lib.cd_create(ctypes.byref(h), *args, None, None) == c.CD_EINVAL, args
    assert lib.cd_create(None, 2, 2, 16, 1.0, 1.0, None, None) == c.CD_EINVAL
    assert lib.cd_destroy(None) == c.CD_EINVAL
    o = c.default_options()
    assert o.rtol == 1e-10 and o.precision == c.CD_PREC_FP32_IR and o.max_batch >= 1
    bad = c.default_options(max_batch=0)
    assert lib.cd_create(ctypes.byref(h), 2, 2, 16, 1.0, 1.0, ctypes.byref(bad), None) == c.CD_EINVAL
    assert lib.cd_strerror(c.CD_NOT_CONVERGED) == b"not converged"


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of cd_options, cd_result and the server structs have the header's
    sizes and field offsets (compiled with the host C compiler, no GPU)."""
    import shutil
    import subprocess
    from paper_1805_10058_gb300 import curldiv as c
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"cd_options": c.Options, "cd_result": c.Result,
               "cd_server_options": c.ServerOptions, "cd_server_stats": c.ServerStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "curldiv.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)
