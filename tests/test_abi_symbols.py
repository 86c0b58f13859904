"""The C-ABI library loads and exports every symbol declared in include/*.h (no GPU needed)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(spdba_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2609_03922_gb300 import build as B
    B.build()
    from paper_2609_03922_gb300 import spdba
    return spdba.lib()


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ["spdba_plan_create", "spdba_step", "spdba_get_field", "spdba_get_mask", "spdba_fft_exec",
              "spdba_block_activity", "spdba_classify"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2609_03922_gb300 import spdba
    for n in declared_symbols():
        assert hasattr(lib, n), "missing export %s" % n
        assert n in spdba.SIGNATURES, "binding lacks %s" % n


def test_host_only_calls(lib):
    """Calls that touch no device: defaults, status strings, argument errors."""
    from paper_2609_03922_gb300 import spdba
    o = spdba.options_default()
    assert o.mode == spdba.SPDBA_MODE_ADAPTIVE and o.transitions == 1 and abs(o.dt - 0.01) < 1e-15
    assert lib.spdba_status_string(spdba.SPDBA_ERR_UNSUPPORTED) == b"unsupported size"
    import ctypes
    p = ctypes.c_void_p()
    # a length with prime factor 5 is rejected before any device work
    dims = (ctypes.c_int64 * 2)(160, 64)
    blk = (ctypes.c_int32 * 2)(16, 16)
    assert lib.spdba_plan_create(ctypes.byref(p), 2, dims, blk, 1e-6, 10, ctypes.byref(o)) == spdba.SPDBA_ERR_UNSUPPORTED
    assert b"not 2^a 3^b" in lib.spdba_last_error()
    assert lib.spdba_step(None, 1) == spdba.SPDBA_ERR_ARG


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the header's layout: every
    field's offset and each structure's size, as the C compiler lays them out
    (a field appended on one side only would shift the rest silently)."""
    import shutil
    import subprocess
    from paper_2609_03922_gb300 import spdba
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [spdba.spdba_options, spdba.spdba_stats, spdba.spdba_tune_report, spdba.spdba_kernel_time]
    lines = ['#include <stdio.h>', '#include "spdba.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in st._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == ctypes_sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, "%s.%s" % (name, f)


def ctypes_sizeof(st):
    import ctypes
    return ctypes.sizeof(st)
