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
