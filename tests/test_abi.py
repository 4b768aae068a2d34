"""The C-ABI library loads and exports every entry point include/gmc.h
declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*([A-Za-z_]\w*)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(n for n in names if n not in ("if", "while", "for", "return", "sizeof")))


@pytest.fixture(scope="module")
def libgmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_13965_gb300 import _abi
    return ctypes.CDLL(_abi.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gmc_create", "gmc_destroy", "gmc_load_weights", "gmc_transmit",
                 "analog_transmit", "transport_solve"):
        assert must in names


def test_every_declared_symbol_is_exported(libgmc):
    missing = [n for n in declared_functions() if not hasattr(libgmc, n)]
    assert not missing, missing


def test_status_strings_and_null_handling(libgmc):
    from paper_2512_13965_gb300 import _abi
    assert _abi.status_name(0) == "GMC_OK"
    assert _abi.status_name(-5) == "GMC_EFORMAT"
    # null context is rejected without touching a device
    assert _abi.lib.gmc_destroy(None) == 0
    assert _abi.lib.gmc_synchronize(None) == _abi.GMC_EINVAL
    assert _abi.lib.gmc_transmit(None, 1, None, None, 0, 0, 1, 0, 0, None, None) == _abi.GMC_EINVAL
