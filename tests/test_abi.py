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


def test_binding_checks_buffer_sizes_and_types(libgmc):
    # The binding checks every array against the layout the call touches
    # before the library runs; nothing here reaches a GPU.
    import numpy as np
    import torch
    from paper_2512_13965_gb300 import _abi
    n = 10
    ok = np.zeros((4, n), np.float32)
    assert _abi._arr(ok, 4, 4 * n, "exit") == ok.ctypes.data
    assert _abi._arr(None, 4, 4 * n, "exit") is None
    assert _abi._arr(torch.zeros(5, n), 4, 5 * n, "cond") is not None
    for bad, why in ((np.zeros((4, n), np.float64), "bytes"), (np.zeros((3, n), np.float32), "needed"),
                     (torch.zeros(4, n, dtype=torch.float16), "bytes")):
        with pytest.raises(_abi.GMCError) as e:
            _abi._arr(bad, 4, 4 * n, "exit")
        assert e.value.status == _abi.GMC_EINVAL and why in str(e.value)
    # the wrappers apply it: a float64 grid is refused before any call is made
    ctx = object.__new__(_abi.Context)
    ctx.handle, ctx.cells = None, {}
    with pytest.raises(_abi.GMCError) as e:
        _abi.transport_solve(ctx, 4, 4, np.ones(16), np.ones(16, np.float32),
                             np.ones(16, np.float32), 10, 0, 1, np.zeros(16))
    assert "tau" in str(e.value)
    with pytest.raises(_abi.GMCError) as e:
        _abi.analog_transmit(ctx, n, *[np.zeros(n, np.float32)] * 5, 0, 0, 0, 0,
                             np.zeros(n, np.int32), np.zeros((4, n - 1), np.float32))
    assert "exit" in str(e.value)
    # the geometry variants' solves: a short flux or wall array is refused
    g16 = [np.ones(16, np.float32)] * 3
    with pytest.raises(_abi.GMCError) as e:
        _abi.transport_solve_rect(ctx, 4, 4, *g16, 0.5, 1.5, 10, 0, 1, np.zeros(15))
    assert "flux" in str(e.value)
    with pytest.raises(_abi.GMCError) as e:
        _abi.transport_solve_xy(ctx, 4, 4, np.ones(16, np.float32), np.ones(16, np.float32),
                                np.ones(16), 10, 0, 1, np.zeros(16))
    assert "source" in str(e.value)
    with pytest.raises(_abi.GMCError) as e:
        _abi.transport_solve_wall_xy(ctx, 4, 4, np.ones(16, np.float32), np.ones(16, np.float32),
                                     np.ones(3, np.float32), 10, 0, 1, np.zeros(16))
    assert "wall" in str(e.value)
    ctx.handle = None


def test_pointer_classification_rejects_another_gpus_memory(tmp_path):
    # The rule every array argument goes through (csrc/ptr_kind.h), compiled
    # into a host-only program: device memory of the context's GPU and managed
    # memory are used directly, another GPU's memory is refused, page-locked
    # host memory with a device address is used in place, other host memory is
    # staged. The memory-type codes are checked against the CUDA runtime's
    # enum, from its header alone (no GPU, no CUDA library call).
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if not gxx or not os.path.exists(os.path.join(inc, "driver_types.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "t.cpp"
    src.write_text(r'''
#include <driver_types.h>
#include "ptr_kind.h"
using namespace gmc;
static_assert(cudaMemoryTypeUnregistered == 0 && cudaMemoryTypeHost == 1 &&
              cudaMemoryTypeDevice == 2 && cudaMemoryTypeManaged == 3, "cudaMemoryType codes");
int main() {
  int bad = 0;
  bad += classify_pointer(cudaMemoryTypeDevice, 0, 0, true) != kPtrDevice;
  bad += classify_pointer(cudaMemoryTypeDevice, 3, 3, true) != kPtrDevice;
  bad += classify_pointer(cudaMemoryTypeDevice, 1, 0, true) != kPtrOtherDevice;
  bad += classify_pointer(cudaMemoryTypeDevice, 0, 1, true) != kPtrOtherDevice;
  bad += classify_pointer(cudaMemoryTypeManaged, 1, 0, true) != kPtrDevice;
  bad += classify_pointer(cudaMemoryTypeHost, 0, 0, true) != kPtrMappedHost;
  bad += classify_pointer(cudaMemoryTypeHost, 0, 0, false) != kPtrHost;
  bad += classify_pointer(cudaMemoryTypeUnregistered, -2, 0, false) != kPtrHost;
  return bad;
}
''')
    exe = tmp_path / "t"
    r = subprocess.run([gxx, "-std=c++17", "-I", inc, "-I",
                        os.path.join(ROOT, "paper_2512_13965_gb300", "csrc"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0


def test_header_is_plain_c(tmp_path):
    # include/gmc.h is the boundary for C callers: it compiles as strict C99
    # (no C++ in it) and as C++, with every warning on and none given
    import shutil
    import subprocess
    inc = os.path.join(ROOT, "include", "gmc.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        exe = shutil.which(cc)
        if not exe:
            pytest.skip("needs " + cc)
        r = subprocess.run([exe, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                            "-x", lang, inc], capture_output=True, text=True)
        assert r.returncode == 0, (cc, r.stderr)
