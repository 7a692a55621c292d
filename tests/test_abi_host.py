"""Host-side checks of the C ABI (no GPU compute): the library builds, loads and
exports every function include/irlnqs.h declares, and the ctypes structures
have the C layout."""
import os
import re
import subprocess

import pytest

import __graft_entry__ as entry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "irlnqs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    entry.build()
    from paper_2601_01437_gb300 import abi
    return abi


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 11
    L = lib.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lib.exported_symbols()) == names


def test_struct_layouts_match_c(lib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "irlnqs.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(lm_system), sizeof(lm_pencil_info), sizeof(irl_params), sizeof(irl_result));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(irl_params, seed), offsetof(irl_params, v0), offsetof(irl_result, status), offsetof(lm_pencil_info, energy), offsetof(lm_system, build_arith));
  printf("%zu %zu\\n", sizeof(lm_stats), offsetof(lm_stats, tri_count));
  printf("%zu %zu %zu %zu %zu\\n", sizeof(lm_batch_item), offsetof(lm_batch_item, irl), offsetof(lm_batch_item, theta_inout), sizeof(lm_response), offsetof(lm_response, t_done_ms));
  printf("%zu %zu\\n", sizeof(lm_pencil_info), offsetof(lm_pencil_info, grid));
  printf("%zu %zu\\n", sizeof(lm_ctx_params), offsetof(lm_ctx_params, hbm_gbs));
  return 0; }
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    import ctypes
    want = [ctypes.sizeof(lib.lm_system), ctypes.sizeof(lib.lm_pencil_info),
            ctypes.sizeof(lib.irl_params), ctypes.sizeof(lib.irl_result),
            lib.irl_params.seed.offset, lib.irl_params.v0.offset, lib.irl_result.status.offset,
            lib.lm_pencil_info.energy.offset, lib.lm_system.build_arith.offset,
            ctypes.sizeof(lib.lm_stats), lib.lm_stats.tri_count.offset,
            ctypes.sizeof(lib.lm_batch_item), lib.lm_batch_item.irl.offset,
            lib.lm_batch_item.theta_inout.offset, ctypes.sizeof(lib.lm_response),
            lib.lm_response.t_done_ms.offset,
            ctypes.sizeof(lib.lm_pencil_info), lib.lm_pencil_info.grid.offset,
            ctypes.sizeof(lib.lm_ctx_params), lib.lm_ctx_params.hbm_gbs.offset]
    assert [int(x) for x in out] == want


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.LMError) as e:
        lib.Context(0)
    assert e.value.code == lib.LM_ERR_CUDA
