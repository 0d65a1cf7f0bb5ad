"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header
declares (CPU only: no compute call is made without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1810_04221_gb300 import build as B

HEADER = os.path.join(B.INCLUDE, "cwm_amg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b((?:amg|cwm)_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_expected_entry_points():
    names = _declared()
    for must in ("amg_setup", "amg_vcycle", "amg_pcg_solve", "amg_free", "cwm_edge_weights",
                 "cwm_suitor_match", "cwm_aggregate", "cwm_galerkin"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    from paper_1810_04221_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_library_loads_and_host_calls_work(lib_path):
    lib = C.CDLL(lib_path)
    for n in _declared():
        getattr(lib, n)
    from paper_1810_04221_gb300 import binding
    p = binding.amg_default_params()
    assert (p.sweeps_per_level, p.coarse_max, p.max_levels) == (2, 40, 40)
    assert (p.pre_sweeps, p.post_sweeps, p.coarse_sweeps) == (1, 1, 20)
    # the remaining documented defaults
    assert (p.vcycle_fp32, p.check_input, p.keep_sweeps, p.loop_cap, p.trace) == (0, 1, 0, 0, 0)
    assert (p.tail_rows, p.stall_ratio, p.gamma, p.galerkin_fp32_from, p.coupled_post) == (-1, 0.0, 1, 0, 0)
    assert (p.block3, p.sliced) == (0, 0)
    assert binding.status_name(binding.AMG_ERR_NOT_SPD) == "AMG_ERR_NOT_SPD"
    # argument checks happen before any device work
    lib.amg_num_levels.restype = C.c_int
    assert lib.amg_num_levels(None) == -1
    binding.load(lib_path)
    L = binding.load()
    ll = C.c_longlong()
    assert L.cwm_copy(None, None, 16, None) == binding.AMG_ERR_INVALID_ARG
    assert L.cwm_copy(C.c_void_p(8), C.c_void_p(16), -1, None) == binding.AMG_ERR_INVALID_ARG
    assert L.cwm_copy(None, None, 0, None) == binding.AMG_OK  # nothing to copy: no device work
    assert L.cwm_div_check(16, 1, None, C.byref(ll), None) == binding.AMG_ERR_INVALID_ARG
    assert L.cwm_div_check(-1, 1, C.byref(ll), C.byref(ll), None) == binding.AMG_ERR_INVALID_ARG


def test_struct_layout_matches_c(tmp_path):
    """sizeof and every field's offsetof of the public structs, compiled by the host C
    compiler, against the ctypes mirrors."""
    from paper_1810_04221_gb300 import binding
    structs = [("amg_params", binding.AmgParams), ("amg_info", binding.AmgInfo)]
    lines = []
    for cname, cls in structs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        lines += [f'printf("%zu\\n", offsetof({cname}, {f}));' for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cwm_amg.h"\n'
                   'int main(void){' + "".join(lines) + 'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = []
    for _, cls in structs:
        want.append(C.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert got == want
