"""The C-ABI library builds, loads and exports every entry point declared in include/prony.h.

No compute call is made here (these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prony.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(prony_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_11430_gb300.build import build
    build()
    from paper_2012_11430_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("prony_solve", "prony_build_S", "prony_eval", "prony_solve_batched", "prony_ctx_create",
                 "prony_ctx_destroy", "prony_expsum_fwd_dev", "prony_expsum_bwd_dev", "prony_toeplitz_mm_dev"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2012_11430_gb300 import binding
    assert set(binding.EXPORTS) == set(_declared_functions())


def test_default_opts_and_status_strings(lib):
    from paper_2012_11430_gb300 import binding
    o = binding.default_opts()
    assert o.oversample_p == -1 and o.rank_mode == 0
    assert binding.status_string(binding.PRONY_ERANK) == "numerical rank below m"
    assert binding.status_string(binding.PRONY_EINVAL) == "invalid argument"


def test_ctx_create_without_device_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.prony_ctx_create(ctypes.byref(h), 0)
    assert rc in (-5, -1) and not h.value


def test_built_for_sm103a():
    from paper_2012_11430_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of prony_opts / prony_info / prony_stats have the C layout: sizes and
    field offsets printed by a C program compiled against include/prony.h."""
    import shutil
    import subprocess
    from paper_2012_11430_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"prony_opts": binding.PronyOpts, "prony_info": binding.PronyInfo, "prony_stats": binding.PronyStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "prony.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('  printf("enum PRONY_FFT32 %d\\n", (int)PRONY_FFT32);')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
    assert got[("enum", "PRONY_FFT32")] == binding.PRONY_FFT32
