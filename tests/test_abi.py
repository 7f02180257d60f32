"""The C ABI: the library builds for sm_103a, loads, exports every function that
include/sfhk.h declares, and the ctypes mirrors match the header's layouts.
No compute calls (runs without a GPU)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(sfhk_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2601_17164_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(libpath):
    names = declared_functions()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(sfhk_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = C.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n)


def test_library_is_built_for_sm_103a_only():
    from paper_2601_17164_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_ctypes_layouts_match_header():
    from paper_2601_17164_gb300 import sfhk as S
    mirrors = {"sfhk_pulse": S.Pulse, "sfhk_field_info": S.FieldInfo, "sfhk_target_desc": S.TargetDesc,
               "sfhk_birth_params": S.BirthParams, "sfhk_births": S.BirthsC, "sfhk_prop_params": S.PropParams,
               "sfhk_endpoints": S.EndpointsC, "sfhk_phase_times": S.PhaseTimes}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sfhk.h"', 'int main(void) {']
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append('printf("sfhk_stats size %zu\\n", sizeof(sfhk_stats));')
    for k, f in enumerate(S.STATS_FIELDS):
        lines.append(f'printf("sfhk_stats {f} %zu\\n", offsetof(sfhk_stats, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            parts = ln.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
    assert got[("sfhk_stats", "size")] == 8 * S.STATS_WORDS
    for k, f in enumerate(S.STATS_FIELDS):
        assert got[("sfhk_stats", f)] == 8 * k, f


def test_binding_refuses_to_run_without_gpu():
    # the product path has no CPU fallback: without a CUDA device a call fails loudly
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2601_17164_gb300 import sfhk as S
    with pytest.raises(Exception):
        S.Field(1e14, 800, 2, 0, 0.02, 0.1)
