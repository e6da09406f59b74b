"""The ctypes mirrors of the header's structs (CPU): compiled against
include/ffgpu.h with the host C compiler, every struct's size and every
field's offset must equal what the Python binding declares, so the binding
and the C ABI cannot drift apart."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_cs_0601133_gb300 import ffgpu as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("ffgpu_options", binding.Options), ("ffgpu_tuned", binding.Tuned),
         ("ffgpu_fgemm_desc", binding.FgemmDesc), ("ffgpu_multimod_desc", binding.MultimodDesc),
         ("ffgpu_request", binding.Request), ("ffgpu_completion", binding.Completion),
         ("ffgpu_server_stats", binding.ServerStats), ("ffgpu_plan_info", binding.PlanInfo),
         ("ffgpu_kernel_time", binding.KernelTime)]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ffgpu.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in PAIRS:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_argument_counts_match_the_header():
    import re
    txt = open(os.path.join(ROOT, "include", "ffgpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    decls = re.findall(r"FFGPU_API\s+[\w\s\*]+?\b(ffgpu_\w+)\s*\(([^)]*)\)\s*;", txt)
    assert len(decls) >= 40
    for name, params in decls:
        params = " ".join(params.split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(binding.SIGNATURES[name]) == n, name
