"""The C-ABI library builds, loads without a GPU and exports every declared symbol.

No compute call is made here (there is no GPU on this host).
"""
import os
import re
import subprocess

import pytest

import paper_1907_00072_gb300 as ppg
from paper_1907_00072_gb300 import build as ppg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ppg_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    ppg_build.build()
    return ppg.load_library()


def test_header_declares_the_binding_table():
    assert _declared_functions() == sorted(ppg.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", ppg.LIB_PATH], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\bT (ppg_[a-z_0-9]+)", out.stdout))
    for name in _declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_status_strings_without_gpu(lib):
    assert ppg.ppg_status_string(ppg.PPG_OK) == "ok"
    assert "clamped" in ppg.ppg_status_string(ppg.PPG_WARN_DEGREE_CLAMPED)
    assert ppg.ppg_version().startswith("ppg")
    assert ppg.load_library().ppg_last_error() is not None


def test_build_targets_sm_103a_only():
    assert ppg_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path):
    import importlib

    mod = importlib.reload(ppg)
    mod._lib = None
    with pytest.raises(ImportError):
        mod.load_library(str(tmp_path / "libppg.so"))


@pytest.mark.parametrize("name", ["ppg_opts", "ppg_stats", "ppg_batch_system"])
def test_struct_layouts_match_the_header(name, tmp_path):
    """The binding's ctypes mirrors of the header's structs have the C compiler's size and field
    offsets (a host program built with gcc against include/ppg.h prints them)."""
    cls = getattr(ppg, name)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ppg.h"', "int main(void) {",
             f'    printf("%zu\\n", sizeof({name}));']
    lines += [f'    printf("%zu\\n", offsetof({name}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    import ctypes

    assert out[0] == ctypes.sizeof(cls), (name, out[0], ctypes.sizeof(cls))
    for f, off in zip(fields, out[1:]):
        assert getattr(cls, f).offset == off, (name, f, off, getattr(cls, f).offset)
