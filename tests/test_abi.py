"""The C-ABI library loads and exports every entry point its header declares (CPU only)."""
import os
import re

import pytest

import paper_2011_05090_gb300 as rgs
from paper_2011_05090_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "librgs.h")).read()
    return sorted(set(re.findall(r"^RGS_API\s+[\w\s\*]+?\b((?:rgs|rgmres|cgs2)_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return rgs.load()


def test_header_declares_the_documented_api():
    names = _declared()
    for must in ("rgs_qr", "rgs_arnoldi_step", "rgmres_solve", "rgmres_solve_batched", "rgmres_set_preconditioner"):
        assert must in names
    assert set(names) == set(rgs.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_only_the_c_api_is_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", rgs.LIB_PATH], capture_output=True, text=True).stdout
    text_syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert text_syms == set(_declared())


def test_status_strings(lib):
    assert lib.rgs_status_string(rgs.RGS_OK) == b"ok"
    assert b"breakdown" in lib.rgs_status_string(rgs.RGS_ERR_BREAKDOWN)
    assert lib.rgs_status_string(99) == b"unknown status"


def test_missing_library_fails_loudly(tmp_path):
    # the binding has no CPU fallback: without librgs.so every entry point raises
    import subprocess
    import sys
    code = (
        "import paper_2011_05090_gb300 as rgs\n"
        f"rgs.LIB_PATH = {str(tmp_path / 'absent.so')!r}\n"
        "rgs._lib = None\n"
        "try:\n"
        "    rgs.rgs_create()\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    raise SystemExit('no error without the library')\n"
    )
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "raised:" in out.stdout and "is missing" in out.stdout


def _header_constants():
    """Integer constants of the header: #define NAME <int> (or another constant), enum NAME = <int>."""
    text = open(os.path.join(ROOT, "include", "librgs.h")).read()
    consts = {}
    for name, val in re.findall(r"^#define\s+(RGS_[A-Z0-9_]+)\s+([A-Za-z0-9_]+)\b", text, re.M):
        if re.fullmatch(r"\d+", val):
            consts[name] = int(val)
        elif val in consts:
            consts[name] = consts[val]
    for name, val in re.findall(r"\b(RGS_[A-Z0-9_]+)\s*=\s*(\d+)", text):
        consts[name] = int(val)
    m = re.search(r"#define\s+RGS_NOALLOC_SCRATCH_BYTES\s+\(\(size_t\)(\d+)\s*<<\s*(\d+)\)", text)
    if m:
        consts["RGS_NOALLOC_SCRATCH_BYTES"] = int(m.group(1)) << int(m.group(2))
    return consts


def test_binding_constants_match_the_header():
    consts = _header_constants()
    for must in ("RGS_OK", "RGS_ERR_BREAKDOWN", "RGS_F32", "RGS_SKETCH_SRHT", "RGS_QR_FP64_FINE",
                 "RGS_QR_FP64_SKETCH", "RGS_PRECOND_LEARNED_CONV", "RGS_PRECOND_CALLBACK", "RGS_ERR_CALLBACK",
                 "RGS_NOALLOC_SCRATCH_BYTES"):
        assert must in consts, must
    for name, val in consts.items():
        if hasattr(rgs, name):
            assert getattr(rgs, name) == val, name
    assert all(hasattr(rgs, n) for n in consts if n.startswith(("RGS_ERR_", "RGS_QR_", "RGS_SKETCH_")))


_STRUCTS = [("rgs_qr_info", rgs.QRInfo), ("rgs_csr", rgs.CSR), ("rgmres_opts", rgs.GmresOpts),
            ("rgmres_info", rgs.GmresInfo), ("rgmres_batch_opts", rgs.BatchOpts), ("rgs_tuning", rgs.Tuning),
            ("rgs_learned_precond", rgs.LearnedPrecond), ("rgs_callback_precond", rgs.CallbackPrecond)]


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (a C program
    compiled against librgs.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "librgs.h"', "int main(void) {"]
    for cname, py in _STRUCTS:
        lines.append(f'    printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=120)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                              text=True, timeout=60).stdout.split("\n") if line)
    for cname, py in _STRUCTS:
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, f"{cname}.{fname}"


def test_precond_trampoline_turns_an_exception_into_a_status():
    """The binding's C callback never lets a Python exception cross the C frame: it returns 1 and
    keeps the exception for the solve's error (with or without a GPU)."""
    errors = []

    def fn(v, z):
        raise ValueError("planted")

    cb = rgs._precond_trampoline(fn, errors)
    assert cb(None, 0, 0, rgs.RGS_F32, 0, rgs.RGS_F32, None) == 1
    assert len(errors) == 1 and isinstance(errors[0], Exception)
