"""The C ABI library builds for sm_103a and exports every entry point that
include/kf.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

from paper_1701_02324_gb300 import _abi, _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kf_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_declared_symbols():
    lib = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (kf_[A-Za-z_0-9]+)", out))
    decl = declared_symbols()
    assert decl, "no declarations found"
    missing = [s for s in decl if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_ctypes_signatures_cover_header():
    assert sorted(_abi.SIGNATURES) == declared_symbols()


def test_library_loads_without_gpu():
    lib = _abi.load()
    assert lib.kf_status_string(4) == b"KF_EILLCOND"
    assert lib.kf_status_string(0) == b"KF_OK"


def test_header_is_plain_c_and_links(tmp_path):
    """include/kf.h compiles as strict C99 with warnings as errors, and a C
    program that takes the address of every declared entry point links
    against libkf.so (run needs no GPU: it is only linked)."""
    lib = _build.build()
    names = declared_symbols()
    src = tmp_path / "use_kf.c"
    src.write_text(
        '#include "kf.h"\n'
        "typedef void (*fp)(void);\n"
        "fp kf_all[] = {\n" + "".join(f"  (fp){n},\n" for n in names) + "};\n"
        "int main(void) {\n"
        "  kf_opts o = {0};\n"
        "  kf_solve_info info = {0};\n"
        "  o.precision = KF_PREC_MIXED;\n"
        "  return (int)(sizeof(kf_all) / sizeof(kf_all[0])) + o.precision + info.iters - 1 - "
        f"{len(names)};\n"
        "}\n")
    obj = tmp_path / "use_kf.o"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(src), "-o", str(obj)], check=True)
    subprocess.run(["gcc", str(obj), "-L", os.path.dirname(lib), "-lkf",
                    "-Wl,--unresolved-symbols=ignore-in-shared-libs", "-o", str(tmp_path / "use_kf")], check=True)
