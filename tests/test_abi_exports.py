"""The C-ABI library builds (nvcc, sm_103a) and exports every function that include/*.h
declares; no GPU is needed (nothing is called)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", header or "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"^\s*int\s+(k2\w+)\s*\(", src, flags=re.M))
    return names


def test_headers_declare_the_abi():
    names = _declared()
    for must in ("k2svd_dgesvd2", "k2svd_sgesvd2", "k2svd_dtrsvd2", "k2svd_strsvd2", "k2svd_dgesvd2_bwd",
                 "k2svd_dkogbet", "k2svd_skogbet", "k2svd_dkogbet_ws", "k2probe_rate"):
        assert must in names


def test_library_exports_every_declared_symbol():
    """libk2svd exports every function of k2svd.h and no probe; libk2probe every function of
    k2probe.h."""
    from paper_2407_13116_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared("k2svd.h")) if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.k2svd_version() == 100
    assert not any(hasattr(lib, n) for n in _declared("k2probe.h"))
    probe = ctypes.CDLL(build.PROBE_LIB)
    missing = [n for n in sorted(_declared("k2probe.h")) if not hasattr(probe, n)]
    assert not missing, missing


def test_headers_compile_as_c99_and_cpp(tmp_path):
    """The public headers are plain C: they compile as C99 (pedantic) and as C++."""
    import shutil
    import subprocess
    inc = os.path.join(ROOT, "include")
    for cc, std, name in (("gcc", "-std=c99", "h.c"), ("g++", "-std=c++11", "h.cpp")):
        if not shutil.which(cc):
            continue
        src = tmp_path / name
        src.write_text('#include "k2svd.h"\n#include "k2probe.h"\nint main(void) { return 0; }\n')
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + inc, "-fsyntax-only", str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
