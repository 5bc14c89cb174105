"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry
point declared in include/mor.h (no compute calls here)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "mor.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mor_[A-Za-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2404_06260_gb300 import _build
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor
    assert sorted(mor.EXPORTED) == _declared()


def test_error_message_without_gpu_work():
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor
    o = mor.basis_opts(rank=12, oversample=3)
    assert o.rank == 12 and o.oversample == 3 and o.precision == mor.MIXED
    rc = mor._lib.mor_build_bases(None, ctypes.byref(o), None, None)
    assert rc == -1 and b"null" in mor._lib.mor_last_error()


def test_binding_fails_loudly_without_the_library():
    # no fallback: with libmor.so absent, importing the binding raises ImportError
    import subprocess
    import sys
    code = ("import os, sys; sys.path.insert(0, %r); real = os.path.exists; "
            "os.path.exists = lambda p: False if str(p).endswith('libmor.so') else real(p)\n"
            "try:\n"
            "    import paper_2404_06260_gb300.mor\n"
            "except ImportError as e:\n"
            "    print('ImportError', e)\n"
            "else:\n"
            "    print('imported')\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.stdout.startswith("ImportError") and "not built" in out.stdout, out
