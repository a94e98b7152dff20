"""The C ABI: libnqs.so builds for sm_103a, loads without a GPU, and exports every function
that include/nqs.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nqs.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(nqs_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["nqs_problem_create", "nqs_connections", "nqs_amplitudes",
                     "nqs_energy_grad", "nqs_pt2", "nqs_status_string", "nqs_diag"]:
        assert required in names


def test_library_loads_and_exports_all_symbols():
    from paper_2601_21310_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding binds exactly the exported entry points
    from paper_2601_21310_b300 import nqs
    assert set(nqs.EXPORTS) <= set(declared_functions())


def test_library_targets_sm103a():
    from paper_2601_21310_b300 import build
    lib_path = build.build()
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    assert out.returncode == 0
    assert "sm_103a" in out.stdout


def test_status_strings_without_gpu():
    from paper_2601_21310_b300 import nqs
    L = nqs.lib()
    assert L.nqs_status_string(0) == b"ok"
    assert b"sorted" in L.nqs_status_string(-2)
    assert L.nqs_version().startswith(b"nqs-b300")
