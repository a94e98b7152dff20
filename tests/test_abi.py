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
    """Every compile and the link of libnqs.so generate sm_103a code only (one -gencode pair,
    arch=compute_103a, code=sm_103a), and the build writes no other architecture."""
    from paper_2601_21310_b300 import build
    gen = ["-gencode", "arch=compute_103a,code=sm_103a"]
    for cmd in (build.compile_cmd("nvcc", "x.cu", "x.o"), build.link_cmd("nvcc", ["x.o"], "l.so")):
        assert cmd.count("-gencode") == 1
        i = cmd.index("-gencode")
        assert cmd[i:i + 2] == gen
        assert not any(a.startswith(("-arch", "--gpu-architecture", "-code")) for a in cmd)


def test_status_strings_without_gpu():
    from paper_2601_21310_b300 import nqs
    L = nqs.lib()
    assert L.nqs_status_string(0) == b"ok"
    assert b"sorted" in L.nqs_status_string(-2)
    assert L.nqs_version().startswith(b"nqs-b300")


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of nqs_opts, nqs_csr and nqs_detset have the C layout: offsets and
    sizes as gcc lays out the header's structs."""
    import shutil

    from paper_2601_21310_b300 import nqs as N
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("gcc not available")
    structs = {"nqs_opts": N.Opts, "nqs_csr": N.CSRStruct, "nqs_detset": N.DetSetStruct}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nqs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_layout = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert c_layout[(cname, "size")] == ctypes.sizeof(py)
        for fname, _ in py._fields_:
            assert c_layout[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def _prototypes():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = {}
    for m in re.finditer(r"^\s*((?:const\s+)?\w+\s*\**)\s*\b(nqs_\w+)\s*\(([^;{]*?)\)\s*;", txt,
                         flags=re.S | re.M):
        params = " ".join(m.group(3).split())
        protos[m.group(2)] = (" ".join(m.group(1).split()),
                              [] if params in ("", "void") else [p.strip()
                                                                 for p in params.split(",")])
    return protos


def test_binding_argtypes_match_the_prototypes():
    """Every bound entry point passes as many arguments as the header declares, each of the
    declared kind (pointer / stream, 32-bit int, int64_t, double)."""
    from paper_2601_21310_b300 import nqs as N
    protos = _prototypes()

    def kind_of_c(p):
        if "*" in p or p.startswith("nqs_stream_t"):
            return "ptr"
        t = p.rsplit(" ", 1)[0] if " " in p else p
        return {"int": "i32", "int64_t": "i64", "double": "f64"}.get(t.replace("const ", ""), t)

    def kind_of_ctypes(t):
        return {ctypes.c_void_p: "ptr", ctypes.c_char_p: "ptr", ctypes.c_int: "i32",
                ctypes.c_int64: "i64", ctypes.c_double: "f64"}[t]

    ret_kinds = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "const char*": ctypes.c_char_p,
                 "void": None}
    for name, (restype, argtypes) in N.EXPORTS.items():
        assert name in protos, name
        ret, params = protos[name]
        assert ret_kinds[ret.replace(" *", "*")] is restype, (name, ret)
        c_kinds = [kind_of_c(p) for p in params]
        assert c_kinds == [kind_of_ctypes(t) for t in argtypes], name
