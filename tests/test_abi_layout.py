"""CPU checks that the Python binding and the C headers agree: every
prototype in include/*.h against the ctypes signature the binding declares
(argument count, width and signedness, pointer-ness, result type), and the
ctypes mirrors of the C structs and enums against offsets, sizes and values
that a C compiler prints from the headers themselves."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2009_10035_gb300 import f2v

ENUMS = {"f2v_status", "f2v_model", "f2v_precision", "f2v_schedule", "f2v_job_state"}
SCALARS = {
    "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint32_t": ctypes.c_uint32,
    "uint64_t": ctypes.c_uint64, "size_t": ctypes.c_size_t, "float": ctypes.c_float,
    "double": ctypes.c_double, "uint8_t": ctypes.c_uint8, "char": ctypes.c_char,
}


def _prototypes():
    out = {}
    for fn in sorted(os.listdir(f2v.INCLUDE)):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(f2v.INCLUDE, fn)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        text = re.sub(r"#[^\n]*", " ", text)
        for m in re.finditer(r"([A-Za-z_][\w \t\*]*?)\b(f2v_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
            ret = " ".join(m.group(1).split())
            params = [" ".join(p.split()) for p in m.group(3).split(",")]
            if params == ["void"]:
                params = []
            out[m.group(2)] = (ret, params)
    return out


def _ctype_of(decl: str):
    """('ptr', depth, base) or ('val', ctypes type) for a C declaration."""
    words = decl.replace("*", " * ").split()
    depth = words.count("*")
    base = [w for w in words if w not in ("*", "const")]
    if len(base) > 1:                          # drop the parameter name
        base = base[:-1]
    base = base[0]
    if depth:
        return ("ptr", depth, base)
    if base in ENUMS:
        return ("val", ctypes.c_int)
    return ("val", SCALARS[base])


def test_every_declared_function_has_a_binding_signature():
    protos, sigs = _prototypes(), f2v.signatures()
    assert set(protos) == set(f2v.header_functions())
    assert set(protos) == set(sigs), (set(protos) ^ set(sigs))


@pytest.mark.parametrize("name", sorted(_prototypes()))
def test_binding_signature_matches_the_prototype(name):
    ret, params = _prototypes()[name]
    args, res = f2v.signatures()[name]
    assert len(args) == len(params), (name, params)
    for decl, ct in zip(params, args):
        kind = _ctype_of(decl)
        if kind[0] == "val":
            assert ct is kind[1], (name, decl, ct)
            continue
        _, depth, base = kind
        if ct is ctypes.c_void_p:
            continue                           # any pointer, passed as an address
        assert issubclass(ct, ctypes._Pointer), (name, decl, ct)
        target = ct._type_
        if depth == 2:
            assert target is ctypes.c_void_p, (name, decl)
        else:
            want = ctypes.c_int if base in ENUMS else SCALARS[base]
            assert ctypes.sizeof(target) == ctypes.sizeof(want), (name, decl, target)
            assert target(-1).value == want(-1).value, (name, decl, target)   # signedness
    if ret == "void":
        assert res is None, name
    elif ret in ("const char *", "const char*"):
        assert res is ctypes.c_char_p, name
    else:
        assert ret == "f2v_status" and res is ctypes.c_int, (name, ret, res)


STRUCTS = {"f2v_tiling": f2v.Tiling, "f2v_job": f2v.JobSpec,
           "f2v_job_info": f2v.JobInfo, "f2v_server_stats": f2v.ServerStats}
CONSTANTS = {
    "F2V_OK": f2v.OK, "F2V_EINVAL": f2v.EINVAL, "F2V_ENOMEM": f2v.ENOMEM,
    "F2V_ECUDA": f2v.ECUDA, "F2V_ETIMEOUT": f2v.ETIMEOUT, "F2V_ESTATE": f2v.ESTATE,
    "F2V_TDIST": f2v.TDIST, "F2V_SIGMOID": f2v.SIGMOID, "F2V_FR": f2v.FR,
    "F2V_LINLOG": f2v.LINLOG, "F2V_FORCEATLAS": f2v.FORCEATLAS,
    "F2V_FP32": f2v.FP32, "F2V_BF16": f2v.BF16,
    "F2V_LR_CONSTANT": f2v.LR_CONSTANT, "F2V_LR_LINEAR": f2v.LR_LINEAR,
    "F2V_FLAG_CHECK_SYMMETRY": f2v.FLAG_CHECK_SYMMETRY,
    "F2V_FLAG_NO_STAGING": f2v.FLAG_NO_STAGING,
    "F2V_FLAG_SHARED_SAMPLES": f2v.FLAG_SHARED_SAMPLES,
    "F2V_FLAG_RANDOM_PARTITION": f2v.FLAG_RANDOM_PARTITION,
    "F2V_JOB_QUEUED": f2v.JOB_QUEUED, "F2V_JOB_RUNNING": f2v.JOB_RUNNING,
    "F2V_JOB_DONE": f2v.JOB_DONE, "F2V_JOB_FAILED": f2v.JOB_FAILED,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "f2v_batch.h"',
             '#include "f2v_serve.h"', 'int main(void) {']
    for cname, st in STRUCTS.items():
        lines.append(f'printf("Z {cname} %zu\\n", sizeof({cname}));')
        for field, _ in st._fields_:
            lines.append(f'printf("S {cname} {field} %zu %zu\\n", offsetof({cname}, {field}), '
                         f'sizeof((({cname} *)0)->{field}));')
    for cname in CONSTANTS:
        lines.append(f'printf("C {cname} %lld\\n", (long long)({cname}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", f2v.INCLUDE, str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        tag, *rest = line.split()
        if tag == "S":
            table[(rest[0], rest[1])] = (int(rest[2]), int(rest[3]))
        else:
            table[rest[0]] = int(rest[1])
    return table


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_mirrors_match_the_c_layout(c_layout, cname):
    st = STRUCTS[cname]
    assert ctypes.sizeof(st) == c_layout[cname]
    for field, _ in st._fields_:
        off, size = c_layout[(cname, field)]
        desc = getattr(st, field)
        assert (desc.offset, desc.size) == (off, size), (cname, field)


def test_python_constants_match_the_headers(c_layout):
    for cname, value in CONSTANTS.items():
        assert c_layout[cname] == value, cname
