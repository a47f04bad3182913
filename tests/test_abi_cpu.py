"""The C-ABI library builds, loads and exports every declared symbol (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2107_05200_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2107_05200_gb300 import build
        build.build()
    return _native, _native.load()


def _declared():
    with open(os.path.join(ROOT, "include", "ffadmm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ffa_[A-Za-z_]+)\s*\(", text)))


def test_header_declares_the_api():
    names = _declared()
    for must in ("ffa_create", "ffa_init", "ffa_iterate", "ffa_energy", "ffa_gradient", "ffa_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound():
    native, lib = _lib()
    names = _declared()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(native.EXPORTED) == names


def test_default_params_and_struct_layout():
    native, lib = _lib()
    p = native.Params()
    assert lib.ffa_default_params(C.byref(p)) == 0
    assert p.energy == 0 and p.rho == 1.0 and p.eps_abs == 1e-6 and p.eps_rel == 1e-5
    assert p.check_every == 10 and p.require_flip_free == 1 and p.refine_sweeps == 2
    assert p.nd_leaf_size == 64
    assert list(p.solve_subtree_height) == [-1, -1]
    assert p.factor_device == 0 and p.top_inverse_levels == 0
    assert lib.ffa_default_params(None) == 1
    assert isinstance(lib.ffa_last_error(None), bytes)


def test_null_arguments_are_rejected_without_a_device():
    native, lib = _lib()
    out = C.c_void_p()
    assert lib.ffa_create(None, None, 0, None, None, None, C.byref(out)) == 1
    assert out.value is None
    assert lib.ffa_create(None, None, 0, None, None, None, None) == 1
    lib.ffa_destroy(None)


def test_bad_parameters_are_rejected_before_any_device_work():
    native, lib = _lib()
    import numpy as np
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    T = np.array([[0, 1, 2]], np.int32)
    mesh = native.Mesh(3, 1, 2, 2, C.c_void_p(V.ctypes.data), C.c_void_p(T.ctypes.data))
    p = native.Params()
    lib.ffa_default_params(C.byref(p))
    p.refine_sweeps = 0
    out = C.c_void_p()
    assert lib.ffa_create(C.byref(mesh), None, 0, None, C.byref(p), None, C.byref(out)) == 1
    assert b"refine_sweeps" in lib.ffa_last_error(None)
    lib.ffa_default_params(C.byref(p))
    p.solve_subtree_height[1] = 9
    assert lib.ffa_create(C.byref(mesh), None, 0, None, C.byref(p), None, C.byref(out)) == 1
    assert b"solve_subtree_height" in lib.ffa_last_error(None)
    for bad in (-2, 33):
        lib.ffa_default_params(C.byref(p))
        p.top_inverse_levels = bad
        assert lib.ffa_create(C.byref(mesh), None, 0, None, C.byref(p), None, C.byref(out)) == 1
        assert b"top_inverse_levels" in lib.ffa_last_error(None)
    lib.ffa_default_params(C.byref(p))
    mesh.d = 4
    assert lib.ffa_create(C.byref(mesh), None, 0, None, C.byref(p), None, C.byref(out)) == 1


def test_no_cpu_fallback_without_a_device():
    """Valid inputs on a machine without a GPU: creation fails with FFA_ERR_CUDA and
    a message, rather than running anywhere else; the state and constraint entry
    points reject a NULL context."""
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    native, lib = _lib()
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    T = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    pins = np.array([0], np.int32)
    pos = np.zeros((1, 2))
    mesh = native.Mesh(4, 2, 2, 2, C.c_void_p(V.ctypes.data), C.c_void_p(T.ctypes.data))
    out = C.c_void_p()
    st = lib.ffa_create(C.byref(mesh), C.c_void_p(pins.ctypes.data), 1, C.c_void_p(pos.ctypes.data), None, None,
                        C.byref(out))
    assert st == 4 and out.value is None
    assert lib.ffa_last_error(None)
    assert lib.ffa_set_state(None, None, None, None, None) == 1
    assert lib.ffa_set_constraints(None, 1, None, None, None, None) == 1


def test_build_compiles_every_source_file():
    """Every .cu and .cpp under csrc/ is a translation unit of libffadmm.so (the GPU
    box rebuilds from build.py alone)."""
    from paper_2107_05200_gb300 import build
    csrc = os.path.join(os.path.dirname(os.path.abspath(build.__file__)), "csrc")
    on_disk = {f for f in os.listdir(csrc) if f.endswith((".cu", ".cpp"))}
    assert on_disk == set(build.CU_SOURCES) | set(build.CXX_SOURCES)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every structure the binding passes by pointer has, field by field, the
    offset and size that a C compiler gives the header's declaration, and the
    same total size; a field the binding names but the header lacks fails to
    compile.  The header is compiled as plain C (it promises a C ABI)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    native, _ = _lib()
    pairs = [(native.Mesh, "ffa_mesh"), (native.Params, "ffa_params"), (native.Stats, "ffa_stats"),
             (native.Info, "ffa_info"), (native.Tuning, "ffa_tuning"), (native.PhaseTimes, "ffa_phase_times")]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ffadmm.h"', "int main(void) {"]
    for cls, cname in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3 and parts[1] == "size":
            got[(parts[0], None)] = (int(parts[2]),)
        elif len(parts) == 4:
            got[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    for cls, cname in pairs:
        assert got[(cname, None)] == (C.sizeof(cls),), cname
        for fname, _ in cls._fields_:
            f = getattr(cls, fname)
            assert got[(cname, fname)] == (f.offset, f.size), (cname, fname)


def test_ctypes_signatures_match_the_header_prototypes():
    """Every prototype of the header against the binding's argtypes and restype:
    the same number of arguments, integers and doubles of the same width, enums as
    a C int, pointers as pointers (to the matching structure where the binding
    names one)."""
    native, lib = _lib()
    with open(os.path.join(ROOT, "include", "ffadmm.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    protos = re.findall(r"([A-Za-z_][\w \t\*]*?)\b(ffa_\w+)\s*\(([^;{}]*?)\)\s*;", text)
    assert len(protos) >= 30
    structs = {"ffa_mesh": native.Mesh, "ffa_params": native.Params, "ffa_stats": native.Stats,
               "ffa_info": native.Info, "ffa_tuning": native.Tuning, "ffa_phase_times": native.PhaseTimes}
    scalars = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double}
    enums = {"ffa_energy_kind", "ffa_status", "ffa_precision"}

    def check(ctype_str, ct, where):
        t = ctype_str.replace("const", " ").split()
        stars = "".join(t).count("*")
        base = "".join(t).replace("*", "")
        if stars:
            assert ct is not None and (ct is C.c_void_p or ct is C.c_char_p or issubclass(ct, C._Pointer)), where
            if stars == 1 and base in structs and ct is not C.c_void_p:
                assert ct._type_ is structs[base], where
            if stars == 2 and ct is not C.c_void_p:
                assert ct._type_ is C.c_void_p, where
        elif base in scalars:
            assert ct is scalars[base], where
        elif base in enums:
            assert ct in (C.c_int, C.c_int32, C.c_uint32) and C.sizeof(ct) == 4, where
        else:
            raise AssertionError(f"unmapped C type {ctype_str!r} in {where}")

    for ret, name, args in protos:
        fn = getattr(lib, name)
        params = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        assert fn.argtypes is not None and len(fn.argtypes) == len(params), name
        for p, ct in zip(params, fn.argtypes):
            ctype_str = p.rsplit(None, 1)[0] if not p.endswith("*") else p
            if "*" in p.rsplit(None, 1)[-1]:          # 'double *x' spelled with the star on the name
                ctype_str = p.replace(p.rsplit(None, 1)[-1], "*")
            check(ctype_str, ct, f"{name}({p})")
        r = ret.strip()
        if r == "void":
            assert fn.restype is None, name
        elif r == "const char*":
            assert fn.restype is C.c_char_p, name
        else:
            check(r, fn.restype, f"{name} return")
