"""The C-ABI library builds, loads and exports every entry point include/*.h declares (no GPU needed)."""

import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fs3?_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0807_2387_gb300 import build
    build.build()
    import paper_0807_2387_gb300 as pkg
    return pkg.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fs_plan_create", "fs_plan_create_fem", "fs_set_charges", "fs_eval_potential", "fs_eval_field",
              "fs_plan_destroy", "fs_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"libfemnfft.so does not export {name}"


def test_binding_covers_every_declared_symbol():
    from paper_0807_2387_gb300 import _native
    import paper_0807_2387_gb300 as pkg
    for name in _declared():
        assert name in _native.EXPORTED, name
        if name not in ("fs_last_error", "fs_version"):
            assert hasattr(pkg, name), f"python binding lacks {name}"


def test_version_and_error_string_without_gpu(lib):
    assert b"sm_103a" in lib.fs_version()
    assert isinstance(lib.fs_last_error(), bytes)


def test_library_is_sm103a_only():
    from paper_0807_2387_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_missing_library_fails_loudly(tmp_path):
    from paper_0807_2387_gb300 import _native
    saved = _native._lib
    try:
        _native._lib = None
        with pytest.raises(_native.NativeLibraryMissing):
            _native.load(str(tmp_path / "absent.so"))
    finally:
        _native._lib = saved


def test_product_path_does_not_import_the_oracle():
    pkg_dir = os.path.join(ROOT, "paper_0807_2387_gb300")
    for path in glob.glob(os.path.join(pkg_dir, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg_dir, "csrc", "*")):
        text = open(path, errors="replace").read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), path


def test_binding_layouts_and_constants_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the header's size and field offsets, and the
    binding's status, dtype and flag constants have the header's values (compiled with gcc)."""
    import ctypes
    import shutil
    import subprocess

    from paper_0807_2387_gb300 import _native as N

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fs_opts": N.FsOpts, "fs_info": N.FsInfo, "fs_instance": N.FsInstance,
               "fs_batch_facts": N.FsBatchFacts}
    consts = ["FS_OK", "FS_EINVAL", "FS_EDOMAIN", "FS_ENOMEM", "FS_ECUDA", "FS_ETIMEOUT", "FS_EUNSUPPORTED",
              "FS_F32", "FS_F64", "FS_FLAG_NO_KAHAN", "FS_FLAG_TIMING", "FS_FLAG_AUTOTUNE", "FS_FLAG_SERIAL",
              "FS_PROBE_FFMA", "FS_PROBE_FFMA2", "FS_PROBE_MUFU", "FS_FLAG_SPREAD_DIRECT", "FS_FLAG_SPREAD_TILES"]
    lines = ['#include <stdio.h>', '#include "femnfft.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("off {cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    for c in consts:
        lines.append(f'printf("const {c} %lld\\n", (long long)({c}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            kind, name, value = line.split()
            got[(kind, name)] = int(value)
    for cname, cls in structs.items():
        assert got[("size", cname)] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[("off", f"{cname}.{field}")] == getattr(cls, field).offset, (cname, field)
    for c in consts:
        assert got[("const", c)] == getattr(N, c), c


def _header_params():
    """Parameter kinds of every fs_/fs3_ entry point, read from the header's declarations."""
    text = ""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text += re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(fs3?_\w+)\s*\(([^()]*)\)\s*;", text):
        params = [p.strip() for p in m.group(2).split(",")]
        if params == ["void"]:
            params = []
        kinds = []
        for p in params:
            if "*" in p:
                kinds.append("ptr")
            elif re.search(r"\bint64_t\b", p):
                kinds.append("i64")
            elif re.search(r"\bdouble\b", p):
                kinds.append("f64")
            else:
                kinds.append("i32")   # int, unsigned, fs_dtype (an enum)
        out[m.group(1)] = kinds
    return out


def test_binding_argument_kinds_match_the_header(lib):
    """The binding passes each entry point as many arguments as the header declares, each of
    the declared kind (pointer, 64-bit integer, 32-bit integer or enum, double)."""
    import ctypes
    decl = _header_params()
    assert decl, "no declarations parsed"
    for name, kinds in decl.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None, name
        got = []
        for t in argtypes:
            if t is ctypes.c_void_p or t is ctypes.c_char_p or hasattr(t, "_type_") and issubclass(t, ctypes._Pointer):
                got.append("ptr")
            elif t is ctypes.c_int64:
                got.append("i64")
            elif t is ctypes.c_double:
                got.append("f64")
            elif t in (ctypes.c_int, ctypes.c_uint):
                got.append("i32")
            else:
                got.append(repr(t))
        assert got == kinds, (name, got, kinds)
