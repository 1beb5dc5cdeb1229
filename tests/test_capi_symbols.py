"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/lxo.h; the binding uses the same names."""
import ctypes
import os
import re

from paper_2203_14354_gb300 import _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lxo_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert {"lxo_create", "lxo_propagate", "lxo_trace_rays", "lxo_build_bvh"} <= names
    lib = ctypes.CDLL(_capi.lib_path() if os.path.exists(_capi.lib_path()) else _capi.lib()._name)
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() == set(_capi._SIGNATURES)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    L = _capi.lib()
    ctx = ctypes.c_void_p()
    assert L.lxo_create(ctypes.byref(ctx), 0) == _capi.LXO_ERR_CUDA  # no CPU fallback
    assert not ctx.value


def test_checked_build_compiles_and_exports_every_symbol():
    """The checked build (bounds compared inside the kernels) is a flag of the
    same sources: it compiles for sm_103a and exports the same entry points."""
    from paper_2203_14354_gb300 import build
    path = build.build(checked=True)
    assert path == build.LIB_CHECKED and path != build.LIB
    lib = ctypes.CDLL(path)
    for n in sorted(declared_symbols()):
        assert hasattr(lib, n), n


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of the binding has the size and field offsets that a C
    compiler gives the declaration in include/lxo.h."""
    import subprocess
    structs = [c for c in vars(_capi).values()
               if isinstance(c, type) and issubclass(c, ctypes.Structure) and c.__name__.startswith("lxo_")]
    assert {"lxo_material", "lxo_source", "lxo_event", "lxo_results", "lxo_run_params"} <= {c.__name__ for c in structs}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lxo.h"', "int main(void) {"]
    for c in structs:
        lines.append(f'printf("{c.__name__} size %zu\\n", sizeof({c.__name__}));')
        for f in c._fields_:
            lines.append(f'printf("{c.__name__} {f[0]} %zu\\n", offsetof({c.__name__}, {f[0]}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for c in structs:
        assert int(got[f"{c.__name__} size"]) == ctypes.sizeof(c), c.__name__
        for f in c._fields_:
            assert int(got[f"{c.__name__} {f[0]}"]) == getattr(c, f[0]).offset, (c.__name__, f[0])


def test_binding_constants_match_the_header(tmp_path):
    """Every LXO_* constant the binding defines has the value of the macro or
    enumerator of the same name in include/lxo.h."""
    import subprocess
    names = [k for k, v in vars(_capi).items() if k.startswith("LXO_") and isinstance(v, (int, float))]
    assert {"LXO_MAX_TBINS", "LXO_FLAG_ADJOINT", "LXO_SURF_NONE", "LXO_ERR_CUDA"} <= set(names)
    lines = ["#include <stdio.h>", '#include "lxo.h"', "int main(void) {"]
    for n in names:
        lines.append(f'printf("{n} %.17g\\n", (double)({n}));')
    lines.append("return 0; }")
    (tmp_path / "consts.c").write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(tmp_path / "consts.c"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = dict(zip(out[0::2], map(float, out[1::2])))
    for n in names:
        assert got[n] == float(getattr(_capi, n)), n
