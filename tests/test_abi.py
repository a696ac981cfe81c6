"""The C-ABI library builds, loads, and exports every entry point include/mg.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1402_1763_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_init", "mg_init_batch", "mg_sweep", "mg_read_s", "mg_read_pk",
                     "mg_read_stats", "mg_sync", "mg_last_error", "mg_destroy", "mg_philox"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_build_exports_every_declared_symbol(lib):
    """The bounds-checked variant (built beside the main library) has the same
    entry points and reports itself through mg_build_flags."""
    from paper_1402_1763_gb300 import build
    chk = ctypes.CDLL(build.LIB_CHECKED)
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing
    chk.mg_build_flags.restype = ctypes.c_int32
    lib.mg_build_flags.restype = ctypes.c_int32
    assert chk.mg_build_flags() == 1 and lib.mg_build_flags() == 0


def test_fault_injection_hook_rejects_bad_arguments_without_gpu(lib):
    from paper_1402_1763_gb300 import _native as nv
    L = nv.library()
    assert L.mg_inject_cuda_error(None, 1) == nv.MG_EINVAL


def test_binding_mirrors_the_abi():
    import paper_1402_1763_gb300 as pkg
    missing = [n for n in declared_functions() if not hasattr(pkg, n)]
    assert not missing, missing


def test_options_defaults_without_gpu(lib):
    from paper_1402_1763_gb300 import mg_options_init
    o = mg_options_init()
    assert o.precision == 64 and o.n_chains == 1 and o.tau_scale == 1.0 and not o.P0
    assert o.persistent == 0 and o.autotune == 0 and o.mixing == 0


def test_binding_structs_match_the_header(tmp_path):
    """Field offsets and sizes of the ctypes mirrors equal the C compiler's
    layout of the structs in include/mg.h."""
    import ctypes
    import shutil
    import subprocess
    from paper_1402_1763_gb300._native import MgGrid, MgOptions, MgStats
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mg_grid": MgGrid, "mg_options": MgOptions, "mg_stats": MgStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "mg.h")}"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_null_arguments_are_rejected_without_gpu(lib):
    from paper_1402_1763_gb300 import _native as nv
    L = nv.library()
    assert L.mg_sweep(None, 1) == nv.MG_EINVAL
    assert L.mg_read_pk(None, 0, None) == nv.MG_EINVAL
    assert L.mg_init(None, None, None, None, None, None, 4, 1, None) == nv.MG_EINVAL
    L.mg_destroy(None)
    assert isinstance(L.mg_last_error(None), bytes)
