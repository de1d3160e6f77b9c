"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hydro.h declares; host-side argument checks (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(hydro_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_10987_gb300 import _build, hydro
    _build.build()
    return hydro._lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hydro_create", "hydro_step", "hydro_update", "hydro_destroy", "hydro_status"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_exposes_same_names(lib):
    from paper_2107_10987_gb300 import hydro
    for name in declared_functions():
        assert callable(getattr(hydro, name, None)), f"binding lacks {name}"


def test_host_side_argument_checks(lib):
    from paper_2107_10987_gb300 import hydro as H
    out = C.c_void_p()
    assert lib.hydro_create(None, 5 / 3, 0.0, C.byref(out)) == H.HYDRO_EINVAL
    assert lib.hydro_create(C.byref(H.Layout(12, 3, 1)), 5 / 3, 0.0, C.byref(out)) == H.HYDRO_EINVAL
    assert lib.hydro_create(C.byref(H.Layout(8, 2, 1)), 5 / 3, 0.0, C.byref(out)) == H.HYDRO_EINVAL
    assert lib.hydro_create(C.byref(H.Layout(8, 3, 0)), 5 / 3, 0.0, C.byref(out)) == H.HYDRO_EINVAL
    assert lib.hydro_create(C.byref(H.Layout(8, 3, 2)), 5 / 3, 0.0, C.byref(out)) == H.HYDRO_EUNSUP
    assert lib.hydro_create(C.byref(H.Layout(8, 3, 1)), 1.0, 0.0, C.byref(out)) == H.HYDRO_EINVAL
    assert lib.hydro_create(C.byref(H.Layout(8, 3, 1)), float("nan"), 0.0, C.byref(out)) == H.HYDRO_EINVAL
    assert lib.hydro_step(None, None, 0.0, None, None, None, None) == H.HYDRO_EINVAL
    assert lib.hydro_update(None, None, None, None, 0.0, None, 0, None, None) == H.HYDRO_EINVAL
    assert lib.hydro_selftest_arith(None, None, -1, None, None) == H.HYDRO_EINVAL
    assert lib.hydro_selftest_arith(None, None, 4, None, None) == H.HYDRO_EINVAL
    assert lib.hydro_selftest_arith(None, None, 0, None, None) == H.HYDRO_OK
    assert lib.hydro_strerror(H.HYDRO_EINVAL).startswith(b"invalid")
    lib.hydro_destroy(None)  # no-op


def test_kernels_compiled_for_sm103a():
    from paper_2107_10987_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's field
    offsets and size (a field added on one side only fails here)."""
    import shutil
    import subprocess
    from paper_2107_10987_gb300 import amr, hydro as H
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(H.Layout, "hydro_layout_t"), (H.Mode, "hydro_mode_t"), (H.Batch, "hydro_batch_t"),
             (H.RK3Desc, "hydro_rk3_desc_t"), (amr.AMRDesc, "hydro_amr_t")]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hydro.h"', "int main(void) {"]
    for cls, cname in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cls, cname in pairs:
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
