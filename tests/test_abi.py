"""The C-ABI library builds, loads and exports every entry point that
include/st.h declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "st.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("st_setup_mesh", "st_residual", "st_jacobian_apply", "st_vanka_smooth", "st_vcycle", "st_newton_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2603_28706_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_binding_lists_every_symbol():
    import paper_2603_28706_gb300 as st
    assert sorted(st.EXPORTED) == declared_symbols()


def test_setup_rejects_bad_parameters_without_gpu():
    # parameter validation happens before any CUDA call
    import paper_2603_28706_gb300 as st
    import st_inputs as si
    lib = st.load()
    h = ctypes.c_void_p()
    for bad in (dict(dim=4), dict(p=2.5), dict(k=7), dict(levels=3, nx=6), dict(delta=0.0), dict(nx=0),
                dict(gamma_cip=-1.0), dict(finest_patches=2), dict(finest_patches=1, gamma_cip=1.0),
                dict(coarse_solve=2), dict(coarse_solve=1, nx=16, ny=16, nz=16, levels=1), dict(pressure_space=2),
                dict(smoother=3), dict(omega_coarse=-1.0), dict(patch_type=2),
                dict(patch_type=1, finest_patches=0), dict(patch_type=1, finest_patches=1, gamma_cip=0.5),
                dict(patch_type=1, finest_patches=1, pressure_space=1)):
        P = st.params(si.base_params(**bad))
        assert lib.st_setup_mesh(ctypes.byref(P), None, ctypes.byref(h)) == st.ST_EINVAL
    assert lib.st_setup_mesh(None, None, ctypes.byref(h)) == st.ST_EINVAL
    assert lib.st_destroy(None) == st.ST_OK


def test_batch_setup_rejects_mixed_dim_or_k_without_gpu():
    # dim / k must agree across a batch; checked before any CUDA call
    import paper_2603_28706_gb300 as st
    import st_inputs as si
    lib = st.load()
    b = ctypes.c_void_p()
    for other in (dict(k=2), dict(dim=2, nx=4, ny=4)):
        arr = (st.StParams * 2)(st.params(si.base_params(k=1)), st.params(si.base_params(**other)))
        assert lib.st_batch_setup(arr, 2, None, ctypes.byref(b)) == st.ST_EINVAL
    assert lib.st_batch_setup(None, 1, None, ctypes.byref(b)) == st.ST_EINVAL
    arr = (st.StParams * 1)(st.params(si.base_params()))
    assert lib.st_batch_setup(arr, 0, None, ctypes.byref(b)) == st.ST_EINVAL
    assert lib.st_batch_destroy(None) == st.ST_OK


def test_binding_carries_the_optional_fields():
    import paper_2603_28706_gb300 as st
    import st_inputs as si
    P = st.params(si.base_params(gamma_cip=0.5, finest_patches=0, pressure_space=1, coarse_solve=1, smoother=1))
    assert P.gamma_cip == 0.5 and P.finest_patches == 0 and P.pressure_space == 1 and P.coarse_solve == 1
    assert P.smoother == 1
    assert st.params(si.base_params(patch_type=1)).patch_type == 1
    # the allocation-free mass norm implements the Q2/Q1 pair only
    with pytest.raises(ValueError):
        st.mnorm_noalloc(si.base_params(pressure_space=1), None)


def test_binding_struct_layout_matches_the_header(tmp_path):
    # the ctypes mirrors of the parameter and info structs against the C
    # compiler's layout of include/st.h (size and every field offset)
    import shutil
    import subprocess
    import paper_2603_28706_gb300 as st
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"st_params": st.StParams, "st_linsolve_info": st.StLinsolveInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "st.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
