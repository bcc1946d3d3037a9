"""The C ABI library builds for sm_103a, loads, and exports every declared symbol.

CPU only: no call here reaches the GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1802_03980_gb300 import build
    return build()


def _declared():
    src = open(os.path.join(ROOT, "include", "kf_track.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["kf_default_params", "kf_track_create", "kf_track_destroy", "kf_set_frame",
              "kf_set_model", "kf_align", "kf_align_batch", "kf_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1802_03980_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()
    for name in _declared():
        assert callable(getattr(_lib, name))


def test_struct_layouts_match_the_header(lib_path, tmp_path):
    # kf_default_params runs on the host only; it fills the struct through the ABI
    from paper_1802_03980_gb300 import _lib
    p = _lib.kf_default_params()
    assert (p.levels, list(p.max_iters)[:3], p.hist_bins) == (3, [10, 5, 4], 512)
    assert p.d_max == pytest.approx(0.16) and p.band_kappa == 1.0 and p.conv_window == 3
    assert p.flags == 7 and p.bilateral_radius == 2 and p.bilateral_sigma_r == pytest.approx(0.03)
    assert (p.normal_mode, p.shoot_radius, p.ii_radius_max) == (_lib.KF_NORMALS_CROSS, 0, 8)
    assert (p.ii_radius_a, p.ii_radius_b) == (2.0, 1.0) and p.ii_depth_change == pytest.approx(0.02)
    # sizes and field offsets as a C compiler lays them out from the header
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"kf_params": _lib.kf_params, "kf_result": _lib.kf_result,
               "kf_intrinsics": _lib.kf_intrinsics, "kf_iter_record": _lib.kf_iter_record,
               "kf_profile": _lib.kf_profile}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kf_track.h"', 'int main(void){']
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {cname}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_invalid_arguments_are_rejected_without_a_gpu(lib_path):
    from paper_1802_03980_gb300 import _lib
    lib = _lib._lib
    assert lib.kf_default_params(None) == _lib.KF_ERR_INVALID_ARG
    p = _lib.kf_default_params()
    p.levels = 9
    h = ctypes.c_void_p()
    assert lib.kf_track_create(ctypes.byref(p), 640, 480, None, ctypes.byref(h)) == _lib.KF_ERR_INVALID_ARG
    # the normal and association variants are checked before any device call
    for field, value in (("normal_mode", 2), ("shoot_radius", 5), ("shoot_radius", -1)):
        q = _lib.kf_default_params()
        setattr(q, field, value)
        assert lib.kf_track_create(ctypes.byref(q), 640, 480, None, ctypes.byref(h)) == _lib.KF_ERR_INVALID_ARG
    q = _lib.kf_default_params()
    q.normal_mode, q.ii_radius_max = _lib.KF_NORMALS_INTEGRAL, 16
    assert lib.kf_track_create(ctypes.byref(q), 640, 480, None, ctypes.byref(h)) == _lib.KF_ERR_INVALID_ARG
    assert lib.kf_align(None, None, None, 0.0, None, None) == _lib.KF_ERR_INVALID_ARG
    assert lib.kf_last_error(None) == b"null tracker"
