"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a,
loads, exports every function include/sidelobe.h declares, and rejects bad
plan descriptions before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_03478_gb300 import _lib
    return _lib.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sidelobe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("sidelobe_plan_create", "synth_spin_maps", "interp_tod", "adjoint_tod", "plan_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2201_03478_gb300 import _lib
    names = _declared_functions()
    assert sorted(_lib.EXPORTS) == names
    for n in names:
        assert getattr(lib, n) is not None


def _desc(**kw):
    from paper_2201_03478_gb300 import _lib
    rt = kw.pop("ring_theta", W.equiangular_ring_theta(16))
    d = dict(lmax=16, kmax=2, ncomp=1, nrings=rt.size, nphi=32, interp_order=4, precision=0, device=0)
    d.update(kw)
    keep = np.ascontiguousarray(rt, dtype=np.float64)
    return _lib.PlanDesc(ring_theta=keep.ctypes.data_as(ctypes.c_void_p), stream=None, **d), keep


@pytest.mark.parametrize("bad,status", [
    (dict(lmax=0), -1), (dict(kmax=17), -1), (dict(kmax=-1), -1), (dict(ncomp=2), -1),
    (dict(nphi=31), -1), (dict(nphi=4), -1), (dict(nphi=14), -2), (dict(interp_order=8), -2),
    (dict(interp_order=3), -1), (dict(interp_order=-2), -1),
    (dict(precision=7), -1), (dict(nrings=3), -1), (dict(nphi=20000), -1), (dict(lmax=200, kmax=129), -1),
])
def test_bad_descriptions_are_rejected(lib, bad, status):
    d, keep = _desc(**bad)
    out = ctypes.c_void_p()
    st = lib.sidelobe_plan_create(ctypes.byref(out), ctypes.byref(d))
    assert st == status
    assert out.value is None
    assert len(lib.sl_last_error()) > 0


def test_asymmetric_or_unsorted_rings_are_rejected(lib):
    rt = W.equiangular_ring_theta(16)
    bad = rt.copy()
    bad[2] += 1e-6
    for r in (bad, rt[::-1].copy(), np.concatenate([[0.0], rt[1:]])):
        d, keep = _desc(ring_theta=r)
        out = ctypes.c_void_p()
        assert lib.sidelobe_plan_create(ctypes.byref(out), ctypes.byref(d)) == -1


def test_null_arguments(lib):
    assert lib.sidelobe_plan_create(None, None) == -1
    assert lib.synth_spin_maps(None, None, None, None) == -1
    assert lib.interp_tod(None, None, None, None, None, 0, None) == -1
    assert lib.adjoint_tod(None, None, None, None, None, 0, None, None, None, None, 0) == -1
    lib.plan_destroy(None)
    assert lib.sl_plan_reserve(None, 10) == -1
    assert lib.sl_plan_set_tile_cols(None, 16) == -1
    assert lib.sl_orbital_moments(None, None, None) == -1
    assert lib.orbital_dipole_tod(None, None, 2.7255, 1.0, None, None, None, 0, None, None, 0, 20, None, 0) == -1


def test_batch_arguments_are_checked_before_any_device_call(lib):
    from paper_2201_03478_gb300 import _lib
    out = ctypes.c_void_p()
    assert lib.sl_batch_create(None, None, 0, None, 0) == -1
    assert lib.sl_batch_create(ctypes.byref(out), None, 1, None, 0) == -1
    items = (_lib.BatchItem * 2)()
    assert lib.sl_batch_create(ctypes.byref(out), items, 0, None, 0) == -1
    assert lib.sl_batch_create(ctypes.byref(out), items, 2, None, 0) == -1        # no plan
    assert b"no plan" in lib.sl_last_error()
    assert not out.value
    assert lib.sl_batch_run(None) == -1
    info = _lib.BatchInfo()
    assert lib.sl_batch_get_info(None, ctypes.byref(info)) == -1
    lib.sl_batch_destroy(None)


def test_oracle_builds():
    import oracle
    assert os.path.exists(oracle.build())


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/sidelobe.h compiles as C99 (no C++ in the boundary) and a C program
    that takes the address of every declared function links against the library
    (nothing is called: no GPU here)."""
    import shutil
    import subprocess
    from paper_2201_03478_gb300 import _build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = _declared_functions()
    src = tmp_path / "use_abi.c"
    src.write_text("#include \"sidelobe.h\"\n#include <stdio.h>\n"
                   "typedef void (*fn)(void);\n"
                   "int main(void) {\n    const fn f[] = {\n"
                   + "".join("        (fn)&%s,\n" % n for n in names)
                   + "    };\n    printf(\"%d\\n\", (int)(sizeof f / sizeof f[0]));\n    return 0;\n}\n")
    libdir = os.path.dirname(_build.LIB)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(tmp_path / "use_abi"), "-L", libdir,
                        "-lsidelobe", "-Wl,-rpath," + libdir, "-Wl,--allow-shlib-undefined"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
