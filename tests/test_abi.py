"""The C-ABI library builds, loads and exports every entry point that
include/dipole.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dipole.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dipole_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2405_16788_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["dipole_build_tree", "dipole_refit", "dipole_forward", "dipole_adjoint",
                 "dipole_tree_destroy", "dipole_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dipole_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_through_binding(lib_path):
    from paper_2405_16788_gb300 import dipole
    lib = dipole.load_library()
    for n in _declared():
        assert hasattr(lib, n)
    assert set(dipole.EXPORTED) <= set(_declared())
    assert isinstance(dipole.dipole_last_error(), str)


def test_argument_errors_without_gpu(lib_path):
    """Host-side validation rejects bad arguments before touching the device."""
    from paper_2405_16788_gb300 import dipole
    lib = dipole.load_library()
    out = ctypes.c_void_p()
    assert lib.dipole_build_tree(None, None, None, None, 10, None, None, ctypes.byref(out)) == -1
    assert "required" in dipole.dipole_last_error()
    assert lib.dipole_forward(None, None, 0, 2.0, None, None) == -1
    assert lib.dipole_refit(None, None, 4, 0, None) == -1
    assert lib.dipole_adjoint(None, None, 0, 2.0, None, None, 0, None) == -1
    assert lib.dipole_forward_grad(None, None, 0, 2.0, None, None, None, None, None) == -1
    assert lib.dipole_adjoint_grad(None, None, 0, 2.0, None, None, None, 0, None, None, None) == -1
    assert lib.dipole_adjoint_stage1(None, None, 0, 2.0, None, None, 0, None, None, None) == -1
    assert lib.dipole_adjoint_stage2(None, None, None, 0, None) == -1
    assert lib.dipole_adjoint_acc_size(None, None) == -1
    assert lib.dipole_adjoint_queries(None, None, 0, 2.0, None, None, 0, None) == -1
    assert lib.dipole_query_packet_counts(None, None, 0, 2.0, None, None, None) == -1
    assert isinstance(dipole.dipole_device_allocations(), int)
    lib.dipole_tree_destroy(None)  # a no-op
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    bad_kernel = dipole._BuildParams(8, 10, 2)
    assert lib.dipole_build_tree(fake, fake, fake, None, 10, ctypes.byref(bad_kernel), None,
                                 ctypes.byref(out)) == -1
    assert "kernel" in dipole.dipole_last_error()


def test_oracle_and_library_share_nothing():
    """The oracle neither includes the library's headers nor imports its package."""
    osrc = open(os.path.join(ROOT, "oracle", "dipole_oracle.c")).read()
    opy = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "#include \"" not in osrc
    assert "paper_2405_16788_gb300" not in re.sub(r'""".*?"""', "", opy, flags=re.S)
    for f in os.listdir(os.path.join(ROOT, "paper_2405_16788_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2405_16788_gb300", "csrc", f)).read()
    pkg = os.path.join(ROOT, "paper_2405_16788_gb300")
    for f in sorted(x for x in os.listdir(pkg) if x.endswith(".py")):
        txt = open(os.path.join(pkg, f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt


def test_tree_import_validates_host_arrays_before_device_work(lib_path):
    """dipole_tree_import rejects out-of-range topology on the host (no GPU
    needed: the device pointers below are never dereferenced)."""
    import numpy as np
    from paper_2405_16788_gb300 import dipole
    lib = dipole.load_library()
    n, nn = 4, 3
    fake = ctypes.c_void_p(16)  # stands in for device pointers; validation fails first
    perm = np.array([0, 1, 2, 3], np.uint32)
    first = np.array([0, 0, 2], np.int32)
    count = np.array([4, 2, 2], np.int32)
    level = np.array([0, 1, 1], np.int32)
    skip = np.array([3, 2, 3], np.int32)
    leaf = np.array([0, 1, 1], np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)

    def call(perm=perm, first=first, count=count, level=level, skip=skip, leaf=leaf, nn=nn):
        out = ctypes.c_void_p()
        return lib.dipole_tree_import(fake, fake, fake, None, n, None, p(perm), p(first), p(count),
                                      p(level), p(skip), p(leaf), nn, None, None, ctypes.byref(out))

    assert call(perm=np.array([0, 1, 1, 3], np.uint32)) == dipole.DIPOLE_EINVAL
    assert "permutation" in dipole.dipole_last_error()
    assert call(skip=np.array([3, 2, 4], np.int32)) == dipole.DIPOLE_EINVAL
    assert call(count=np.array([4, 2, 3], np.int32)) == dipole.DIPOLE_EINVAL
    assert call(level=np.array([0, 11, 1], np.int32)) == dipole.DIPOLE_EINVAL
    assert call(leaf=np.array([0, 2, 1], np.int32)) == dipole.DIPOLE_EINVAL
    assert call(nn=0) == dipole.DIPOLE_EINVAL


def test_every_entry_point_is_documented_with_its_passage():
    """Each declaration in include/dipole.h follows a comment that names the
    paper passage it implements (section, equation, algorithm, appendix) or
    states that the paper has no counterpart (one comment may head a group of
    declarations)."""
    src = open(HEADER).read()
    for n in _declared():
        i = re.search(r"^[A-Za-z].*\b%s\(" % n, src, re.M).start()  # the declaration
        j = src.rfind("*/", 0, i)
        k = src.rfind("/*", 0, j)
        assert j >= 0 and k >= 0, n
        doc = " ".join(src[k:j].replace("*", " ").split())
        assert re.search(r"Sec\.|eq\.|Alg\.|App\.|no counterpart", doc), n


def test_binding_has_the_same_names():
    txt = open(os.path.join(ROOT, "paper_2405_16788_gb300", "dipole.py")).read()
    missing = [n for n in _declared() if not re.search(r"^def %s\(" % n, txt, re.M)]
    assert not missing, missing
