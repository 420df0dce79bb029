"""The checked build of the library (nvcc -DDIPOLE_CHECKED): the traversals
test every index they read from an array (work items and their order, the query
permutation, parents, a leaf's point range) before using it and report
DIPOLE_EBOUNDS instead of an out-of-range access.  compute-sanitizer is not
available here; this build stands in for its bounds checking.  The library is
compiled separately (libdipole_checked.so), and the forward, adjoint, gradient,
stage, appearance, grid, bf16-moment and treelet tests run against it in a child process, where
every status check (dipole_sync_status) would report a caught index."""
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_tests_pass_on_the_checked_build():
    from paper_2405_16788_gb300 import _build
    path = _build.build(checked=True)
    env = dict(os.environ, DIPOLE_LIBRARY=path)
    probe = subprocess.run(
        [sys.executable, "-c", "from paper_2405_16788_gb300 import dipole; "
         "print(int(dipole.dipole_checked_build()))"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert probe.stdout.strip() == "1", probe.stdout + probe.stderr
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu and not slow",
         "tests/test_gpu_forward.py", "tests/test_gpu_adjoint.py", "tests/test_gpu_grad.py",
         "tests/test_gpu_stages.py", "tests/test_gpu_appearance.py", "tests/test_gpu_grid.py",
         "tests/test_gpu_bf16_moments.py", "tests/test_gpu_treelet.py"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]


def test_normal_build_is_not_checked():
    from paper_2405_16788_gb300 import dipole
    if os.environ.get("DIPOLE_LIBRARY"):
        pytest.skip("another build was selected")
    assert not dipole.dipole_checked_build()
