"""dipole_forward_noalloc: the forward query entry point that allocates nothing.

Some callers cannot call cudaMalloc: code that runs under a fixed device-memory
budget or inside an application whose allocator owns all device memory, and
loops that must not allocate because cudaMalloc/cudaFree can synchronize the
device or fail part way through under memory pressure.  For them the library
keeps the forward pass's scratch (query sort buffers and the work counter) in a
static device array.  This test calls that entry point through the C ABI,
twice in a row on different query sets (the second call finds the first call's
leftovers in the shared array), and checks each result against dipole_forward
and against the CPU oracle with the forward tolerance used everywhere else
(1e-4, max norm per channel); it also checks, through the library's
allocation counter, that those calls allocated nothing, and that q = 0 is a
no-op.  It lives in a file that pytest collects last and passes both alone and
after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2405_16788_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _normwise(y, ref):
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.max(np.abs(ref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return np.max(np.abs(y - ref), axis=0) / den


def _call(lib, tree, q, n, out, stream):
    return lib.dipole_forward_noalloc(ctypes.c_void_p(tree.handle),
                                      ctypes.c_void_p(q.data_ptr() if q is not None else None),
                                      n, ctypes.c_float(2.0),
                                      ctypes.c_void_p(out.data_ptr() if out is not None else None),
                                      stream)


def test_forward_noalloc_matches_forward_and_oracle_twice():
    import torch
    import oracle
    from paper_2405_16788_gb300 import dipole

    lib = dipole.load_library()
    w = syn.workload("scene-200k", scale=0.1)
    c = w.cloud
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tree = dipole.DipoleTree(t(c.points), t(c.normals), t(c.areas), t(c.eps))
    tree.refit(t(w.mu))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ot = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    ot.update(w.mu)

    # two calls in a row with different sizes; the second one reuses the array
    for qs in (w.queries[:50000], w.queries[60000:60000 + 3001]):
        q = t(qs)
        ref = tree.forward(q, 2.0).cpu().numpy()
        out = torch.full((len(qs), tree.C), float("nan"), device=dev)
        torch.cuda.synchronize()
        allocs0 = dipole.dipole_device_allocations()
        rc = _call(lib, tree, q, len(qs), out, stream)
        assert rc == dipole.DIPOLE_OK, dipole.dipole_last_error()
        assert dipole.dipole_device_allocations() == allocs0  # nothing allocated
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(_normwise(got, ref) <= TOL), _normwise(got, ref)
        # against the oracle's FP64 Barnes-Hut on a sample of the queries
        idx = np.random.default_rng(len(qs)).choice(len(qs), 2000, replace=False)
        oref = ot.forward(qs[idx], 2.0)
        assert np.all(_normwise(got[idx], oref) <= TOL), _normwise(got[idx], oref)
    # q = 0 is a no-op that touches nothing
    allocs0 = dipole.dipole_device_allocations()
    assert _call(lib, tree, None, 0, None, stream) == dipole.DIPOLE_OK
    assert dipole.dipole_device_allocations() == allocs0
    tree.sync_status()


def test_forward_noalloc_rejects_more_than_its_limit():
    import torch
    from paper_2405_16788_gb300 import dipole

    lib = dipole.load_library()
    w = syn.workload("sphere-2k")
    c = w.cloud
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tree = dipole.DipoleTree(t(c.points), t(c.normals), t(c.areas), t(c.eps))
    tree.refit(t(w.mu))
    n_big = (1 << 18) + 1
    q = torch.zeros((n_big, 3), device="cuda")
    out = torch.empty((n_big, 1), device="cuda")
    rc = lib.dipole_forward_noalloc(ctypes.c_void_p(tree.handle), ctypes.c_void_p(q.data_ptr()),
                                    n_big, ctypes.c_float(2.0), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == dipole.DIPOLE_EINVAL
    assert "262144" in dipole.dipole_last_error()
    tree.sync_status()
