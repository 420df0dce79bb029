"""Pins for the oracle's octree (Sec. 6.1 / 6.3, "tree construction").

The paper says only "octree" and "follow libigl"; the tree used here is the
compressed 30-bit Morton octree stated in the oracle's header.  These tests
check the oracle's recursive construction against a second, non-recursive
statement of the same definition written here from scratch (enumerate every
run of equal code prefixes at every level and keep the runs the definition
keeps), plus invariants, on small inputs with many duplicate points.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16788_gb300 import synthetic as syn


def test_interleave_bits():
    assert oracle.interleave(1, 0, 0) == 0b100
    assert oracle.interleave(0, 1, 0) == 0b010
    assert oracle.interleave(0, 0, 1) == 0b001
    assert oracle.interleave(1023, 1023, 1023) == (1 << 30) - 1
    assert oracle.interleave(2, 0, 0) == 0b100000
    assert oracle.interleave(512, 0, 0) == 1 << 29
    rng = np.random.default_rng(0)
    for qx, qy, qz in rng.integers(0, 1024, size=(200, 3)):
        ref = 0
        for k in range(10):
            ref |= ((int(qx) >> k) & 1) << (3 * k + 2)
            ref |= ((int(qy) >> k) & 1) << (3 * k + 1)
            ref |= ((int(qz) >> k) & 1) << (3 * k)
        assert oracle.interleave(int(qx), int(qy), int(qz)) == ref


def test_morton_cell_centres():
    """Points at the centres of cells of the 1024^3 grid over their bounding
    cube quantise to those cells."""
    rng = np.random.default_rng(1)
    cells = rng.integers(0, 1024, size=(300, 3))
    cells[0] = [0, 0, 0]
    cells[1] = [1023, 1023, 1023]  # makes the bounding cube [lo, lo + ext] exact-ish
    lo = np.array([-0.75, 0.5, 2.0])
    ext = 2.0  # powers of two keep the cell centres exactly representable
    pts = lo + (cells + 0.5) * (ext / 1024)
    lo32, ext32, codes = oracle.morton(pts.astype(np.float32))
    assert np.allclose(lo32, lo + 0.5 * ext / 1024)
    for (qx, qy, qz), c in zip(cells, codes):
        # the cube starts at the first centre, so cells shift by at most one
        q = [(int(c) >> (3 * k + 2)) & 1 for k in range(10)]
        qx_got = sum(b << k for k, b in enumerate(q))
        assert abs(qx_got - qx) <= 1


def test_morton_degenerate_extent():
    """All points equal: ext = 1 and every code is 0."""
    lo, ext, codes = oracle.morton(np.full((5, 3), 0.3, np.float32))
    assert ext == 1.0 and np.all(codes == 0)


def _definition_tree(codes_sorted, leaf_size, max_depth):
    """Nodes of the compressed octree, enumerated from the definition: every
    maximal run of sorted codes with equal top 3l bits at every level l, kept
    when it is a branching internal node or a leaf whose parent run is open.
    Returns a list of (first, count, level, is_leaf) in (first, level) order."""
    n = len(codes_sorted)
    runs = {}  # level -> list of (s, e)
    for l in range(max_depth + 1):
        key = codes_sorted >> np.uint32(30 - 3 * l) if l > 0 else np.zeros(n, np.uint32)
        bounds = [0] + [i for i in range(1, n) if key[i] != key[i - 1]] + [n]
        runs[l] = list(zip(bounds[:-1], bounds[1:]))

    def run_at(l, i):
        for s, e in runs[l]:
            if s <= i < e:
                return s, e
        raise AssertionError

    nodes = []
    for l in range(max_depth + 1):
        for s, e in runs[l]:
            cnt = e - s
            if l < max_depth and cnt > leaf_size:
                kids = sum(1 for (a, b) in runs[l + 1] if s <= a and b <= e)
                if kids >= 2:
                    nodes.append((s, cnt, l, 0))
                continue
            # leaf candidate: count <= leaf_size, or at the deepest level
            if l == 0:
                nodes.append((s, cnt, l, 1))
                continue
            ps, pe = run_at(l - 1, s)
            if pe - ps > leaf_size:
                nodes.append((s, cnt, l, 1))
    nodes.sort(key=lambda t: (t[0], t[2]))
    return nodes


def _cases():
    rng = np.random.default_rng(42)
    out = []
    for n in [1, 2, 3, 8, 9, 17, 40, 64]:
        p = rng.uniform(-1, 1, size=(n, 3))
        out.append(("uniform", p))
    # many duplicates and clusters: forces level-10 leaves with > leaf_size points
    base = rng.uniform(-1, 1, size=(5, 3))
    p = base[rng.integers(0, 5, 60)]
    out.append(("dups", p))
    p = np.concatenate([np.zeros((20, 3)), rng.uniform(-1, 1, (12, 3)), np.full((11, 3), 0.5)])
    out.append(("dups2", p))
    # a tight cluster far from the rest: long single-child chains
    p = np.concatenate([rng.normal(scale=1e-4, size=(30, 3)), [[1.0, 1.0, 1.0]]])
    out.append(("chain", p))
    return out


@pytest.mark.parametrize("leaf_size,max_depth", [(8, 10), (1, 10), (2, 10), (8, 3), (4, 0)])
def test_tree_matches_definition(leaf_size, max_depth):
    for name, p in _cases():
        p = p.astype(np.float32)
        n = len(p)
        nrm = syn._unit(np.random.default_rng(3).normal(size=(n, 3))).astype(np.float32)
        a = np.full(n, 0.1, np.float32)
        T = oracle.Tree(p, nrm, a, None, leaf_size=leaf_size, max_depth=max_depth)
        e = T.export()
        # order: stable sort by code, ties by input index
        lo, ext, codes = oracle.morton(p)
        order = np.lexsort((np.arange(n), codes))
        assert np.array_equal(e["perm"], order.astype(np.uint32)), name
        assert np.array_equal(e["code"], codes[order]), name
        ref = _definition_tree(codes[order], leaf_size, max_depth)
        got = list(zip(e["first"], e["count"], e["level"], e["is_leaf"]))
        assert [tuple(map(int, g)) for g in got] == ref, (name, leaf_size, max_depth)
        nn = len(ref)
        # skip: first node whose range starts at or after this node's end
        firsts = np.array([r[0] for r in ref])
        for t in range(nn):
            end = ref[t][0] + ref[t][1]
            nxt = next((u for u in range(t + 1, nn) if firsts[u] >= end), nn)
            assert e["skip"][t] == nxt
        # parent: the deepest enclosing node
        for t in range(nn):
            s, c, l, _ = ref[t]
            cands = [u for u in range(nn) if ref[u][2] < l and ref[u][0] <= s and
                     s + c <= ref[u][0] + ref[u][1]]
            par = max(cands, key=lambda u: ref[u][2]) if cands else -1
            assert e["parent"][t] == par


def test_tree_invariants_scene():
    w = syn.workload("scene-200k", scale=0.05)
    c = w.cloud
    T = oracle.Tree(c.points, c.normals, c.areas, c.eps)
    e = T.export()
    n, nn = c.n, T.nn
    assert np.array_equal(np.sort(e["perm"]), np.arange(n, dtype=np.uint32))
    assert np.all(np.diff(e["code"].astype(np.int64)) >= 0)
    leaf = e["is_leaf"].astype(bool)
    cover = np.zeros(n, int)
    for t in np.nonzero(leaf)[0]:
        cover[e["first"][t]:e["first"][t] + e["count"][t]] += 1
        assert e["count"][t] <= 8 or e["level"][t] == 10
    assert np.all(cover == 1)
    for t in np.nonzero(~leaf)[0]:
        kids = []
        k = t + 1
        while k < e["skip"][t]:
            kids.append(k)
            assert e["parent"][k] == t
            k = e["skip"][k]
        assert len(kids) >= 2
        assert e["first"][kids[0]] == e["first"][t]
        assert sum(e["count"][k] for k in kids) == e["count"][t]
    # node geometry (eq. farfield_dipole)
    P = c.points[e["perm"]].astype(np.float64)
    A = c.areas[e["perm"]].astype(np.float64)
    rng = np.random.default_rng(0)
    for t in rng.choice(nn, 200, replace=False):
        s, k = e["first"][t], e["count"][t]
        a = A[s:s + k]
        cen = (a[:, None] * P[s:s + k]).sum(0) / a.sum()
        # leaves sum in float (the oracle's reading R7): a few float roundings of the exact sums
        assert abs(e["area"][t] - a.sum()) <= 1e-6 * a.sum()
        assert np.allclose(e["cen"][t], cen, rtol=0, atol=2e-6)
        d = np.linalg.norm(P[s:s + k] - e["cen32"][t].astype(np.float64), axis=1).max()
        assert abs(e["r32"][t] - d) <= 3e-7 * max(d, 1e-30)
    # R7 exactly: a leaf's area is its points' float sum in Morton order; an
    # internal node's is its children's areas added in double, in order
    A32 = c.areas[e["perm"]].astype(np.float32)
    for t in np.nonzero(leaf)[0][:300]:
        acc = np.float32(0.0)
        for m in range(e["first"][t], e["first"][t] + e["count"][t]):
            acc = np.float32(acc + A32[m])
        assert e["area"][t] == np.float64(acc)
    for t in np.nonzero(~leaf)[0][:300]:
        acc, k = 0.0, t + 1
        while k < e["skip"][t]:
            acc += e["area"][k]
            k = e["skip"][k]
        assert e["area"][t] == acc


def test_tree_rejects_bad_input():
    p = np.zeros((3, 3), np.float32)
    nrm = np.tile([0, 0, 1.0], (3, 1)).astype(np.float32)
    with pytest.raises(ValueError):
        oracle.Tree(p, nrm, np.array([1.0, 0.0, 1.0], np.float32))
    with pytest.raises(ValueError):
        oracle.Tree(p, nrm, np.ones(3, np.float32), leaf_size=0)
    with pytest.raises(ValueError):
        oracle.Tree(p, nrm, np.ones(3, np.float32), max_depth=11)
