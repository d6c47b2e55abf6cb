"""Pins of the oracle's nested dissection and interface hierarchy (no GPU).

Hand-derived facts for small grids under the readings stated in oracle/nd.py
(Section 2.2 and Fig. 2-3 of the paper describe the modified nested
dissection only by figures): box cuts, separator sizes, the separation
property of nested dissection, and the interface counts per stage of the
clustering hierarchy (Fig. 3(d)-(e) show a separator's interfaces merging
level by level).
"""
import numpy as np

from inputs.grid_ls import grid_problem
from oracle import nd


def test_tree_8x8_depth3_by_hand():
    nodes = nd.build_tree((8, 8, 1), 3)
    assert nodes[0].axis == 0 and nodes[0].mid == 4 and nodes[0].verts.size == 8
    assert nodes[1].hi == (4, 8, 1) and nodes[1].axis == 1 and nodes[1].mid == 4
    assert nodes[1].verts.size == 4 and nodes[2].verts.size == 3
    assert [nodes[i].verts.size for i in (3, 4, 5, 6)] == [16, 12, 12, 9]
    allv = np.concatenate([n.verts for n in nodes])
    assert np.array_equal(np.sort(allv), np.arange(64))


def _node_of(nodes, n):
    owner = np.full(n, -1)
    for nd_ in nodes:
        owner[nd_.verts] = nd_.id
    return owner


def _ancestors(i):
    out = set()
    while i > 0:
        i = (i - 1) // 2
        out.add(i)
    return out


def test_separation_property_2d_and_3d():
    for dims, depth in (((16, 16, 1), 5), ((8, 8, 8), 6), ((13, 7, 1), 4)):
        nodes = nd.build_tree(dims, depth)
        prob = grid_problem(*dims)
        owner = _node_of(nodes, prob.n)
        assert np.all(owner >= 0)
        A = prob.to_scipy()
        for r in range(prob.m):
            cols = A.indices[A.indptr[r] : A.indptr[r + 1]]
            if cols.size == 2:
                a, b = owner[cols[0]], owner[cols[1]]
                # an edge joins a node to itself, an ancestor or a descendant
                assert a == b or a in _ancestors(b) or b in _ancestors(a), (a, b)


def test_interfaces_8x8_by_hand():
    nodes = nd.build_tree((8, 8, 1), 3)
    keys = nd.finest_keys(nodes, (8, 8, 1), 3)
    st3 = nd.clusters_at_stage(nodes, keys, 3, 3)
    root = [c for c in st3 if c.node == 0]
    assert [c.verts.size for c in root] == [4, 1, 3]  # y<4, y=4, y>4
    assert [c.key for c in root] == [((1, -1), (2, -1)), ((1, 0), (2, 0)), ((1, 1), (2, 1))]
    assert len(st3) == 3 + 2 + 4
    st2 = nd.clusters_at_stage(nodes, keys, 3, 2)
    assert [(c.node, c.verts.size) for c in st2] == [(0, 8), (1, 4), (2, 3)]
    st1 = nd.clusters_at_stage(nodes, keys, 3, 1)
    assert [(c.node, c.verts.size) for c in st1] == [(0, 8)]


def test_interface_hierarchy_16x16():
    nodes = nd.build_tree((16, 16, 1), 5)
    keys = nd.finest_keys(nodes, (16, 16, 1), 5)
    counts = {}
    for k in (5, 4, 3, 2, 1):
        cl = nd.clusters_at_stage(nodes, keys, 5, k)
        counts[k] = [c.verts.size for c in cl if c.node == 0]
        # every stage partitions the live vertices exactly once
        live = np.concatenate([c.verts for c in cl])
        assert live.size == np.unique(live).size
    # root column x=8.  Level 2 cuts y=8 on both sides.  Level 3: the boxes
    # [0,8)x[0,8), [0,8)x[9,16), [9,16)x[9,16) cut x (parallel to the root)
    # but [9,16)x[0,8) (extents 7 x 8) cuts y=4.  Level 4 adds y=4 on the left
    # and y=12 on both sides.
    assert counts[5] == [4, 1, 3, 1, 3, 1, 3]
    assert counts[4] == [4, 1, 3, 1, 7]
    assert counts[3] == [8, 1, 7]
    assert counts[2] == [16] and counts[1] == [16]
    # merging: each stage-k cluster maps into exactly one stage-(k-1) cluster
    for k in (5, 4, 3, 2):
        child = nd.clusters_at_stage(nodes, keys, 5, k)
        par = {(c.node, c.key): c for c in nd.clusters_at_stage(nodes, keys, 5, k - 1)}
        for c in child:
            if c.level == k:
                continue
            P = par[(c.node, nd.parent_key(c.key, nodes, k))]
            assert set(c.verts.tolist()) <= set(P.verts.tolist())


def test_3d_interfaces_partition():
    dims = (8, 8, 8)
    nodes = nd.build_tree(dims, 6)
    keys = nd.finest_keys(nodes, dims, 6)
    for k in range(6, 0, -1):
        cl = nd.clusters_at_stage(nodes, keys, 6, k)
        live = np.concatenate([c.verts for c in cl])
        assert live.size == np.unique(live).size
        assert all(c.verts.size > 0 for c in cl)
    root = [c for c in nd.clusters_at_stage(nodes, keys, 6, 3) if c.node == 0]
    # at stage 3 only the level-2 cuts (y=4 on both sides) split the root plane x=4
    assert sum(c.verts.size for c in root) == 64 and len(root) == 3
