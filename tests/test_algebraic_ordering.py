"""Algebraic ordering for matrices without a grid (Section 2.2, no GPU).

Oracle pins (oracle/algebraic.py):
* nested dissection by level structures, hand-derived on a path graph;
* the nested-dissection separation property and the partition of the
  vertices on irregular k-nearest-neighbour graphs;
* the interface construction reduces to the geometric one: fed the geometric
  tree of a 2D or 3D grid it yields the geometric interfaces of every stage
  (oracle/nd.py), and its merge map nests the interfaces the same way;
* the maximum-weight matching against brute force over all matchings of
  small matrices.
Library parity (host-only C ABI, exact integer work): spaqr_analyze_matrix
gives the oracle's clusters and merge map at every stage; spaqr_match returns
a valid matching with the oracle's optimal objective (the optimum is often
not unique: an edge row has the same |w| in both of its columns), and refuses
a structurally rank-deficient matrix.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from inputs.grid_ls import grid_problem
from inputs.irregular import knn_problem
from oracle.algebraic import AlgebraicOrdering, column_graph, max_weight_matching, nested_dissection, node_level
from oracle.spaqr import GeometricOrdering


def test_nested_dissection_of_a_path_by_hand():
    # path 0-1-2-3-4-5-6: the first search from 0 ends at 6 (degree 1), the second
    # from 6 has levels {6},{5},...,{0}; the prefix {6,5,4,3} is the first to hold
    # half of the 7 vertices, so {3} separates, the left child takes {4,5,6}
    A = sp.csr_matrix(np.array([[1.0 if j in (i, i + 1) else 0.0 for j in range(7)] for i in range(6)] + [np.eye(7)[0]]))
    nodes = nested_dissection(column_graph(A), 2)
    assert nodes == [[3], [4, 5, 6], [0, 1, 2]]
    nodes3 = nested_dissection(column_graph(A), 3)
    # {4,5,6}: search from 4 ends at 6, from 6: {6},{5},{4} -> separator {5}; {0,1,2} likewise -> {1}
    assert nodes3[:3] == [[3], [5], [1]] and nodes3[3:] == [[6], [4], [2], [0]]


def _ancestors(t):
    out = set()
    while t > 0:
        t = (t - 1) // 2
        out.add(t)
    return out


@pytest.mark.parametrize("n,k,depth,seed", [(300, 4, 5, 0), (2000, 6, 8, 1), (1500, 3, 7, 2)])
def test_separation_and_partition(n, k, depth, seed):
    p = knn_problem(n, k=k, seed=seed)
    A = p.to_scipy()
    adj = column_graph(A)
    nodes = nested_dissection(adj, depth)
    owner = np.full(n, -1)
    for t, V in enumerate(nodes):
        assert np.all(owner[V] == -1)
        owner[V] = t
    assert np.all(owner >= 0)
    for v in range(n):
        for w in adj[v]:
            a, b = owner[v], owner[int(w)]
            assert a == b or a in _ancestors(b) or b in _ancestors(a)
    # a usable tree: no leaf holds more than eight times an even share
    assert max(len(V) for t, V in enumerate(nodes) if node_level(t) == depth) < 8 * n / 2 ** (depth - 1)


@pytest.mark.parametrize("dims,depth", [((16, 16, 1), 5), ((13, 7, 1), 4), ((8, 8, 8), 6), ((12, 10, 6), 7)])
def test_interfaces_reduce_to_the_geometric_ones(dims, depth):
    p = grid_problem(*dims)
    geo = GeometricOrdering(dims, depth)
    alg = AlgebraicOrdering(p.to_scipy(), depth, nodes=[list(map(int, nd.verts)) for nd in geo.nodes])
    for k in range(depth, 0, -1):
        G = geo.clusters_at_stage(k)
        Al = alg.clusters_at_stage(k)
        assert sorted((c.node, tuple(c.verts)) for c in G) == sorted((c.node, tuple(c.verts)) for c in Al)
        if k > 1:  # the merge maps agree: parents hold the same vertex sets
            Gp = {(c.node, c.key): tuple(c.verts) for c in geo.clusters_at_stage(k - 1)}
            Ap = {(c.node, c.key): tuple(c.verts) for c in alg.clusters_at_stage(k - 1)}
            pg = {tuple(c.verts): Gp[(c.node, geo.parent_key(c.key, k))] for c in G if c.level < k}
            pa = {tuple(c.verts): Ap[(c.node, alg.parent_key(c.key, k, c.node))] for c in Al if c.level < k}
            assert pg == pa


def test_matching_is_the_brute_force_optimum():
    rng = np.random.default_rng(7)
    for trial in range(30):
        n = int(rng.integers(2, 6))
        m = n + int(rng.integers(0, 3))
        M = rng.uniform(0.1, 3.0, size=(m, n)) * (rng.random((m, n)) < 0.6)
        for j in range(n):  # a structurally full-rank pattern
            M[j, j] = rng.uniform(0.1, 3.0)
        A = sp.csr_matrix(M)
        mt = max_weight_matching(A)
        assert len(set(mt.tolist())) == n and all(M[mt[j], j] != 0 for j in range(n))
        best = max(sum(np.log(M[r[j], j]) for j in range(n)) for r in itertools.permutations(range(m), n)
                   if all(M[r[j], j] != 0 for j in range(n)))
        assert abs(sum(np.log(M[mt[j], j]) for j in range(n)) - best) < 1e-12


def _lib_stage(an, k):
    node, level, vptr, verts = an.stage_clusters(k)
    return [(int(node[c]), tuple(int(v) for v in verts[vptr[c] : vptr[c + 1]])) for c in range(len(node))]


@pytest.mark.parametrize(
    "prob,depth",
    [(knn_problem(300, seed=1), 5), (knn_problem(5000, k=6, law="c2", seed=3), 9), (knn_problem(20000, seed=4), 11),
     (grid_problem(8, 8, 8), 6), (grid_problem(13, 7, 1), 4)],
)
def test_library_analysis_matches_oracle(prob, depth):
    import paper_2102_09878_gb300 as sq

    an = sq.Analysis.from_matrix(prob, depth)
    o = AlgebraicOrdering(prob.to_scipy(), depth)
    for k in range(1, depth + 1):
        assert _lib_stage(an, k) == [(c.node, tuple(int(v) for v in c.verts)) for c in o.clusters_at_stage(k)]


@pytest.mark.parametrize("prob,depth", [(knn_problem(2000, k=6, seed=1), 8), (knn_problem(3000, k=4, law="c2", seed=2), 9)])
def test_merge_map_is_containment(prob, depth):
    """The oracle's merge map (parent_key) sends every stage-k interface to the
    stage-(k-1) interface of the same separator that contains its vertices."""
    o = AlgebraicOrdering(prob.to_scipy(), depth)
    for k in range(depth, 1, -1):
        nxt = o.clusters_at_stage(k - 1)
        where = {}
        for i, c in enumerate(nxt):
            for v in c.verts:
                where[int(v)] = i
        index = {(c.node, c.key): i for i, c in enumerate(nxt)}
        for c in o.clusters_at_stage(k):
            if c.level >= k:
                continue
            i = index[(c.node, o.parent_key(c.key, k, c.node))]
            assert all(where[int(v)] == i for v in c.verts)


@pytest.mark.parametrize("prob", [knn_problem(300, seed=1), knn_problem(5000, k=6, law="c2", seed=3),
                                  grid_problem(16, 16, 1)])
def test_library_matching_is_optimal(prob):
    import paper_2102_09878_gb300 as sq

    A = prob.to_scipy().tocsr()
    ml = sq.match(prob)
    assert len(set(ml.tolist())) == prob.n and all(A[int(ml[j]), j] != 0 for j in range(prob.n))
    mo = max_weight_matching(A)
    w = lambda mt: sum(np.log(abs(A[int(mt[j]), j])) for j in range(prob.n))
    assert abs(w(ml) - w(mo)) <= 1e-12 * abs(w(mo))


def test_library_matching_refuses_structural_rank_deficiency():
    import paper_2102_09878_gb300 as sq

    # two columns that only one row touches
    M = np.array([[1.0, 2.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.0, 3.0]])

    class P:
        m, n = 3, 3
        rowptr = sp.csr_matrix(M).indptr
        colidx = sp.csr_matrix(M).indices
        vals = sp.csr_matrix(M).data

    with pytest.raises(sq.SpaqrError) as ei:
        sq.match(P)
    assert ei.value.code == sq.capi.SPAQR_ERR_RANK_DEFICIENT


def test_oracle_factor_with_algebraic_ordering_is_exact_at_eps0():
    """Algorithm 1 over the algebraic ordering of an irregular matrix with its
    maximum-weight matching: at eps = 0 W^T W = A~^T A~ (Section 2.7) and
    CGLS stops at once on the normal-equation solution; at eps > 0 it converges."""
    import scipy.sparse.linalg as spla

    from oracle.spaqr import OracleSpaQR

    p = knn_problem(600, k=5, seed=5)
    A = p.to_scipy()
    p.match = max_weight_matching(A)
    o = OracleSpaQR(p, 6, 0.0, ordering=AlgebraicOrdering(A, 6)).factor()
    W = o.apply_W(np.eye(p.n))
    AtA = (o.At.T @ o.At).toarray()
    assert np.linalg.norm(W.T @ W - AtA) <= 1e-12 * np.linalg.norm(AtA)
    x, info = o.solve(p.b)
    xr = spla.spsolve((A.T @ A).tocsc(), A.T @ p.b)
    assert info["iters"] <= 2 and np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)
    o2 = OracleSpaQR(p, 6, 1e-3, ordering=AlgebraicOrdering(A, 6)).factor()
    x2, info2 = o2.solve(p.b)
    assert info2["converged"] and np.linalg.norm(x2 - xr) <= 1e-8 * np.linalg.norm(xr)
    assert sum(op.kind == "Qp" for op in o2.ops) > 0
