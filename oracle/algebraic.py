"""Oracle: algebraic ordering for matrices without a grid (Section 2.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper partitions graph(A^T A) with a third-party nested dissection and
matches rows to columns with a third-party maximum-weight matching; its
interfaces follow the cited modified nested dissection, described only by
figures.  The readings here (the library implements the same ones in its own
code):

A1  Graph: columns i != j are adjacent when some row of A has entries in both.
A2  Nested dissection to depth L (complete binary tree, heap numbering, root
    0, children 2t+1 and 2t+2, level(t) = floor(log2(t+1)) + 1).  A node t
    with vertex set V (level < L):
      * r0 = the smallest id in V; a breadth-first search of the subgraph
        induced by V from r0 (neighbours visited in ascending id); u = the
        vertex of its last level with the smallest induced degree (ties: the
        smallest id); a second search from u gives the levels L_0..L_h of u's
        component C; vertices of V outside C come after L_h;
      * the separator is the first level L_j, j >= 1, whose prefix L_0..L_j
        holds at least half of V (none when h = 0: then S is empty, the
        left child gets V and the right child nothing);
      * separator vertices without a neighbour beyond L_j move to the left;
      * left child: L_0..L_{j-1} and the moved vertices; right child: the
        rest (levels beyond j and the other components).
    A node at level L keeps its whole set (an interior).  Every edge joins a
    node to itself, an ancestor or a descendant.
A3  Interfaces: at stage k a separator S (level l < k) splits into the sets
    of vertices with equal key_k(v) = { a_k(t) : t the node of a neighbour of
    v, t a proper descendant of S }, where a_k(t) = t when level(t) < k and
    the level-k ancestor of t otherwise (the whole subdomain below level k).
    key_{k-1} is the image of key_k under a_{k-1}, so every stage-k interface
    lies in one stage-(k-1) interface: the merge of Section 2.6.  On grids
    with the geometric tree this gives the geometric interfaces (pinned).
    Clusters of a stage are ordered by (node id, sorted key).
A4  Matching: a row-to-column matching of maximum sum of log|a_ij| (the
    objective of the maximum-product matching), computed by a library
    assignment routine; a matched row belongs to its column's cluster.
"""
from __future__ import annotations

import numpy as np

from .nd import Cluster


def node_level(t: int) -> int:
    return int(np.floor(np.log2(t + 1))) + 1


def column_graph(A) -> list[np.ndarray]:
    """A1: sorted neighbour arrays of graph(A^T A) without self loops."""
    import scipy.sparse as sp

    B = sp.csr_matrix(A)
    B.data = np.ones_like(B.data)
    G = (B.T @ B).tocsr()
    G.setdiag(0)
    G.eliminate_zeros()
    G.sort_indices()
    return [G.indices[G.indptr[i] : G.indptr[i + 1]].copy() for i in range(G.shape[0])]


def _bfs_levels(adj, inside, root):
    levels, seen = [[root]], {root}
    while True:
        nxt = []
        for v in levels[-1]:
            for w in adj[v]:
                w = int(w)
                if w in inside and w not in seen:
                    seen.add(w)
                    nxt.append(w)
        if not nxt:
            return levels
        nxt.sort()
        levels.append(nxt)


def _bisect(adj, V):
    """A2 for one node: (separator, left, right) as sorted lists."""
    inside = set(V)
    r0 = V[0]
    last = _bfs_levels(adj, inside, r0)[-1]
    deg = lambda v: sum(1 for w in adj[v] if int(w) in inside)
    u = min(last, key=lambda v: (deg(v), v))
    lev = _bfs_levels(adj, inside, u)
    if len(lev) == 1:
        return [], sorted(V), []
    reached = set(v for L in lev for v in L)
    others = sorted(v for v in V if v not in reached)
    half = len(V) / 2.0
    cum, j = 0, None
    for t, L in enumerate(lev):
        cum += len(L)
        if t >= 1 and cum >= half:
            j = t
            break
    if j is None:
        j = len(lev) - 1
    beyond = set(v for L in lev[j + 1 :] for v in L)
    sep, moved = [], []
    for v in lev[j]:
        (sep if any(int(w) in beyond for w in adj[v]) else moved).append(v)
    left = sorted([v for L in lev[:j] for v in L] + moved)
    right = sorted(list(beyond) + others)
    return sorted(sep), left, right


def nested_dissection(adj, depth: int) -> list[list[int]]:
    """A2: vertex sets of the 2^depth - 1 nodes (heap numbering)."""
    n = len(adj)
    nodes: list[list[int]] = [[] for _ in range(2**depth - 1)]
    work = {0: list(range(n))}
    for t in range(2**depth - 1):
        V = work.pop(t, [])
        if node_level(t) == depth or not V:
            nodes[t] = sorted(V)
            if node_level(t) < depth:
                work[2 * t + 1], work[2 * t + 2] = [], []
            continue
        s, a, b = _bisect(adj, V)
        nodes[t] = s
        work[2 * t + 1], work[2 * t + 2] = a, b
    return nodes


def _ancestor_at(t: int, level: int) -> int:
    while node_level(t) > level:
        t = (t - 1) // 2
    return t


def _is_proper_descendant(t: int, s: int) -> bool:
    while t > s:
        t = (t - 1) // 2
        if t == s:
            return True
    return False


class AlgebraicOrdering:
    """Clusters of every stage from A2/A3 (the oracle's counterpart of the
    geometric tree of oracle/nd.py, with the same Cluster records).

    A cluster label at stage k is (t, -1) for a node t whose whole subtree is
    one subdomain (level(t) >= k: its level-k ancestor) and (t, i) for the
    i-th interface of separator t (level(t) < k).  A separator vertex v's key
    at stage k is the sorted tuple of the labels of its neighbours in proper
    descendants of its node; the interfaces of a separator are ranked by key,
    deeper separators first, so every label is known when it is used."""

    def __init__(self, A, depth: int, nodes: list[list[int]] | None = None):
        self.adj = column_graph(A)
        self.L = depth
        self.nodes = nodes if nodes is not None else nested_dissection(self.adj, depth)
        n = len(self.adj)
        self.node_of = np.full(n, -1, dtype=np.int64)
        for t, V in enumerate(self.nodes):
            self.node_of[V] = t
        assert np.all(self.node_of >= 0), "vertex without a node"
        self._stages = {}
        for k in range(depth, 0, -1):
            self._stages[k] = self._build(k)

    def _build(self, k: int):
        """label[v] and key[v] of every vertex at stage k."""
        label, key = {}, {}
        order = sorted(range(len(self.nodes)), key=lambda t: (-node_level(t), t))
        for t in order:
            V = self.nodes[t]
            lv = node_level(t)
            if lv >= k:
                a = _ancestor_at(t, k)
                for v in V:
                    label[v] = (a, -1)
                continue
            for v in V:
                key[v] = tuple(sorted({label[int(w)] for w in self.adj[v]
                                       if _is_proper_descendant(int(self.node_of[w]), t)}))
            ranks = {kk: i for i, kk in enumerate(sorted({key[v] for v in V}))}
            for v in V:
                label[v] = (t, ranks[key[v]])
        return label, key

    def clusters_at_stage(self, k: int) -> list[Cluster]:
        label, key = self._stages[k]
        out = []
        for t, V in enumerate(self.nodes):
            lv = node_level(t)
            if lv > k or not V:
                continue
            if lv == k:
                out.append(Cluster(t, lv, (), np.array(V, dtype=np.int64)))
                continue
            groups = {}
            for v in V:
                groups.setdefault(key[v], []).append(v)
            for kk in sorted(groups):
                out.append(Cluster(t, lv, kk, np.array(sorted(groups[kk]), dtype=np.int64)))
        out.sort(key=lambda c: (c.node, c.key))
        return out

    def parent_key(self, key: tuple, k: int, node: int) -> tuple:
        """The stage-(k-1) key of the vertices of separator `node` whose stage-k
        key is `key`: the stage-(k-1) key of any one of them (A3 makes it the
        same for all).  Two separators can share a key, hence the node."""
        if node_level(node) >= k - 1:  # eliminated at stage k - 1: one cluster
            return ()
        kk = self._stages[k][1]
        if not hasattr(self, "_first"):
            self._first = {}
        idx = self._first.setdefault(k, {})
        if not idx:
            for v, x in kk.items():
                idx.setdefault((int(self.node_of[v]), x), v)
        return self._stages[k - 1][1][idx[(node, key)]]


def max_weight_matching(A) -> np.ndarray:
    """A4: match[j] = the row matched to column j, maximising sum log|a_ij|
    (scipy's sparse assignment on -log|a_ij| shifted positive)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import min_weight_full_bipartite_matching

    C = sp.csc_matrix(A).copy()
    C.data = np.abs(C.data)
    C.eliminate_zeros()
    logs = np.log(C.data)
    C.data = (logs.max() - logs) + 1.0  # positive costs; a constant shift keeps the optimum of a full matching
    Ct = C.T.tocsr()  # columns of A as the row side: every column gets a row
    cols, rows = min_weight_full_bipartite_matching(Ct)
    match = np.full(Ct.shape[0], -1, dtype=np.int64)
    match[np.asarray(cols)] = np.asarray(rows)
    return match
