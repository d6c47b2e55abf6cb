"""Oracle: geometric nested dissection, interfaces and the clustering hierarchy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package; only tests/, the smoke check and the benchmark's CPU-baseline leg do.

Follows Section 2.2 of the paper (vertex separators by nested dissection on
graph(A^T A) -- for grids, "regular geometric partitioning" (Section 4.1) --
then interfaces by the modified nested dissection, Fig. 2-3, and the cluster
hierarchy merged level by level, Section 2.6).  The paper fixes neither the
cut rule nor the interface rule for grids; the readings taken here are:

* Tree: a complete binary tree of depth L in heap numbering (root 0, children
  2i+1 and 2i+2, level(i) = floor(log2(i+1)) + 1, leaves at level L).  A
  node's box is half-open [lo, hi) per axis.  A non-leaf node cuts its
  longest axis (ties to the lowest axis index, x < y < z) at
  mid = (lo + hi) // 2; its separator is the plane {v_axis = mid} inside the
  box and its children are [lo, mid) and [mid + 1, hi) on that axis.  An empty
  box has an empty separator and empty children.  A leaf's vertex set is its
  whole box (an interior).
* Interfaces: a separator S splits into interfaces at stage k (while the
  level-k separators are eliminated).  For a vertex v of S the key is the
  sorted list of pairs (D, sign(v[axis_D] - mid_D)) over the descendants D of
  S with level(S) < level(D) < k whose cut axis differs from S's and whose box,
  widened by one vertex on every side, contains v.  Vertices with equal keys
  form one interface.  Merging after stage k drops the pairs of level k-1.
* Cluster numbering at stage k: clusters are ordered by (node id, key) with
  Python's lexicographic order on the key lists; a cluster's slots are its
  vertex ids in ascending order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Node:
    id: int
    level: int
    lo: tuple
    hi: tuple
    axis: int = -1
    mid: int = -1
    verts: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))

    def empty(self) -> bool:
        return any(h <= l for l, h in zip(self.lo, self.hi))


def node_level(i: int) -> int:
    return int(np.floor(np.log2(i + 1))) + 1


def build_tree(dims, depth: int) -> list[Node]:
    """Geometric nested dissection of the nx*ny*nz grid to the given depth."""
    nx, ny, nz = dims
    vid = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    nnodes = 2**depth - 1
    nodes: list[Node | None] = [None] * nnodes
    nodes[0] = Node(0, 1, (0, 0, 0), (nx, ny, nz))
    for i in range(nnodes):
        nd = nodes[i]
        lo, hi = nd.lo, nd.hi
        if nd.level == depth:
            if not nd.empty():
                nd.verts = np.sort(vid[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].ravel())
            continue
        ext = [h - l for l, h in zip(lo, hi)]
        if nd.empty():
            nd.axis, nd.mid = 0, lo[0]
            for c in (2 * i + 1, 2 * i + 2):
                nodes[c] = Node(c, nd.level + 1, lo, lo)
            continue
        a = int(np.argmax(ext))  # first maximum = lowest axis on ties
        mid = (lo[a] + hi[a]) // 2
        nd.axis, nd.mid = a, mid
        slo, shi = list(lo), list(hi)
        slo[a], shi[a] = mid, mid + 1
        nd.verts = np.sort(vid[slo[2]:shi[2], slo[1]:shi[1], slo[0]:shi[0]].ravel())
        left_hi = list(hi)
        left_hi[a] = mid
        right_lo = list(lo)
        right_lo[a] = mid + 1
        nodes[2 * i + 1] = Node(2 * i + 1, nd.level + 1, lo, tuple(left_hi))
        nodes[2 * i + 2] = Node(2 * i + 2, nd.level + 1, tuple(right_lo), hi)
    return nodes  # type: ignore[return-value]


def vertex_coords(dims, verts: np.ndarray) -> np.ndarray:
    nx, ny, _ = dims
    return np.stack([verts % nx, (verts // nx) % ny, verts // (nx * ny)], axis=1)


def finest_keys(nodes: list[Node], dims, depth: int) -> dict[int, list[list[tuple]]]:
    """For every non-leaf separator S, per vertex (in S.verts order) the list of
    (level_D, D, sign) over every descendant D that applies (any level)."""
    keys: dict[int, list[list[tuple]]] = {}
    nnodes = len(nodes)
    for s in nodes:
        if s.level == depth or s.verts.size == 0:
            continue
        xyz = vertex_coords(dims, s.verts)
        per_v: list[list[tuple]] = [[] for _ in range(s.verts.size)]
        stack = [2 * s.id + 1, 2 * s.id + 2]
        while stack:
            d = stack.pop()
            if d >= nnodes:
                continue
            dn = nodes[d]
            if dn.empty():
                continue
            inside = np.ones(s.verts.size, dtype=bool)
            for b in range(3):
                inside &= (xyz[:, b] >= dn.lo[b] - 1) & (xyz[:, b] <= dn.hi[b])
            if not inside.any():
                continue  # no descendant of d can apply either
            if dn.level < depth and dn.axis != s.axis:
                sg = np.sign(xyz[:, dn.axis] - dn.mid).astype(int)
                for t in np.nonzero(inside)[0]:
                    per_v[t].append((dn.level, d, int(sg[t])))
            stack.extend([2 * d + 1, 2 * d + 2])
        keys[s.id] = per_v
    return keys


@dataclass
class Cluster:
    """One cluster (interface or whole separator) at a given stage."""
    node: int
    level: int
    key: tuple
    verts: np.ndarray  # ascending vertex ids


def clusters_at_stage(nodes: list[Node], keys, depth: int, k: int) -> list[Cluster]:
    """Clusters alive at stage k, in canonical order (node id, key)."""
    out: list[Cluster] = []
    for nd in nodes:
        if nd.level > k or nd.verts.size == 0:
            continue
        if nd.level == k:
            out.append(Cluster(nd.id, nd.level, (), nd.verts))
            continue
        per_v = keys[nd.id]
        groups: dict[tuple, list[int]] = {}
        for t, lst in enumerate(per_v):
            key = tuple(sorted((d, sg) for (lv, d, sg) in lst if lv < k))
            groups.setdefault(key, []).append(int(nd.verts[t]))
        for key in sorted(groups):
            out.append(Cluster(nd.id, nd.level, key, np.array(sorted(groups[key]), dtype=np.int64)))
    out.sort(key=lambda c: (c.node, c.key))
    return out


def parent_key(key: tuple, nodes: list[Node], k: int) -> tuple:
    """Key of the stage-(k-1) parent of a stage-k cluster: drop level k-1 pairs."""
    return tuple((d, sg) for (d, sg) in key if nodes[d].level < k - 1)
