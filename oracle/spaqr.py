"""Oracle: the spaQR factorization (Algorithm 1) and W-preconditioned CGLS, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain and slow: Python
loops over clusters and row groups, numpy for the dense steps, no blocking,
fusion or reordering beyond what Algorithm 1 states.

The evolving matrix is held as *row groups*: rows that share an owner cluster
and a column support (a set of clusters).  A group keeps one dense block per
cluster of its support.  Readings of the paper used here (the paper leaves
these open):

R1  Column scaling (Section 2.7): D = diag(1 / ||A[:, j]||_2), A~ = A D.  The
    row heuristics run on A~ (Section 2.7 scales before it reorders rows).
R2  Rows (Section 2.2): a row matched to column v (the problem's matching,
    prob.match[v] = row, when it has one; otherwise the vertex row of v, which
    the max-norm rule sends to v's cluster anyway) belongs to v's cluster; every
    other row goes to argmax_c sum_{j in c} A~[r, j]^2, the candidates being
    the clusters it touches that belong to the deepest nested-dissection node
    among them (rows="tree", the default; rows="maxnorm" takes every touched
    cluster); ties go to the deeper cluster, then to the lower cluster id.
    The restriction keeps every row's support on one root-to-leaf chain of the
    tree, which is what Section 2.5.2's statement that disjoint subtrees stay
    disjoint requires.  Initial groups: rows sorted by (owner, support, row id).
R3  Group order: groups are numbered in creation order; a front stacks the
    eliminated cluster's own groups (by number) and then the other owners'
    groups touching it (by owner id, then number).  Front columns: s first,
    then the other clusters by id.
R4  Elimination (Section 2.3): after the Householder QR of the s columns the
    first c_s rows are R_s = [R_ss R_sn] (diag >= 0); the rows at positions
    r_s.. return to their owners (one new group per owner, in owner order);
    positions c_s..r_s-1 are the extra rows, each sent by the R2 rule to a
    cluster it touches (one new group per destination).  At the root
    they are dropped (all zero).
R5  Same-level eliminations run in rounds: each round takes, in ascending
    separator id, every separator whose front shares no row group with a
    separator already taken in that round (the paper loops over S_l
    sequentially and gives no order; eliminating s creates fill among the
    clusters of its front, which can couple two same-level separators).
R6  Scaling (Section 2.4) of every remaining interface p; p's rows become a
    group p1 (c_p rows, identity on p) and a group p2 (r_p - c_p rows, zero on
    p); every other row touching p gets X <- X R_pp^{-1}.
R7  Step 1 (Section 2.5.1) replaces p2 by the first k' rows of Q'^T A_{p2 n},
    each row signed so that its diagonal entry R_ii is >= 0 (the sign of a
    row of R is a free choice of the orthogonal factor Q'; the same
    convention as the front R factors, Section 2.3).
R8  Step 2 (Section 2.5.2): M_p = [A_np^T  A_{p1 n}]; coarse = the first k
    pivoted directions, fine = the last c_p - k slots of p; nothing happens
    when k = c_p.  Interfaces are processed by a greedy colouring (ascending
    id) of the graph p ~ q iff q is in the support of p's p1 group or vice
    versa; colour by colour.
R9  Scaling and sparsification run at stage k only when k <= L - skip
    (default skip 2: "skip sparsification for two levels", Section 4.2).
R10 W = W_1 ... W_L, W_l = (prod Q_p^T)(prod R_p)(prod R_s) for the
    operations of stage l (root stage 1 leftmost); W^{-1} replays the
    operations in reverse factorization order, W^{-T} in factorization order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import dense as dn
from . import nd


class RankDeficient(RuntimeError):
    pass


@dataclass
class Group:
    gid: int
    owner: int
    rows: int
    blocks: dict  # cluster id -> ndarray (rows x c_cluster)


@dataclass
class Op:
    kind: str  # "Rs", "Rp" or "Qp"
    stage: int
    slots: np.ndarray  # slots of s or p
    R: np.ndarray | None = None  # Rss or Rpp (upper triangular)
    Rn: np.ndarray | None = None  # Rsn
    nslots: np.ndarray | None = None  # slots of the R_sn columns
    V: np.ndarray | None = None  # Q_p reflectors (c_p x k)
    taus: np.ndarray | None = None
    color: int = 0


@dataclass
class Stats:
    fronts: list = field(default_factory=list)  # (stage, m, n, c)
    scale: list = field(default_factory=list)  # (stage, r_p, c_p)
    step1: list = field(default_factory=list)  # (stage, rows, cols, k')
    step2: list = field(default_factory=list)  # (stage, c_p, ncols, k)
    elim_rounds: list = field(default_factory=list)  # (stage, rounds)


def column_scaling(A: sp.csr_matrix):
    """R1: D with unit column norms; returns (D, A D)."""
    norms = np.sqrt(np.asarray(A.multiply(A).sum(axis=0)).ravel())
    if np.any(norms == 0.0):
        raise RankDeficient("zero column")
    D = 1.0 / norms
    return D, sp.csr_matrix(A @ sp.diags(D))


class GeometricOrdering:
    """The geometric nested dissection of a grid (oracle/nd.py readings)."""

    def __init__(self, dims, depth: int):
        self.dims, self.L = dims, depth
        self.nodes = nd.build_tree(dims, depth)
        self.keys = nd.finest_keys(self.nodes, dims, depth)

    def clusters_at_stage(self, k: int):
        return nd.clusters_at_stage(self.nodes, self.keys, self.L, k)

    def parent_key(self, key: tuple, k: int, node: int = -1) -> tuple:
        return nd.parent_key(key, self.nodes, k)


class OracleSpaQR:
    def __init__(self, prob, depth: int, eps: float, skip: int = 2, mode: str = "spaqr", rows: str = "tree",
                 within: str = "asc", ordering=None):
        # the clusters of every stage and their merge map: the geometric tree of
        # the grid (oracle/nd.py) unless an ordering (oracle/algebraic.py) is given
        self.ordering = ordering
        self.rows_rule = rows
        # Order inside one elimination round (R5) and one step-2 colour (R8):
        # "asc" (the reading) or "desc".  Members of a round or a colour are
        # independent, so both orders give identical results; tests use
        # "desc" to check that independence.
        self.within = within
        # Records for tests (no arithmetic): the owner cluster of every row at
        # the finest stage, and (stage, cluster, position, destination) of
        # every extra row sent on by the max-norm rule (R4).
        self.row_owner = None
        self.extra_dest = []
        self.prob = prob
        self.L = depth
        self.eps = eps
        self.skip = skip
        self.mode = mode
        self.ops: list[Op] = []
        self.stats = Stats()
        self.next_gid = 0

    # ------------------------------------------------------------ helpers
    def _new_group(self, owner, rows, blocks):
        g = Group(self.next_gid, owner, rows, blocks)
        self.next_gid += 1
        self.groups[g.gid] = g
        self._index(g)
        return g

    # Lookup tables only (no arithmetic): the groups each cluster owns and the
    # groups whose support contains each cluster.  A group's support changes
    # only at a merge, which rebuilds both tables.
    def _index(self, g):
        self.owned.setdefault(g.owner, set()).add(g.gid)
        for c in g.blocks:
            self.touch.setdefault(c, set()).add(g.gid)

    def _del_group(self, gid):
        g = self.groups.pop(gid)
        self.owned[g.owner].discard(gid)
        for c in g.blocks:
            self.touch[c].discard(gid)

    def _reindex(self):
        self.owned, self.touch = {}, {}
        for g in self.groups.values():
            self._index(g)

    def _owned_by(self, c):
        return sorted((self.groups[i] for i in self.owned.get(c, ())), key=lambda g: g.gid)

    def _touching(self, c):
        """Groups of other owners whose support contains c, by (owner, number)."""
        return sorted(
            (self.groups[i] for i in self.touch.get(c, ()) if self.groups[i].owner != c),
            key=lambda g: (g.owner, g.gid),
        )

    def _argmax_cluster(self, scores):
        """R2/R4 max-norm rule with the deeper-then-lower-id tie break."""
        best = None
        if self.rows_rule == "tree":
            deep = max(self.level[c] for c, _ in scores)
            scores = [(c, sc) for c, sc in scores if self.level[c] == deep]
        for cid, sc in scores:
            key = (sc, self.level[cid], -cid)
            if best is None or key > best[0]:
                best = (key, cid)
        return best[1]

    def _stack(self, glist, cols):
        widths = [self.slots[c].size for c in cols]
        offs = np.concatenate([[0], np.cumsum(widths)]).astype(int)
        m = sum(g.rows for g in glist)
        F = np.zeros((m, int(offs[-1])))
        r = 0
        for g in glist:
            for t, c in enumerate(cols):
                if c in g.blocks:
                    F[r : r + g.rows, offs[t] : offs[t + 1]] = g.blocks[c]
            r += g.rows
        return F, offs

    def _split(self, F, cols, offs):
        return {c: F[:, offs[t] : offs[t + 1]].copy() for t, c in enumerate(cols)}

    def _sparsify_here(self, k):
        return self.mode == "spaqr" and k <= self.L - self.skip and k >= 2

    # ------------------------------------------------------------ factor
    def factor(self):
        prob = self.prob
        A = prob.to_scipy()
        self.D, self.At = column_scaling(A)
        if self.ordering is None:
            self.ordering = GeometricOrdering(prob.dims, self.L)
        self._init_stage(self.L)
        for k in range(self.L, 0, -1):
            self.stage = k
            self._eliminate(k)
            if self._sparsify_here(k):
                self._scale(k)
                self._step1(k)
                self._step2(k)
            if k > 1:
                self._merge(k)
        assert not self.groups, "rows left after the root"
        return self

    def _init_stage(self, L):
        self.clusters = self.ordering.clusters_at_stage(L)
        nvert = self.prob.n
        cid_of = np.full(nvert, -1, dtype=np.int64)
        pos_in = np.zeros(nvert, dtype=np.int64)
        self.slots = {}
        self.level = {}
        for cid, c in enumerate(self.clusters):
            cid_of[c.verts] = cid
            pos_in[c.verts] = np.arange(c.verts.size)
            self.slots[cid] = c.verts.copy()
            self.level[cid] = c.level
        assert np.all(cid_of >= 0), "vertex without a cluster"
        self.alive = set(self.slots)
        At = self.At
        # R2: a row matched to column j belongs to j's cluster (the problem's
        # matching when it has one, else no row is matched explicitly)
        match = getattr(self.prob, "match", None)
        matched = {} if match is None else {int(match[j]): int(cid_of[j]) for j in range(nvert)}
        rows_by = {}
        self.row_owner = np.full(At.shape[0], -1, dtype=np.int64)
        for r in range(At.shape[0]):
            a, b = At.indptr[r], At.indptr[r + 1]
            cols = At.indices[a:b]
            vals = At.data[a:b]
            cls = cid_of[cols]
            support = tuple(sorted(set(cls.tolist())))
            if r in matched:
                owner = matched[r]
            else:
                scores = [(c, float(np.sum(vals[cls == c] ** 2))) for c in support]
                owner = self._argmax_cluster(scores)
            rows_by.setdefault((owner, support), []).append(r)
            self.row_owner[r] = owner
        self.groups, self.owned, self.touch = {}, {}, {}
        for (owner, support) in sorted(rows_by):
            rlist = rows_by[(owner, support)]
            blocks = {c: np.zeros((len(rlist), self.slots[c].size)) for c in support}
            for t, r in enumerate(rlist):
                a, b = At.indptr[r], At.indptr[r + 1]
                for j, v in zip(At.indices[a:b], At.data[a:b]):
                    blocks[int(cid_of[j])][t, pos_in[j]] += v
            self._new_group(owner, len(rlist), blocks)

    def _front_groups(self, s):
        return self._owned_by(s), self._touching(s)

    @staticmethod
    def _greedy_colour(items, conflicts):
        colour = {}
        for it in items:
            used = {colour[o] for o in conflicts[it] if o in colour}
            c = 0
            while c in used:
                c += 1
            colour[it] = c
        return colour

    def _eliminate(self, k):
        """R5: rounds of greedy maximal independent sets (ascending id) over
        the separators of level k still to be eliminated, recomputed on the
        current groups before every round (an elimination creates fill among
        the clusters of its front, which can couple two same-level separators)."""
        todo = sorted(c for c in self.alive if self.level[c] == k)
        rnd = 0
        while todo:
            taken, used, batch = set(), set(), []
            for s in todo:
                own, oth = self._front_groups(s)
                ids = {g.gid for g in own + oth}
                if ids & used:
                    continue
                used |= ids
                batch.append((s, own, oth))
            if self.within == "desc":
                batch = batch[::-1]
            for s, own, oth in batch:
                self._eliminate_one(k, s, own, oth, rnd)
                taken.add(s)
            todo = [s for s in todo if s not in taken]
            rnd += 1
        for c in [c for c in self.alive if self.level[c] == k]:
            self.alive.discard(c)
        self.stats.elim_rounds.append((k, rnd))

    def _eliminate_one(self, k, s, own, oth, col):
        cs = self.slots[s].size
        rs = sum(g.rows for g in own)
        fg = own + oth
        support = set()
        for g in fg:
            support |= set(g.blocks)
        cols = [s] + sorted(support - {s})
        F, offs = self._stack(fg, cols)
        m = F.shape[0]
        if rs < cs:
            raise RankDeficient(f"cluster {s}: {rs} rows < {cs} columns")
        dn.householder_qr(F, cs)
        dn.sign_fix_rows(F, cs)
        if cs and np.any(np.diag(F[:cs, :cs]) == 0.0):
            raise RankDeficient(f"cluster {s}: zero pivot")
        self.stats.fronts.append((k, m, F.shape[1], cs))
        rest = cols[1:]
        if cs > 0:  # a cluster whose slots were all dropped stores no factor
            self.ops.append(
                Op(
                    "Rs",
                    k,
                    self.slots[s].copy(),
                    R=np.triu(F[:cs, :cs]).copy(),
                    Rn=F[:cs, cs:].copy(),
                    nslots=np.concatenate([self.slots[c] for c in rest]) if rest else np.zeros(0, np.int64),
                    color=col,
                )
            )
        roffs = offs[1:] - offs[1]
        for g in fg:
            self._del_group(g.gid)
        # rows at positions r_s.. go back to their owners (R4)
        pos = rs
        owners = sorted({g.owner for g in oth})
        for o in owners:
            cnt = sum(g.rows for g in oth if g.owner == o)
            self._new_group(o, cnt, self._split(F[pos : pos + cnt, cs:], rest, roffs))
            pos += cnt
        # extra rows c_s..r_s-1 are reassigned by the max-norm rule (R4)
        if rest and rs > cs:
            dest = {}
            for i in range(cs, rs):
                scores = [
                    (c, float(np.sum(F[i, cs + roffs[t] : cs + roffs[t + 1]] ** 2)))
                    for t, c in enumerate(rest)
                ]
                c_to = self._argmax_cluster(scores)
                dest.setdefault(c_to, []).append(i)
                self.extra_dest.append((k, s, i, c_to))
            for c in sorted(dest):
                idx = dest[c]
                self._new_group(c, len(idx), self._split(F[idx, cs:], rest, roffs))

    def _scale(self, k):
        self.p1_of, self.p2_of = {}, {}
        for p in sorted(self.alive):
            cp = self.slots[p].size
            if cp == 0:
                continue
            own = self._owned_by(p)
            rp = sum(g.rows for g in own)
            if rp < cp:
                raise RankDeficient(f"interface {p}: {rp} rows < {cp} columns")
            support = set()
            for g in own:
                support |= set(g.blocks)
            cols = [p] + sorted(support - {p})
            F, offs = self._stack(own, cols)
            dn.householder_qr(F, cp)
            dn.sign_fix_rows(F, cp)
            Rpp = np.triu(F[:cp, :cp]).copy()
            if np.any(np.diag(Rpp) == 0.0):
                raise RankDeficient(f"interface {p}: singular A_pp")
            self.stats.scale.append((k, rp, cp))
            self.ops.append(Op("Rp", k, self.slots[p].copy(), R=Rpp))
            for g in own:
                self._del_group(g.gid)
            rest = cols[1:]
            roffs = offs[1:] - offs[1]
            b1 = self._split(F[:cp, cp:], rest, roffs)
            b1[p] = np.eye(cp)
            self.p1_of[p] = self._new_group(p, cp, b1).gid
            if rp > cp and rest:
                self.p2_of[p] = self._new_group(p, rp - cp, self._split(F[cp:, cp:], rest, roffs)).gid
            for g in self._touching(p):
                # X <- X R_pp^{-1}  (solve Y R_pp = X)
                g.blocks[p] = sla.solve_triangular(Rpp, g.blocks[p].T, trans="T", lower=False).T

    def _step1(self, k):
        for p in sorted(self.p2_of):
            g = self.groups[self.p2_of[p]]
            cols = sorted(g.blocks)
            X, offs = self._stack([g], cols)
            kk, Rrows = dn.qrcp_rows(X, self.eps, sign_fix=True)
            self.stats.step1.append((k, X.shape[0], X.shape[1], kk))
            if kk < g.rows:
                if kk == 0:
                    self._del_group(g.gid)
                    continue
                g.blocks = self._split(Rrows, cols, offs)
                g.rows = kk

    def _step2(self, k):
        ps = sorted(p for p in self.p1_of)
        p1 = {p: self.groups[self.p1_of[p]] for p in ps}
        conflicts = {
            p: [q for q in ps if q != p and (q in p1[p].blocks or p in p1[q].blocks)] for p in ps
        }
        colour = self._greedy_colour(ps, conflicts)
        ncol = max(colour.values()) + 1 if colour else 0
        for col in range(ncol):
            members = [q for q in ps if colour[q] == col]
            for p in (members[::-1] if self.within == "desc" else members):
                self._step2_one(k, p, p1[p], col)

    def _step2_one(self, k, p, g1, col):
        cp = self.slots[p].size
        nb = self._touching(p)
        Anp = np.vstack([g.blocks[p] for g in nb]) if nb else np.zeros((0, cp))
        ncols = sorted(c for c in g1.blocks if c != p)
        Ap1n = np.hstack([g1.blocks[c] for c in ncols]) if ncols else np.zeros((cp, 0))
        M = np.hstack([Anp.T, Ap1n])
        kk, _, _, V, taus = dn.qrcp(M, self.eps)
        self.stats.step2.append((k, cp, M.shape[1], kk))
        if kk == cp:
            return
        self.ops.append(Op("Qp", k, self.slots[p].copy(), V=V.copy(), taus=taus.copy(), color=col))
        for g in nb:
            g.blocks[p] = dn.apply_q_right(g.blocks[p], V, taus)[:, :kk]
        for c in ncols:
            g1.blocks[c] = dn.apply_qt_left(g1.blocks[c], V, taus)[:kk, :]
        g1.blocks[p] = np.eye(kk)
        g1.rows = kk
        self.slots[p] = self.slots[p][:kk]
        if kk == 0:
            self._del_group(g1.gid)

    def _merge(self, k):
        new = self.ordering.clusters_at_stage(k - 1)
        index = {(c.node, c.key): i for i, c in enumerate(new)}
        parent = {}
        for cid in sorted(self.alive):
            c = self.clusters[cid]
            parent[cid] = index[(c.node, self.ordering.parent_key(c.key, k, c.node))]
        children = {}
        for cid in sorted(self.alive):
            children.setdefault(parent[cid], []).append(cid)
        slots = {P: np.concatenate([self.slots[c] for c in ch]) for P, ch in children.items()}
        for g in self.groups.values():
            g.owner = parent[g.owner]
            nb = {}
            for P in sorted({parent[c] for c in g.blocks}):
                nb[P] = np.hstack(
                    [g.blocks[c] if c in g.blocks else np.zeros((g.rows, self.slots[c].size)) for c in children[P]]
                )
            g.blocks = nb
        self._reindex()
        self.clusters = new
        self.slots = slots
        self.level = {P: new[P].level for P in slots}
        self.alive = set(slots)

    # ------------------------------------------------------------ apply
    def apply_Winv(self, z: np.ndarray) -> np.ndarray:
        """W^{-1} z: operations in reverse factorization order (R10)."""
        z = np.array(z, dtype=np.float64, copy=True)
        vec = z.ndim == 1
        if vec:
            z = z[:, None]
        for op in reversed(self.ops):
            if op.kind == "Rs":
                y = z[op.slots] - op.Rn @ z[op.nslots]
                z[op.slots] = sla.solve_triangular(op.R, y, lower=False)
            elif op.kind == "Rp":
                z[op.slots] = sla.solve_triangular(op.R, z[op.slots], lower=False)
            else:
                z[op.slots] = dn.apply_q_left(z[op.slots], op.V, op.taus)
        return z[:, 0] if vec else z

    def apply_WinvT(self, z: np.ndarray) -> np.ndarray:
        """W^{-T} z: transposed operations in factorization order (R10)."""
        z = np.array(z, dtype=np.float64, copy=True)
        vec = z.ndim == 1
        if vec:
            z = z[:, None]
        for op in self.ops:
            if op.kind == "Rs":
                y = sla.solve_triangular(op.R, z[op.slots], trans="T", lower=False)
                z[op.slots] = y
                z[op.nslots] -= op.Rn.T @ y
            elif op.kind == "Rp":
                z[op.slots] = sla.solve_triangular(op.R, z[op.slots], trans="T", lower=False)
            else:
                z[op.slots] = dn.apply_qt_left(z[op.slots], op.V, op.taus)
        return z[:, 0] if vec else z

    def apply_W(self, z: np.ndarray) -> np.ndarray:
        """W z (for tests): inverse operations in factorization order."""
        z = np.array(z, dtype=np.float64, copy=True)
        vec = z.ndim == 1
        if vec:
            z = z[:, None]
        for op in self.ops:
            if op.kind == "Rs":
                z[op.slots] = op.R @ z[op.slots] + op.Rn @ z[op.nslots]
            elif op.kind == "Rp":
                z[op.slots] = op.R @ z[op.slots]
            else:
                z[op.slots] = dn.apply_qt_left(z[op.slots], op.V, op.taus)
        return z[:, 0] if vec else z

    def nnz_W(self) -> int:
        total = 0
        for op in self.ops:
            c = op.slots.size
            if op.kind == "Rs":
                total += c * (c + 1) // 2 + op.Rn.size
            elif op.kind == "Rp":
                total += c * (c + 1) // 2
            else:
                total += op.V.size
        return total

    # ------------------------------------------------------------ solve
    def solve(self, b: np.ndarray, tol: float = 1e-10, maxit: int = 500):
        """Right-preconditioned CGLS on min ||A~ W^{-1} y - b|| (Section 4);
        stops when ||A^T (A x - b)|| / ||A^T b|| < tol with the unscaled A."""
        At, D = self.At, self.D
        b = np.asarray(b, dtype=np.float64)
        n = At.shape[1]
        xt = np.zeros(n)
        r = b.copy()
        u = At.T @ r
        norm0 = float(np.linalg.norm(u / D))
        hist = [1.0]
        if norm0 == 0.0:
            return xt, dict(iters=0, rel=0.0, hist=hist)
        s = self.apply_WinvT(u)
        p = s.copy()
        gamma = float(s @ s)
        rel = 1.0
        it = 0
        for it in range(1, maxit + 1):
            t = self.apply_Winv(p)
            q = At @ t
            alpha = gamma / float(q @ q)
            xt += alpha * t
            r -= alpha * q
            u = At.T @ r
            rel = float(np.linalg.norm(u / D)) / norm0
            hist.append(rel)
            if rel < tol:
                break
            s = self.apply_WinvT(u)
            gamma_new = float(s @ s)
            beta = gamma_new / gamma
            gamma = gamma_new
            p = s + beta * p
        return D * xt, dict(iters=it, rel=rel, hist=hist, converged=rel < tol)

    def solve_csne(self, b: np.ndarray, tol: float = 1e-10, maxit: int = 100):
        """Corrected seminormal equations (Section 1, after Bjorck): W^T W
        xt = A~^T b, then refinement steps xt += W^{-1} W^{-T} A~^T (b - A~ xt)
        until ||A^T (A x - b)|| / ||A^T b|| < tol with the unscaled A.  With
        eps = 0 the first solve is exact up to rounding; with eps > 0 the
        refinement is a stationary iteration that converges when W^T W is
        close enough to A~^T A~."""
        At, D = self.At, self.D
        b = np.asarray(b, dtype=np.float64)
        xt = np.zeros(At.shape[1])
        r = b.copy()
        norm0 = float(np.linalg.norm((At.T @ b) / D))
        hist = [1.0]
        if norm0 == 0.0:
            return xt, dict(iters=0, rel=0.0, hist=hist, converged=True)
        rel, it = 1.0, 0
        for it in range(1, maxit + 1):
            xt += self.apply_Winv(self.apply_WinvT(At.T @ r))
            r = b - At @ xt
            rel = float(np.linalg.norm((At.T @ r) / D)) / norm0
            hist.append(rel)
            if rel < tol:
                break
        return D * xt, dict(iters=it, rel=rel, hist=hist, converged=rel < tol)


def solve_diag_cgls(prob, b: np.ndarray, tol: float = 1e-10, maxit: int = 100000):
    """The paper's "Diag." comparator (Section 4): CGLS preconditioned by the
    diagonal of A^T A only, i.e. CGLS on A~ = A D with D the column scaling
    (R1) and no W; same stopping rule as OracleSpaQR.solve."""
    A = prob.to_scipy()
    D, At = column_scaling(A)
    b = np.asarray(b, dtype=np.float64)
    xt = np.zeros(At.shape[1])
    r = b.copy()
    s = At.T @ r
    norm0 = float(np.linalg.norm(s / D))
    hist = [1.0]
    if norm0 == 0.0:
        return xt, dict(iters=0, rel=0.0, hist=hist, converged=True)
    p = s.copy()
    gamma = float(s @ s)
    rel, it = 1.0, 0
    for it in range(1, maxit + 1):
        q = At @ p
        alpha = gamma / float(q @ q)
        xt += alpha * p
        r -= alpha * q
        s = At.T @ r
        rel = float(np.linalg.norm(s / D)) / norm0
        hist.append(rel)
        if rel < tol:
            break
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return D * xt, dict(iters=it, rel=rel, hist=hist, converged=rel < tol)
