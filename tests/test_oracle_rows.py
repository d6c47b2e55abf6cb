"""Pins of the oracle's row rule, its orders and its W applies (no GPU).

* The max-norm row rule (Section 2.2; the rule for extra rows of Section
  2.3): a row goes to argmax_c sum_{j in c} A~[r, j]^2 over its candidate
  clusters, ties to the deeper cluster and then to the lower cluster id.  On a
  4 x 4 grid with planted values every score is a ratio of small integers,
  so the owner of every row and the destination of the extra rows of one
  front are derived by hand below, for the "tree" candidates (the clusters of
  the deepest nested-dissection node the row touches) and for the literal
  "maxnorm" candidates (every touched cluster).  An argmin, a flipped tie
  break or a shallowest-node filter changes several entries.
* The same-level rounds and the step-2 colours (Algorithm 1 loops over
  separators and interfaces one at a time without fixing an order): members
  of one round or one colour are independent, so processing them in reverse
  order gives the same factor up to rounding; a round or colouring that lets
  two coupled members share a batch does not.
* The greedy colouring itself on small graphs coloured by hand.
* W^{-1} W = I and W^{-T} = (W^{-1})^T as dense matrices at eps > 0 (Section
  2.7: W is a product of triangular and orthogonal factors), which pins the
  Q_p branch of both applies against the independent W product.
"""
import numpy as np
import pytest

from inputs.grid_ls import grid_problem
from oracle import dense as dn
from oracle.spaqr import OracleSpaQR


def planted_4x4():
    """4 x 4 grid, every edge weight 1, every vertex weight 1 except d_1 = d_9 = 3.

    Squared column norms (degree + d^2): vertex 0: 3, 1: 12, 2: 4, 3: 3, 4: 4,
    5: 5, 6: 5, 7: 4, 8: 4, 9: 13, 10: 5, 11: 4, 12: 3, 13: 4, 14: 4, 15: 3.
    An edge row (u, v) of the scaled matrix has the score 1 / |A_:u|^2 at u's
    cluster and 1 / |A_:v|^2 at v's, so it goes to the endpoint with the
    smaller column norm; equal norms are exact ties.
    """
    p = grid_problem(4, 4, 1, "u12", 0)
    ne = p.m - p.n
    p.vals[0 : 2 * ne : 2] = 1.0
    p.vals[1 : 2 * ne : 2] = -1.0
    d = np.ones(16)
    d[1] = d[9] = 3.0
    p.vals[2 * ne :] = d
    return p


# Depth 3 on the 4 x 4 grid (oracle/nd.py readings): the root cuts x at 2
# (vertices 2, 6, 10, 14); node 1 (x < 2) cuts y at 2 (8, 9); node 2 (x = 3)
# cuts y at 2 (11); leaves 3: {0, 1, 4, 5}, 4: {12, 13}, 5: {3, 7}, 6: {15}.
# At the finest stage the root splits by the side of the two level-2 cuts:
# cluster 0 = {2, 6} (y < 2), 1 = {10} (y = 2), 2 = {14} (y > 2); then
# 3 = node 1, 4 = node 2, 5..8 = the leaves.  Levels: 0-2 -> 1, 3-4 -> 2,
# 5-8 -> 3.  Rows: x-edges (0,1) (1,2) (2,3) (4,5) (5,6) (6,7) (8,9) (9,10)
# (10,11) (12,13) (13,14) (14,15), then y-edges (0,4) (1,5) (2,6) (3,7) (4,8)
# (5,9) (6,10) (7,11) (8,12) (9,13) (10,14) (11,15), then vertex rows 0..15.
VERTEX_ROWS = [5, 5, 0, 7, 5, 5, 0, 7, 3, 3, 1, 4, 6, 6, 2, 8]

# Tree candidates: an edge between clusters of different levels goes to the
# deeper one whatever the scores; only (6,10) and (10,14) join two clusters of
# the root: (6,10) ties at 1/5 : 1/5 -> the lower id 0; (10,14) 1/5 : 1/4 -> 2.
TREE_EDGE_ROWS = [5, 5, 7, 5, 5, 7, 3, 3, 4, 6, 6, 8, 5, 5, 0, 7, 5, 5, 0, 7, 6, 6, 2, 8]

# Every touched cluster a candidate: (1,2) 1/12 : 1/4 -> 0; (2,3) 1/4 : 1/3 -> 7;
# (5,6) tie -> deeper 5; (6,7) 1/5 : 1/4 -> 7; (9,10) 1/13 : 1/5 -> 1;
# (10,11) 1/5 : 1/4 -> 4; (13,14) tie -> deeper 6; (14,15) 1/4 : 1/3 -> 8;
# (4,8) tie -> deeper 5; (5,9) 1/5 : 1/13 -> 5; (6,10) tie, same level -> 0;
# (7,11) tie -> deeper 7; (8,12) 1/4 : 1/3 -> 6; (9,13) 1/13 : 1/4 -> 6;
# (10,14) 1/5 : 1/4 -> 2; (11,15) 1/4 : 1/3 -> 8.
MAXNORM_EDGE_ROWS = [5, 0, 7, 5, 5, 7, 3, 1, 4, 6, 6, 8, 5, 5, 0, 7, 5, 5, 0, 7, 6, 6, 2, 8]


@pytest.mark.parametrize("rule,edges", [("tree", TREE_EDGE_ROWS), ("maxnorm", MAXNORM_EDGE_ROWS)])
def test_row_owners_by_hand(rule, edges):
    o = OracleSpaQR(planted_4x4(), 3, 0.0, rows=rule).factor()
    assert o.row_owner.tolist() == edges + VERTEX_ROWS


def test_extra_row_destinations_by_hand():
    """The front of leaf {15} (cluster 8): rows (14,15), (11,15) and the vertex
    row of 15, in that order (groups by (owner, support)); columns 15, 14, 11.
    With a = 1/sqrt(3) (D_15) and D_14 = D_11 = 1/2 it is
        [-a 1/2 0; -a 0 1/2; a 0 0].
    The reflector of x = (-a, -a, a) has beta = +1, tau = 1 + a,
    v = (1, a/(1+a), -a/(1+a)); H e_1 = x and H e_2 = e_2 - a v.  The extra
    rows (positions 1, 2) are then, on columns (14 | 11):
        row 1: (-a/2 | (1 - a^2/(1+a))/2) = (-0.2887 | 0.3943)
        row 2: ( a/2 | a^2/(2(1+a)))     = ( 0.2887 | 0.1057)
    Scores at cluster 2 ({14}) and 4 ({11}): row 1 1/12 : 0.1555 -> 4,
    row 2 1/12 : 0.0112 -> 2.  Tree candidates keep only the deeper cluster 4
    (level 2 against the root's level 1): both rows -> 4."""
    for rule, want in (("maxnorm", [(1, 4), (2, 2)]), ("tree", [(1, 4), (2, 4)])):
        o = OracleSpaQR(planted_4x4(), 3, 0.0, rows=rule).factor()
        got = [(i, c) for (k, s, i, c) in o.extra_dest if k == 3 and s == 8]
        assert got == want, (rule, got)


def test_greedy_colouring_by_hand():
    col = OracleSpaQR._greedy_colour
    # 5-cycle 0-1-2-3-4-0: 0, 1, 0, 1, then 4 sees 0 and 1 -> 2
    cyc = {0: [1, 4], 1: [0, 2], 2: [1, 3], 3: [2, 4], 4: [3, 0]}
    assert col([0, 1, 2, 3, 4], cyc) == {0: 0, 1: 1, 2: 0, 3: 1, 4: 2}
    # star with centre 3 and a pendant edge 1-2: 0 -> 0, 1 -> 0, 2 (sees 1) -> 1,
    # 3 (sees 0, 1, 2 with colours 0, 0, 1) -> 2, 4 (sees 3) -> 0
    star = {0: [3], 1: [3, 2], 2: [3, 1], 3: [0, 1, 2, 4], 4: [3]}
    assert col([0, 1, 2, 3, 4], star) == {0: 0, 1: 0, 2: 1, 3: 2, 4: 0}
    # no edges: one colour; the visiting order decides, not the labels
    assert col([7, 3, 5], {7: [], 3: [], 5: []}) == {7: 0, 3: 0, 5: 0}
    assert col([2, 1], {2: [1], 1: [2]}) == {2: 0, 1: 1}


def _op_key(op):
    return (op.kind, op.stage, tuple(np.sort(op.slots).tolist()))


def _max_rel_diff(a, b):
    A = {_op_key(o): o for o in a.ops}
    B = {_op_key(o): o for o in b.ops}
    assert A.keys() == B.keys() and len(A) == len(a.ops)
    worst = 0.0
    for k, x in A.items():
        y = B[k]
        assert np.array_equal(x.slots, y.slots)
        if x.kind == "Qp":
            c = x.slots.size
            qx = dn.apply_q_left(np.eye(c), x.V, x.taus)
            qy = dn.apply_q_left(np.eye(c), y.V, y.taus)
            worst = max(worst, float(np.abs(qx - qy).max()))
            continue
        for f in ("R", "Rn"):
            u, v = getattr(x, f), getattr(y, f)
            if u is not None and u.size:
                worst = max(worst, float(np.abs(u - v).max() / np.abs(u).max()))
    return worst


@pytest.mark.parametrize(
    "dims,depth,law,rule,eps",
    [((32, 32, 1), 5, "c3", "maxnorm", 1e-2), ((8, 8, 8), 6, "u12", "maxnorm", 1e-3), ((64, 64, 1), 6, "u12", "tree", 1e-2)],
)
def test_rounds_and_colours_are_independent(dims, depth, law, rule, eps):
    """Reversing the order inside every elimination round and every step-2
    colour leaves every stored op unchanged up to rounding.  The first two
    cases have stages of two and three rounds and colours with several Q_p
    ops; putting every interface in one colour makes the 32 x 32 case differ
    by O(1), and one round per stage reuses consumed row groups."""
    p = grid_problem(*dims, law, 0)
    a = OracleSpaQR(p, depth, eps, rows=rule).factor()
    b = OracleSpaQR(p, depth, eps, rows=rule, within="desc").factor()
    if rule == "maxnorm":
        assert max(r for _, r in a.stats.elim_rounds) >= 2
    assert _max_rel_diff(a, b) < 1e-11


def test_winv_inverts_w_and_transpose_at_eps_positive():
    """On 64 x 64 at eps = 1e-2 (many Q_p ops): W^{-1} (W I) = I and the dense
    W^{-T} equals the transpose of the dense W^{-1}.  apply_W multiplies by
    the stored factors, the inverse applies solve with them, so a wrong
    reflector order or a Q in place of Q^T in either inverse apply fails."""
    p = grid_problem(64, 64, 1, "u12", 0)
    o = OracleSpaQR(p, 6, 1e-2).factor()
    assert sum(op.kind == "Qp" for op in o.ops) >= 5
    n = p.n
    eye = np.eye(n)
    W = o.apply_W(eye)
    Wi = o.apply_Winv(eye)
    WiT = o.apply_WinvT(eye)
    assert np.abs(o.apply_Winv(W) - eye).max() < 1e-9
    assert np.abs(W @ Wi - eye).max() < 1e-9
    assert np.abs(WiT - Wi.T).max() < 1e-12 * max(1.0, np.abs(Wi).max())
