"""GPU parity with the oracle on the paper's own Inverse-Poisson workload
(A = J^T, Appendices A and B) through the C ABI, with the u-row matching
passed in spaqr_csr.match (Section 2.2).

* eps = 0 (2D 32^2): every stored factor equals the oracle's to 1e-10, CGLS
  converges in at most 2 iterations and x equals the oracle's to 1e-9.
* eps > 0 (2D 32^2 with and without the flat region, 3D 12^3):
  ||A^T r|| / ||A^T b|| < 1e-10 and the iteration count within
  max(1, ceil(0.1 * it_oracle)) of the oracle's.
* Mixed precision on 2D 64^2 reaches the same residual.
* A matching that is not one is rejected with SPAQR_ERR_INVALID_ARG.
"""
import math

import numpy as np
import pytest

from inputs.inverse_poisson import inverse_poisson
from oracle.spaqr import OracleSpaQR

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _gpu(prob, depth, **kw):
    import paper_2102_09878_gb300 as sq

    return sq.SpaQR(prob, sq.Analysis(prob.dims, depth), **kw)


def _rel_normal(p, x):
    A = p.to_scipy()
    return np.linalg.norm(A.T @ (A @ x - p.b)) / np.linalg.norm(A.T @ p.b)


def test_eps0_factors_match_oracle():
    p = inverse_poisson(32, 2, seed=1)
    o = OracleSpaQR(p, 5, 0.0).factor()
    g = _gpu(p, 5, eps=0.0)
    gops, oops = g.ops(), o.ops
    assert len(gops) == len(oops)
    for a, b in zip(gops, oops):
        assert a["kind"] == b.kind and a["stage"] == b.stage
        np.testing.assert_array_equal(a["slots"], b.slots)
        if b.kind == "Rs":
            assert _rel(np.hstack([a["R"], a["Rn"]]), np.hstack([b.R, b.Rn])) < 1e-10
        elif b.kind == "Rp":
            assert _rel(a["R"], b.R) < 1e-10
        else:
            assert _rel(a["V"], b.V) < 1e-10 and _rel(a["taus"], b.taus) < 1e-10
    x = g.solve(p.b)
    assert g.last_info["iters"] <= 2
    xo, _ = o.solve(p.b)
    assert _rel(x, xo) < 1e-9


@pytest.mark.parametrize("n,dim,flat,depth,eps", [(32, 2, 0.0, 5, 1e-4), (32, 2, 0.9, 5, 1e-3),
                                                  (12, 3, 0.0, 6, 1e-3)])
def test_eps_solve_matches_oracle(n, dim, flat, depth, eps):
    p = inverse_poisson(n, dim, flat, seed=1)
    o = OracleSpaQR(p, depth, eps).factor()
    _, io = o.solve(p.b)
    g = _gpu(p, depth, eps=eps)
    x = g.solve(p.b)
    assert _rel_normal(p, x) < 1e-10
    it, ito = g.last_info["iters"], io["iters"]
    assert abs(it - ito) <= max(1, math.ceil(0.1 * ito)), (it, ito)


def test_mixed_precision_converges():
    p = inverse_poisson(64, 2, seed=2)
    g = _gpu(p, 6, eps=1e-4, precision="mixed")
    x = g.solve(p.b)
    assert _rel_normal(p, x) < 1e-10


def test_bad_matching_is_rejected():
    import paper_2102_09878_gb300 as sq

    p = inverse_poisson(16, 2, seed=0)
    p.match = p.match.copy()
    p.match[1] = p.match[0]  # two columns share a row
    with pytest.raises(sq.SpaqrError) as e:
        _gpu(p, 4, eps=1e-4)
    assert "match" in str(e.value)
