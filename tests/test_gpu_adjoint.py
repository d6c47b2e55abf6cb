"""GPU adjoint of the least-squares solve (torch.autograd) against the
reference gradient of oracle/adjoint.py, through the C ABI.

* lambda = (A^T A)^{-1} g by W-preconditioned CG matches a sparse direct solve.
* dL/db and dL/dvals of one fused kernel match the definition for the same
  x and lambda (1e-12), and end to end (autograd) the reference gradient.
* Central finite differences (h = 1e-6) of the GPU solve agree with the
  GPU gradient.
* Batches: side-by-side solves and adjoints of several problems with one
  pattern (per-problem seeds, weights 10^U[-2,2]); the 64 x 128^2 batch is
  checked against the reference gradient on sampled problems.
"""
import numpy as np
import pytest

from inputs.grid_ls import grid_problem
from oracle import adjoint

pytestmark = pytest.mark.gpu


def _solver(p, depth, **kw):
    import paper_2102_09878_gb300 as sq

    an = sq.Analysis(p.dims, depth)
    return sq.SpaQR(p, an, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_normal_solve_matches_direct(precision):
    p = grid_problem(32, 32, 1, "c2", 1)
    s = _solver(p, 5, eps=1e-3, precision=precision)
    g = np.random.default_rng(3).standard_normal(p.n)
    lam = s.solve_normal(g, tol=1e-12)
    assert s.last_normal_info["converged"]
    ref = adjoint.normal_solve(p.to_scipy().tocsr(), g)
    assert _rel(lam, ref) < 1e-9


def test_grad_kernel_matches_definition():
    p = grid_problem(24, 20, 1, "c2", 2)
    s = _solver(p, 5, eps=1e-3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(p.n)
    lam = rng.standard_normal(p.n)
    gb, gv = s.lstsq_grad(p.b, x, lam)
    A = p.to_scipy().tocsr()
    r = p.b - A @ x
    al = A @ lam
    rows = np.repeat(np.arange(p.m), np.diff(A.indptr))
    np.testing.assert_allclose(gb, al, rtol=1e-12, atol=1e-12 * np.abs(al).max())
    ref = r[rows] * lam[A.indices] - al[rows] * x[A.indices]
    np.testing.assert_allclose(gv, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def _torch_problem(p):
    import torch

    vals = torch.tensor(p.vals, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(p.b, dtype=torch.float64, device="cuda", requires_grad=True)
    return vals, b


def test_autograd_matches_reference_gradient():
    import torch
    from paper_2102_09878_gb300.lstsq import lstsq

    p = grid_problem(32, 32, 1, "c2", 5)
    s = _solver(p, 5, eps=1e-4, tol=1e-12)
    vals, b = _torch_problem(p)
    c = torch.tensor(np.random.default_rng(9).standard_normal(p.n), device="cuda")
    x = lstsq(vals, b, s)
    (c * x).sum().backward()
    xr, lamr, gbr, gvr = adjoint.lstsq_grad(p.to_scipy().tocsr(), p.b, c.cpu().numpy())
    assert _rel(x.detach().cpu().numpy(), xr) < 1e-9
    assert _rel(b.grad.cpu().numpy(), gbr) < 1e-9
    assert _rel(vals.grad.cpu().numpy(), gvr) < 1e-8


def test_autograd_central_differences():
    import torch
    from paper_2102_09878_gb300.lstsq import lstsq

    p = grid_problem(16, 16, 1, "c2", 6)
    s = _solver(p, 4, eps=1e-4, tol=1e-14, maxit=2000)
    vals, b = _torch_problem(p)
    c = torch.tensor(np.random.default_rng(2).standard_normal(p.n), device="cuda")
    x = lstsq(vals, b, s)
    (c * x).sum().backward()
    gv = vals.grad.cpu().numpy()
    gb = b.grad.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(8)

    def loss(v, bb):
        with torch.no_grad():
            return float((c * lstsq(v, bb, s)).sum())

    for e in rng.choice(p.nnz, 16, replace=False):
        vp, vm = vals.detach().clone(), vals.detach().clone()
        vp[e] += h
        vm[e] -= h
        fd = (loss(vp, b.detach()) - loss(vm, b.detach())) / (2 * h)
        assert abs(fd - gv[e]) <= 1e-5 * max(1.0, abs(fd)), (e, fd, gv[e])
    for i in rng.choice(p.m, 8, replace=False):
        bp, bm = b.detach().clone(), b.detach().clone()
        bp[i] += h
        bm[i] -= h
        fd = (loss(vals.detach(), bp) - loss(vals.detach(), bm)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, gb[i])


def _batch_check(nx, depth, count, sample, eps):
    import torch
    import paper_2102_09878_gb300 as sq
    from paper_2102_09878_gb300.lstsq import lstsq_batch

    probs = [grid_problem(nx, nx, 1, "c2", q) for q in range(count)]
    an = sq.Analysis(probs[0].dims, depth)
    solvers = sq.factor_batch(probs, an, eps=eps, tol=1e-13)  # concurrent factorizations
    vals = torch.tensor(np.stack([p.vals for p in probs]), device="cuda", requires_grad=True)
    bs = torch.tensor(np.stack([p.b for p in probs]), device="cuda", requires_grad=True)
    C = torch.tensor(np.random.default_rng(11).standard_normal((count, probs[0].n)), device="cuda")
    X = lstsq_batch(vals, bs, solvers)
    (C * X).sum().backward()
    for q in sample:
        A = probs[q].to_scipy().tocsr()
        xr, lamr, gbr, gvr = adjoint.lstsq_grad(A, probs[q].b, C[q].cpu().numpy())
        assert _rel(X[q].detach().cpu().numpy(), xr) < 1e-8
        assert _rel(bs.grad[q].cpu().numpy(), gbr) < 1e-8
        assert _rel(vals.grad[q].cpu().numpy(), gvr) < 1e-7
    # every problem: the normal-equation residual of its solution
    for q in range(count):
        A = probs[q].to_scipy().tocsr()
        x = X[q].detach().cpu().numpy()
        assert np.linalg.norm(A.T @ (A @ x - probs[q].b)) < 1e-9 * np.linalg.norm(A.T @ probs[q].b)


def test_batch_small():
    _batch_check(24, 5, 4, [0, 1, 2, 3], 1e-3)


def test_batch_64_problems_128():
    # 64 independent 128 x 128 problems (seeds 0..63), reference gradient on two of them
    _batch_check(128, 8, 64, [0, 37], 1e-3)


def test_update_values_refactor():
    import copy

    p = grid_problem(24, 24, 1, "c2", 0)
    s = _solver(p, 5, eps=1e-3)
    # values moved by 1 %: the old factor still preconditions well
    q = copy.deepcopy(p)
    q.vals = p.vals * (1.0 + 0.01 * np.random.default_rng(5).standard_normal(p.nnz))
    s.update_values(q.vals, refactor=False)
    x1 = s.solve(q.b)
    xr = adjoint.lstsq(q.to_scipy().tocsr(), q.b)
    assert _rel(x1, xr) < 1e-8
    # other weights altogether (seed 1): refactorize
    r = grid_problem(24, 24, 1, "c2", 1)
    s.update_values(r.vals, refactor=True)
    x2 = s.solve(r.b)
    assert _rel(x2, adjoint.lstsq(r.to_scipy().tocsr(), r.b)) < 1e-8


def test_factor_batch_matches_single_factorizations():
    import paper_2102_09878_gb300 as sq

    probs = [grid_problem(48, 40, 1, "c2", q) for q in range(6)]
    an = sq.Analysis(probs[0].dims, 6)
    batch = sq.factor_batch(probs, an, eps=1e-3)
    for p, b in zip(probs, batch):
        s = sq.SpaQR(p, an, eps=1e-3)
        xb, xs = b.solve(p.b), s.solve(p.b)
        assert b.last_info["iters"] == s.last_info["iters"]
        assert _rel(xb, xs) < 1e-12
        ob, os_ = b.ops(), s.ops()
        assert len(ob) == len(os_)
        for u, v in zip(ob, os_):
            assert u["kind"] == v["kind"] and np.array_equal(u["slots"], v["slots"])
