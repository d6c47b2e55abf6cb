"""GB300-native spaQR: hierarchical sparse QR preconditioning for sparse least squares.

Python face of the C ABI (include/spaqr.h).  Every floating-point step of the
factorization and of the solve runs in the CUDA library; PyTorch only supplies
device memory and streams.  See ``capi`` for the raw binding.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import SpaqrError

__all__ = ["Analysis", "SpaQR", "SpaqrError", "match", "dense_front_qr", "dense_front_qr_f32", "dense_qrcp", "dense_tc_gemm",
           "factor_batch", "solve_batch", "solve_normal_batch", "autotune", "load_tuning", "capi"]


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream))


def _csr_struct(A):
    """(spaqr_csr, arrays kept alive) for any object with m, n, rowptr, colidx, vals (and optional match)."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
    va = np.ascontiguousarray(A.vals, dtype=np.float64)
    mt = getattr(A, "match", None)
    mt = None if mt is None else np.ascontiguousarray(mt, dtype=np.int32)
    csr = capi.Csr(int(A.m), int(A.n), int(rp[-1]), capi.ptr(rp), capi.ptr(ci), capi.ptr(va),
                   None if mt is None else capi.ptr(mt))
    return csr, (rp, ci, va, mt)


def match(A) -> np.ndarray:
    """Maximum-weight row-to-column matching of A (spaqr_match): match[j] = row of column j."""
    csr, keep = _csr_struct(A)
    out = np.zeros(int(A.n), np.int32)
    capi.check(capi.load().spaqr_match(C.byref(csr), capi.ptr(out)))
    return out


class Analysis:
    """Symbolic analysis of an nx*ny*nz grid to nested-dissection depth L (host only);
    Analysis.from_matrix builds it from graph(A^T A) of a matrix without a grid."""

    def __init__(self, dims, depth: int, _handle=None):
        lib = capi.load()
        nx, ny, nz = (tuple(dims) + (1, 1))[:3]
        self.dims = (int(nx), int(ny), int(nz))
        self.depth = int(depth)
        if _handle is not None:
            self._h = _handle
            return
        ordg = capi.GridOrdering(self.dims[0], self.dims[1], self.dims[2], self.depth)
        h = C.c_void_p()
        capi.check(lib.spaqr_analyze(C.byref(ordg), C.byref(h)))
        self._h = h

    @classmethod
    def from_matrix(cls, A, depth: int):
        csr, keep = _csr_struct(A)
        h = C.c_void_p()
        capi.check(capi.load().spaqr_analyze_matrix(C.byref(csr), int(depth), C.byref(h)))
        return cls((int(A.n), 1, 1), depth, _handle=h)

    @property
    def handle(self):
        return self._h

    def stage_clusters(self, k: int):
        """(node, level, vptr, verts) of the clusters alive at stage k."""
        lib = capi.load()
        nc, nv = C.c_int64(), C.c_int64()
        capi.check(lib.spaqr_analysis_stage_size(self._h, k, C.byref(nc), C.byref(nv)))
        node = np.zeros(nc.value, np.int32)
        level = np.zeros(nc.value, np.int32)
        vptr = np.zeros(nc.value + 1, np.int64)
        verts = np.zeros(nv.value, np.int32)
        capi.check(
            lib.spaqr_analysis_stage_clusters(
                self._h, k, capi.ptr(node), capi.ptr(level), capi.ptr(vptr), capi.ptr(verts)
            )
        )
        return node, level, vptr, verts

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                capi.load().spaqr_analysis_destroy(self._h)
                self._h = None
        except Exception:
            pass


def _options(eps, skip, precision, mode, tol, maxit, use_graphs, verbose, stream, rows, persistent_apply,
             step1_qr_width=1280):
    o = capi.default_options()
    o.eps = float(eps)
    o.skip = int(skip)
    o.precision = capi.PREC[precision]
    o.mode = capi.MODE[mode]
    o.tol = float(tol)
    o.maxit = int(maxit)
    o.use_graphs = 1 if use_graphs else 0
    o.verbose = 1 if verbose else 0
    o.stream = _stream_ptr(stream)
    o.row_rule = capi.ROWS[rows]
    o.apply_persistent = 1 if persistent_apply else 0
    o.step1_qr_width = int(step1_qr_width)
    return o


class SpaQR:
    """spaQR factorization of A (CSR arrays on the host) and its CGLS solve.

    ``A`` is any object with m, n, rowptr (int64), colidx (int32), vals (float64).
    """

    def __init__(self, A, analysis: Analysis, eps: float = 1e-4, skip: int = 2, precision: str = "fp64",
                 mode: str = "spaqr", tol: float = 1e-10, maxit: int = 500, use_graphs: bool = True,
                 verbose: bool = False, stream=None, rows: str = "tree", persistent_apply: bool = False,
                 step1_qr_width: int = 1280, _handle=None):
        lib = capi.load()
        self._keep_csr(A)
        o = _options(eps, skip, precision, mode, tol, maxit, use_graphs, verbose, stream, rows, persistent_apply,
                     step1_qr_width)
        self.precision = precision
        self.options = o
        if _handle is None:
            csr = self._csr()
            h = C.c_void_p()
            capi.check(lib.spaqr_factor(C.byref(csr), analysis.handle, C.byref(o), C.byref(h)))
            _handle = h
        self._h = _handle
        self._analysis = analysis

    def _keep_csr(self, A):
        self.m, self.n = int(A.m), int(A.n)
        self._rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        self._colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
        self._vals = np.ascontiguousarray(A.vals, dtype=np.float64)
        match = getattr(A, "match", None)  # optional row matching: match[j] = row of column j
        self._match = None if match is None else np.ascontiguousarray(match, dtype=np.int32)

    def _csr(self):
        return capi.Csr(self.m, self.n, int(self._rowptr[-1]), capi.ptr(self._rowptr), capi.ptr(self._colidx),
                        capi.ptr(self._vals), None if self._match is None else capi.ptr(self._match))

    # ------------------------------------------------------------- solve
    def solve(self, b, check_convergence: bool = True):
        """x = argmin ||A x - b|| by W-preconditioned CGLS.  numpy in -> numpy out
        (host copies inside the call); a CUDA float64 tensor in -> a CUDA tensor
        out (device pointers)."""
        return self._solve(b, check_convergence, capi.load().spaqr_solve)

    def solve_csne(self, b, check_convergence: bool = True):
        """x = argmin ||A x - b|| by the corrected seminormal equations with
        refinement (spaqr_solve_csne); same conventions as solve()."""
        return self._solve(b, check_convergence, capi.load().spaqr_solve_csne)

    def _solve(self, b, check_convergence, fn):
        info = capi.SolveInfo()
        if hasattr(b, "is_cuda") and b.is_cuda:
            import torch

            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
            bb = b.contiguous()
            rc = fn(self._h, capi.ptr(bb), capi.ptr(x), 1, C.byref(info))
        else:
            bb = np.ascontiguousarray(b, dtype=np.float64)
            x = np.zeros(self.n)
            rc = fn(self._h, capi.ptr(bb), capi.ptr(x), 0, C.byref(info))
        if rc != capi.SPAQR_OK and (check_convergence or rc != 4):
            capi.check(rc)
        self.last_info = dict(iters=info.iters, rel=info.rel_resid, converged=bool(info.converged),
                              seconds=info.seconds)
        return x

    def solve_normal(self, g, tol: float = 1e-12, check_convergence: bool = True):
        """lambda = (A^T A)^{-1} g by CG preconditioned with W^{-1} W^{-T} (numpy or CUDA float64)."""
        lib = capi.load()
        info = capi.SolveInfo()
        if hasattr(g, "is_cuda") and g.is_cuda:
            import torch

            lam = torch.empty(self.n, dtype=torch.float64, device=g.device)
            gg = g.contiguous()
            rc = lib.spaqr_solve_normal(self._h, capi.ptr(gg), capi.ptr(lam), 1, float(tol), C.byref(info))
        else:
            gg = np.ascontiguousarray(g, dtype=np.float64)
            lam = np.zeros(self.n)
            rc = lib.spaqr_solve_normal(self._h, capi.ptr(gg), capi.ptr(lam), 0, float(tol), C.byref(info))
        if rc != capi.SPAQR_OK and (check_convergence or rc != 4):
            capi.check(rc)
        self.last_normal_info = dict(iters=info.iters, rel=info.rel_resid, converged=bool(info.converged),
                                     seconds=info.seconds)
        return lam

    def lstsq_grad(self, b, x, lam):
        """(dL/db, dL/dvals) of x = argmin ||A x - b|| given lambda = (A^T A)^{-1} dL/dx."""
        lib = capi.load()
        if hasattr(b, "is_cuda") and b.is_cuda:
            import torch

            gb = torch.empty(self.m, dtype=torch.float64, device=b.device)
            gv = torch.empty(int(self._rowptr[-1]), dtype=torch.float64, device=b.device)
            bb, xx, ll = b.contiguous(), x.contiguous(), lam.contiguous()
            capi.check(lib.spaqr_lstsq_grad(self._h, capi.ptr(bb), capi.ptr(xx), capi.ptr(ll), capi.ptr(gb),
                                            capi.ptr(gv), 1))
        else:
            bb, xx, ll = (np.ascontiguousarray(v, dtype=np.float64) for v in (b, x, lam))
            gb = np.zeros(self.m)
            gv = np.zeros(int(self._rowptr[-1]))
            capi.check(lib.spaqr_lstsq_grad(self._h, capi.ptr(bb), capi.ptr(xx), capi.ptr(ll), capi.ptr(gb),
                                            capi.ptr(gv), 0))
        return gb, gv

    def update_values(self, vals, refactor: bool = False):
        """New values of A (same pattern, CSR order).  refactor=False keeps the
        factor as the preconditioner; refactor=True redoes the factorization."""
        lib = capi.load()
        an = self._analysis.handle if refactor else None
        if hasattr(vals, "is_cuda") and vals.is_cuda:
            vv = vals.contiguous()
            capi.check(lib.spaqr_update_values(self._h, an, capi.ptr(vv), 1, 1 if refactor else 0))
        else:
            vv = np.ascontiguousarray(vals, dtype=np.float64)
            capi.check(lib.spaqr_update_values(self._h, an, capi.ptr(vv), 0, 1 if refactor else 0))

    def apply_Winv(self, z, transpose: bool = False):
        """In place z <- W^{-1} z (or W^{-T} z) for a CUDA float64 tensor of length n."""
        assert z.is_cuda and z.dtype.is_floating_point and z.element_size() == 8 and z.is_contiguous()
        capi.check(capi.load().spaqr_apply_Winv(self._h, capi.ptr(z), 1 if transpose else 0))
        return z

    def apply_A(self, x, forward: bool = True):
        """A D x (forward) or (A D)^T x on CUDA float64 tensors."""
        import torch

        y = torch.empty(self.m if forward else self.n, dtype=torch.float64, device=x.device)
        capi.check(capi.load().spaqr_apply_A(self._h, capi.ptr(x.contiguous()), capi.ptr(y), 1 if forward else 0))
        return y

    def stats(self) -> dict:
        st = capi.Stats()
        capi.check(capi.load().spaqr_get_stats(self._h, C.byref(st)))
        out = {f: getattr(st, f) for f, _ in capi.Stats._fields_ if f not in ("t_phase", "t_kernel", "n_kernel")}
        out["t_phase"] = dict(zip(["eliminate", "prep", "scale", "step1", "step2", "merge"], list(st.t_phase)))
        fam = ["copy", "front_qr", "qrcp", "other", "apply", "spmv"]
        out["t_kernel"] = dict(zip(fam, list(st.t_kernel)))
        out["n_kernel"] = dict(zip(fam, list(st.n_kernel)))
        return out

    def ops(self):
        """The stored factors of W in factorization order (host copies)."""
        lib = capi.load()
        cnt = C.c_int64()
        capi.check(lib.spaqr_num_ops(self._h, C.byref(cnt)))
        out = []
        for i in range(cnt.value):
            kind, stage, c, w = C.c_int(), C.c_int(), C.c_int(), C.c_int()
            capi.check(lib.spaqr_op_info(self._h, i, C.byref(kind), C.byref(stage), C.byref(c), C.byref(w)))
            c_, w_ = c.value, w.value
            slots = np.zeros(c_, np.int32)
            if kind.value == 0:
                nslots = np.zeros(w_, np.int32)
                R = np.zeros(c_ * c_)
                Rn = np.zeros(c_ * w_)
                capi.check(lib.spaqr_op_copy(self._h, i, capi.ptr(slots), capi.ptr(nslots), capi.ptr(R),
                                             capi.ptr(Rn), None))
                out.append(dict(kind="Rs", stage=stage.value, slots=slots, nslots=nslots,
                                R=R.reshape(c_, c_, order="F"), Rn=Rn.reshape(c_, w_, order="F")))
            elif kind.value == 1:
                R = np.zeros(c_ * c_)
                capi.check(lib.spaqr_op_copy(self._h, i, capi.ptr(slots), None, capi.ptr(R), None, None))
                out.append(dict(kind="Rp", stage=stage.value, slots=slots, R=R.reshape(c_, c_, order="F")))
            else:
                V = np.zeros(c_ * w_)
                taus = np.zeros(w_)
                capi.check(lib.spaqr_op_copy(self._h, i, capi.ptr(slots), None, capi.ptr(V), None, capi.ptr(taus)))
                out.append(dict(kind="Qp", stage=stage.value, slots=slots, V=V.reshape(c_, w_, order="F"),
                                taus=taus))
        return out

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                capi.load().spaqr_destroy(self._h)
                self._h = None
        except Exception:
            pass


def autotune(precision: str = "mixed", max_m: int = 2048, max_n: int = 4096, path: str | None = None) -> float:
    """Time the column-pivoted QR launch shapes per size class and install the
    fastest for later factorizations of this process; returns seconds spent."""
    secs = C.c_double()
    capi.check(capi.load().spaqr_autotune(capi.PREC[precision], int(max_m), int(max_n),
                                          path.encode() if path else None, C.byref(secs)))
    return secs.value


def load_tuning(path: str | None):
    """Install a table written by autotune(path=...); None removes the table."""
    capi.check(capi.load().spaqr_load_tuning(path.encode() if path else None))


def _batch(fn, solvers, vecs, n_out, *extra):
    lib = capi.load()
    cnt = len(solvers)
    hs = (C.c_void_p * cnt)(*[s._h.value for s in solvers])
    infos = (capi.SolveInfo * cnt)()
    on_dev = hasattr(vecs[0], "is_cuda") and vecs[0].is_cuda
    if on_dev:
        import torch

        ins = [v.contiguous() for v in vecs]
        outs = [torch.empty(n_out(s), dtype=torch.float64, device=v.device) for s, v in zip(solvers, vecs)]
    else:
        ins = [np.ascontiguousarray(v, dtype=np.float64) for v in vecs]
        outs = [np.zeros(n_out(s)) for s in solvers]
    ip = (C.c_void_p * cnt)(*[capi.ptr(v) for v in ins])
    op = (C.c_void_p * cnt)(*[capi.ptr(v) for v in outs])
    capi.check(getattr(lib, fn)(cnt, hs, ip, op, 1 if on_dev else 0, *extra, infos))
    return outs, [dict(iters=i.iters, rel=i.rel_resid, converged=bool(i.converged)) for i in infos]


def factor_batch(problems, analysis: Analysis, **kw):
    """Factor several matrices with one analysis concurrently (own handle and
    stream each, host planning on several threads); returns SpaQR objects."""
    lib = capi.load()
    kw = dict(kw)
    args = dict(eps=1e-4, skip=2, precision="fp64", mode="spaqr", tol=1e-10, maxit=500, use_graphs=True,
                verbose=False, stream=None, rows="tree", persistent_apply=False, step1_qr_width=1280)
    args.update(kw)
    o = _options(**args)
    holders = []
    for A in problems:
        s = SpaQR.__new__(SpaQR)
        s._keep_csr(A)
        holders.append(s)
    csrs = [s._csr() for s in holders]
    arr = (C.c_void_p * len(csrs))(*[C.addressof(c) for c in csrs])
    out = (C.c_void_p * len(csrs))()
    capi.check(lib.spaqr_factor_batch(len(csrs), arr, analysis.handle, C.byref(o), out))
    res = []
    for s, A, hv in zip(holders, problems, out):
        s.precision = args["precision"]
        s.options = o
        s._h = C.c_void_p(hv)
        s._analysis = analysis
        res.append(s)
    return res


def solve_batch(solvers, bs):
    """x_i = argmin ||A_i x - b_i|| for several factorizations, iterated side by side."""
    return _batch("spaqr_solve_batch", solvers, bs, lambda s: s.n)


def solve_normal_batch(solvers, gs, tol: float = 1e-12):
    """lambda_i = (A_i^T A_i)^{-1} g_i for several factorizations, iterated side by side."""
    return _batch("spaqr_solve_normal_batch", solvers, gs, lambda s: s.n, C.c_double(tol))


# ----------------------------------------------------------- dense kernels
def _colmajor_cuda(A):
    import torch

    A = np.asarray(A, dtype=np.float64)
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()  # (n, m) row-major = m x n column-major


def _from_colmajor(t, m, n):
    return t.cpu().numpy().reshape(n, m).T.copy()


def dense_front_qr(mats, cs, stream=None):
    """Batched front QR (Section 2.3) of numpy matrices; returns the results."""
    lib = capi.load()
    ts = [_colmajor_cuda(A) for A in mats]
    ptrs = (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    m = np.array([A.shape[0] for A in mats], np.int32)
    n = np.array([A.shape[1] for A in mats], np.int32)
    c = np.array(cs, np.int32)
    ld = np.maximum(m, 1).astype(np.int32)
    capi.check(lib.spaqr_dense_front_qr(len(ts), ptrs, capi.ptr(m), capi.ptr(n), capi.ptr(c), capi.ptr(ld),
                                        _stream_ptr(stream)))
    return [_from_colmajor(t, A.shape[0], A.shape[1]) for t, A in zip(ts, mats)]


def _colmajor_cuda32(A):
    import torch

    A = np.asarray(A, dtype=np.float32)
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()


def dense_front_qr_f32(mats, cs, stream=None):
    """FP32 front QR as the mixed-precision factor runs it (tensor-core trailing
    updates on the blocked path); numpy in, numpy (float32) out."""
    lib = capi.load()
    ts = [_colmajor_cuda32(A) for A in mats]
    ptrs = (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    m = np.array([A.shape[0] for A in mats], np.int32)
    n = np.array([A.shape[1] for A in mats], np.int32)
    c = np.array(cs, np.int32)
    ld = np.maximum(m, 1).astype(np.int32)
    capi.check(lib.spaqr_dense_front_qr_f32(len(ts), ptrs, capi.ptr(m), capi.ptr(n), capi.ptr(c), capi.ptr(ld),
                                            _stream_ptr(stream)))
    return [_from_colmajor(t, A.shape[0], A.shape[1]) for t, A in zip(ts, mats)]


def dense_tc_gemm(A, B, Cm, stream=None):
    """Cm - A @ B on the tensor cores (3xTF32, FP32 accumulation); float32 numpy in and out."""
    lib = capi.load()
    m, k = A.shape
    k2, n = B.shape
    assert k == k2 and Cm.shape == (m, n)
    a, b, c = _colmajor_cuda32(A), _colmajor_cuda32(B), _colmajor_cuda32(Cm)
    capi.check(lib.spaqr_dense_tc_gemm(m, n, k, capi.ptr(a), max(m, 1), capi.ptr(b), max(k, 1), capi.ptr(c), max(m, 1),
                                       _stream_ptr(stream)))
    return _from_colmajor(c, m, n)


_QRCP_ROUTE = {"cluster": 1, "auto": 0, "grid": 2}


def _dense_qrcp(mats, eps, stream, route, f32):
    import torch

    lib = capi.load()
    dt = torch.float32 if f32 else torch.float64
    ts = [(_colmajor_cuda32 if f32 else _colmajor_cuda)(A) for A in mats]
    Vs = [torch.zeros(max(min(A.shape), 1) * max(A.shape[0], 1), dtype=dt, device="cuda") for A in mats]
    Ts = [torch.zeros(max(min(A.shape), 1), dtype=dt, device="cuda") for A in mats]
    ptrs = (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    vp = (C.c_void_p * len(ts))(*[t.data_ptr() for t in Vs])
    tp = (C.c_void_p * len(ts))(*[t.data_ptr() for t in Ts])
    m = np.array([A.shape[0] for A in mats], np.int32)
    n = np.array([A.shape[1] for A in mats], np.int32)
    ld = np.maximum(m, 1).astype(np.int32)
    rank = np.zeros(len(ts), np.int32)
    fn = lib.spaqr_dense_qrcp_f32 if f32 else lib.spaqr_dense_qrcp_route
    capi.check(fn(len(ts), ptrs, capi.ptr(m), capi.ptr(n), capi.ptr(ld), float(eps), vp, tp, capi.ptr(rank),
                  _QRCP_ROUTE[route], _stream_ptr(stream)))
    rows, Vout, Tout = [], [], []
    for i, A in enumerate(mats):
        k = int(rank[i])
        out = _from_colmajor(ts[i], A.shape[0], A.shape[1]).astype(np.float64)
        rows.append(out[:k] if k < A.shape[0] else np.array(A, dtype=np.float64))
        Vout.append(Vs[i].double().cpu().numpy()[: A.shape[0] * k].reshape(k, A.shape[0]).T.copy())
        Tout.append(Ts[i].double().cpu().numpy()[:k].copy())
    return rank, rows, Vout, Tout


def release_cached_memory():
    """Return the device and pinned host blocks the library keeps for reuse
    (freed by earlier factorizations) to the driver; returns the bytes that
    were cached."""
    lib = capi.load()
    n = int(lib.spaqr_cached_bytes())
    lib.spaqr_release_cached_memory()
    return n


def dense_qrcp(mats, eps: float, stream=None, route: str = "cluster"):
    """Batched rank-revealing QR; returns (ranks, leading rows of Q^T A, V, taus).
    route: "cluster" (clusters of <= 16 CTAs), "auto" (as the factorization:
    CTA groups over global memory for matrices too large for a cluster) or
    "grid" (CTA groups for every matrix above the one-warp size)."""
    return _dense_qrcp(mats, eps, stream, route, False)


def dense_qrcp_f32(mats, eps: float, stream=None, route: str = "cluster"):
    """dense_qrcp in FP32 (the mixed-precision factorization's kernels); results
    are returned in float64 arrays."""
    return _dense_qrcp(mats, eps, stream, route, True)
