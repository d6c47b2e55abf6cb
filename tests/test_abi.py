"""C-ABI library: loads, exports every declared symbol, and its host-only
symbolic analysis (nested dissection + interfaces + hierarchy, Section 2.2 and
2.6) equals the oracle's independent implementation.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import nd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2102_09878_gb300 import build as b

    b.build()
    from paper_2102_09878_gb300 import capi

    return capi.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "spaqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spaqr_[a-z_A-Z0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    from paper_2102_09878_gb300 import capi

    assert set(names) == set(capi.SIGNATURES), set(names) ^ set(capi.SIGNATURES)


def test_compute_entry_points_fail_cleanly_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2102_09878_gb300 import capi

    rc = lib.spaqr_dense_front_qr(0, None, None, None, None, None, None)
    assert rc == 8  # SPAQR_ERR_NO_DEVICE
    assert b"device" in lib.spaqr_last_error()


def test_block_cache_is_empty_and_releasable_without_gpu(lib):
    """Host-only cache bookkeeping: nothing cached before any factorization,
    and releasing an empty cache is a no-op (the device wait it starts with
    finds no device here)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    assert lib.spaqr_cached_bytes() == 0
    lib.spaqr_release_cached_memory()
    assert lib.spaqr_cached_bytes() == 0


def test_analyze_rejects_bad_grid(lib):
    from paper_2102_09878_gb300 import capi

    o = capi.GridOrdering(0, 4, 1, 3)
    h = ctypes.c_void_p()
    assert lib.spaqr_analyze(ctypes.byref(o), ctypes.byref(h)) == 1
    o = capi.GridOrdering(4, 4, 1, 0)
    assert lib.spaqr_analyze(ctypes.byref(o), ctypes.byref(h)) == 1


@pytest.mark.parametrize(
    "dims,depth",
    [((8, 8, 1), 3), ((16, 16, 1), 5), ((64, 64, 1), 6), ((13, 29, 1), 6), ((8, 8, 8), 6), ((12, 9, 7), 7),
     ((1, 40, 1), 4), ((5, 5, 1), 6)],
)
def test_symbolic_analysis_matches_oracle(lib, dims, depth):
    import paper_2102_09878_gb300 as sq

    an = sq.Analysis(dims, depth)
    nodes = nd.build_tree(dims, depth)
    keys = nd.finest_keys(nodes, dims, depth)
    for k in range(depth, 0, -1):
        node, level, vptr, verts = an.stage_clusters(k)
        cl = nd.clusters_at_stage(nodes, keys, depth, k)
        assert len(cl) == len(node), k
        for i, c in enumerate(cl):
            assert c.node == node[i] and c.level == level[i]
            np.testing.assert_array_equal(c.verts, verts[vptr[i] : vptr[i + 1]])


def test_factor_checks_its_input_before_the_device(lib):
    """spaqr_factor validates the matrix, the matching and the options on the
    host (INVALID_ARG with a message), before it asks for a GPU; valid input
    on a machine without one then gets NO_DEVICE."""
    import torch

    import paper_2102_09878_gb300 as sq
    from inputs.inverse_poisson import inverse_poisson
    from paper_2102_09878_gb300 import capi

    p = inverse_poisson(8, 2, seed=0)
    an = sq.Analysis(p.dims, 3)

    def factor(rowptr=None, colidx=None, m=None, match="keep", **opt):
        rp = np.ascontiguousarray(p.rowptr if rowptr is None else rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(p.colidx if colidx is None else colidx, dtype=np.int32)
        va = np.ascontiguousarray(p.vals, dtype=np.float64)
        mt = p.match if isinstance(match, str) else match
        mt = None if mt is None else np.ascontiguousarray(mt, dtype=np.int32)
        csr = capi.Csr(p.m if m is None else m, p.n, int(rp[-1]), capi.ptr(rp), capi.ptr(ci), capi.ptr(va),
                       None if mt is None else capi.ptr(mt))
        o = capi.default_options()
        for k, v in opt.items():
            setattr(o, k, v)
        h = ctypes.c_void_p()
        rc = lib.spaqr_factor(ctypes.byref(csr), an.handle, ctypes.byref(o), ctypes.byref(h))
        return rc, lib.spaqr_last_error().decode()

    bad_rowptr = p.rowptr.copy()
    bad_rowptr[0] = 1
    bad_cols = p.colidx.copy()
    bad_cols[3] = p.n
    dup = p.match.copy()
    dup[1] = dup[0]
    # a row with no entry in column 0: some z row far from grid point 0
    A = p.to_scipy().tocsc()
    far = next(r for r in range(p.n, p.m) if A[r, 0] == 0)
    nomatch = p.match.copy()
    nomatch[0] = far
    for kw, msg in [(dict(m=p.n - 1), "m >= n"), (dict(rowptr=bad_rowptr), "rowptr"),
                    (dict(colidx=bad_cols), "column index"), (dict(match=dup), "matching"),
                    (dict(match=nomatch), "no entry"), (dict(row_rule=7), "row rule"), (dict(eps=-1.0), "eps"),
                    (dict(precision=5), "precision"), (dict(step1_qr_width=-1), "step1_qr_width")]:
        rc, err = factor(**kw)
        assert rc == 1 and msg in err, (kw.keys(), rc, err)
    if not torch.cuda.is_available():
        assert factor()[0] == 8  # SPAQR_ERR_NO_DEVICE
        assert factor(match=None)[0] == 8
