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
