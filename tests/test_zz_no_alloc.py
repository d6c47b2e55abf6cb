"""The allocation-free batched column-pivoted QR (spaqr_dense_qrcp_static).

Some callers cannot allocate device memory: code under a memory manager that
owns every device byte, or latency-critical code that cannot take the
synchronisation cudaMalloc/cudaFree may cause.  This entry point serves them
from a fixed static device array.  The test calls it through the C ABI twice
in a row (the array keeps the previous call's contents) and checks it against
the allocating entry point spaqr_dense_qrcp on the same inputs; it also checks
that an oversized batch is refused.  The file name makes pytest collect it
last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(fn_name, mats, eps):
    import torch

    from paper_2102_09878_gb300 import capi

    lib = capi.load()
    ts = [torch.from_numpy(np.ascontiguousarray(A.T)).cuda() for A in mats]
    Vs = [torch.zeros(max(min(A.shape), 1) * max(A.shape[0], 1), dtype=torch.float64, device="cuda") for A in mats]
    Ts = [torch.zeros(max(min(A.shape), 1), dtype=torch.float64, device="cuda") for A in mats]
    P = lambda xs: (C.c_void_p * len(xs))(*[x.data_ptr() for x in xs])  # noqa: E731
    m = np.array([A.shape[0] for A in mats], np.int32)
    n = np.array([A.shape[1] for A in mats], np.int32)
    ld = np.maximum(m, 1).astype(np.int32)
    rank = np.zeros(len(mats), np.int32)
    torch.cuda.synchronize()
    rc = getattr(lib, fn_name)(len(mats), P(ts), capi.ptr(m), capi.ptr(n), capi.ptr(ld), float(eps), P(Vs), P(Ts),
                               capi.ptr(rank), None)
    capi.check(rc)
    out = [t.cpu().numpy().reshape(A.shape[1], A.shape[0]).T.copy() for t, A in zip(ts, mats)]
    V = [v.cpu().numpy() for v in Vs]
    T = [t.cpu().numpy() for t in Ts]
    return rank, out, V, T


def _batch(seed):
    rng = np.random.default_rng(seed)
    shapes = [(16, 150), (40, 25), (9, 9), (120, 700), (200, 1500), (1, 5)]
    mats = []
    for (mm, nn) in shapes:
        r = min(mm, nn)
        mats.append((rng.standard_normal((mm, r)) * np.logspace(0, -8, r)) @ rng.standard_normal((r, nn)))
    return mats


def test_static_scratch_matches_allocating_entry_point_twice():
    for seed, eps in ((1, 1e-4), (2, 0.0)):  # two calls in a row on fresh inputs
        mats = _batch(seed)
        r0, out0, V0, T0 = _run("spaqr_dense_qrcp", mats, eps)
        r1, out1, V1, T1 = _run("spaqr_dense_qrcp_static", mats, eps)
        np.testing.assert_array_equal(r0, r1)
        for a, b in zip(out0, out1):
            assert np.linalg.norm(a - b) <= 1e-10 * max(np.linalg.norm(a), 1e-300)
        for a, b in zip(V0, V1):
            assert np.linalg.norm(a - b) <= 1e-10 * max(np.linalg.norm(a), 1e-300)
        for a, b in zip(T0, T1):
            assert np.linalg.norm(a - b) <= 1e-10 * max(np.linalg.norm(a), 1e-300)


def test_static_scratch_refuses_oversized_batch():
    from paper_2102_09878_gb300 import capi

    rng = np.random.default_rng(3)
    A = rng.standard_normal((400, 3000))  # 9.6 MB work copy > 4 MiB
    with pytest.raises(capi.SpaqrError) as ei:
        _run("spaqr_dense_qrcp_static", [A], 1e-4)
    assert ei.value.name == "CAPACITY" and "4194304" in str(ei.value)
