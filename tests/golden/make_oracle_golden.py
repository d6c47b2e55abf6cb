"""Write the oracle's results at the headline workload sizes as golden files.

Calls only the CPU oracle (oracle/) and the seeded generators (inputs/); no
value here comes from the CUDA library.  One JSON file per case under
tests/golden/oracle_headline/, read by tests/test_gpu_headline.py:

* the CGLS iteration count, the final ||A^T r|| / ||A^T b|| and its history
  (CGLS of Section 4, right-preconditioned by the spaQR factor W of
  Algorithm 1, stopped below 1e-10 with the unscaled A);
* the stored size nnz(W) (Section 3 memory measure), the number of stored
  operations, the root front and the largest front;
* x at 64 seeded positions and ||x||;
* per stage, the sparsification shapes (Section 2.5: step-1 blocks and the
  step-2 matrices M_p, with their ranks).

Usage: python tests/golden/make_oracle_golden.py CASE [CASE ...]   (or "all").
Each case runs in this process, one after the other; run several processes
for several cases.  The 1024 x 1024 cases take about 10-20 minutes each on
one core.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from inputs.grid_ls import grid_problem  # noqa: E402
from oracle.spaqr import OracleSpaQR  # noqa: E402

OUT = os.path.join(HERE, "oracle_headline")

# name -> (dims, weight law, nested-dissection depth, eps); seed 0 throughout.
CASES = {
    # 2D 1024 x 1024, w = 10^U[-3,3], depth 16, the eps sweep of the 2D headline workload
    "grid2d_1024_eps1e-2": ((1024, 1024, 1), "c3", 16, 1e-2),
    "grid2d_1024_eps1e-4": ((1024, 1024, 1), "c3", 16, 1e-4),
    "grid2d_1024_eps1e-6": ((1024, 1024, 1), "c3", 16, 1e-6),
    # 3D 64^3, w ~ U[1,2), depth 15, eps 1e-3
    "grid3d_64_eps1e-3": ((64, 64, 64), "u12", 15, 1e-3),
    # the high-contrast 3D family of the 128^3 workload (w = 10^U[-3,3]) at 24^3 and 32^3,
    # leaves of about 14 and 16 vertices as at 128^3 with depth 18
    "grid3d_24_c3_eps1e-4": ((24, 24, 24), "c3", 11, 1e-4),
    "grid3d_32_c3_eps1e-4": ((32, 32, 32), "c3", 12, 1e-4),
    "grid3d_32_c3_eps1e-2": ((32, 32, 32), "c3", 12, 1e-2),
}
SAMPLE_SEED = 20210219
SAMPLE_COUNT = 64


def sample_positions(n: int) -> np.ndarray:
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, size=min(n, SAMPLE_COUNT), replace=False))


def shapes_by_stage(stats):
    out = {}
    for name, rows in (("step1", stats.step1), ("step2", stats.step2)):
        for (k, r, c, kk) in rows:
            e = out.setdefault(str(k), {}).setdefault(name, dict(count=0, max_rows=0, max_cols=0, sum_rank=0,
                                                                 max_rank=0, sum_rows_cols_rank=0.0))
            e["count"] += 1
            e["max_rows"] = max(e["max_rows"], int(r))
            e["max_cols"] = max(e["max_cols"], int(c))
            e["sum_rank"] += int(kk)
            e["max_rank"] = max(e["max_rank"], int(kk))
            e["sum_rows_cols_rank"] += float(r) * float(c) * float(kk)
    return out


def run_case(name: str) -> dict:
    dims, law, depth, eps = CASES[name]
    prob = grid_problem(*dims, law, 0)
    t0 = time.time()
    o = OracleSpaQR(prob, depth, eps).factor()
    t1 = time.time()
    x, info = o.solve(prob.b, tol=1e-10, maxit=500)
    t2 = time.time()
    pos = sample_positions(prob.n)
    fronts = o.stats.fronts
    top = [f for f in fronts if f[0] == 1]
    big = max(fronts, key=lambda f: f[1] * f[2])
    return dict(
        case=name,
        dims=list(dims),
        law=law,
        depth=depth,
        eps=eps,
        seed=0,
        m=int(prob.m),
        n=int(prob.n),
        tol=1e-10,
        maxit=500,
        iters=int(info["iters"]),
        rel=float(info["rel"]),
        converged=bool(info["converged"]),
        hist=[float(h) for h in info["hist"]],
        nnz_W=int(o.nnz_W()),
        n_ops=len(o.ops),
        top_front=[int(top[0][1]), int(top[0][2])] if top else [0, 0],
        max_front=[int(big[1]), int(big[2])],
        x_norm=float(np.linalg.norm(x)),
        x_pos=[int(i) for i in pos],
        x_val=[float(x[i]) for i in pos],
        shapes=shapes_by_stage(o.stats),
        oracle_seconds=dict(factor=round(t1 - t0, 1), solve=round(t2 - t1, 1),
                            note="one core of the machine that ran this script; context only"),
        source="oracle/spaqr.py OracleSpaQR (Algorithm 1, Section 2.7) + CGLS (Section 4)",
    )


def main(argv):
    names = list(CASES) if argv == ["all"] else argv
    os.makedirs(OUT, exist_ok=True)
    for name in names:
        res = run_case(name)
        with open(os.path.join(OUT, name + ".json"), "w") as f:
            json.dump(res, f, indent=1)
            f.write("\n")
        print(name, res["iters"], res["rel"], res["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
