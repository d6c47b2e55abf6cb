"""Autotuner of the column-pivoted QR launch shapes (cluster size / global mode
per size class): the table is written and read back, a malformed table is
refused, and factorizations that use a tuned table keep their parity with the
oracle (the launch shape changes the rounding order at most)."""
import numpy as np
import pytest

from inputs.grid_ls import grid_problem
from oracle.spaqr import OracleSpaQR

pytestmark = pytest.mark.gpu


def test_autotune_table_roundtrip_and_parity(tmp_path):
    import paper_2102_09878_gb300 as sq

    path = str(tmp_path / "qrcp_table.txt")
    try:
        secs = sq.autotune("mixed", max_m=512, max_n=1024, path=path)
        assert secs > 0
        rows = [ln.split() for ln in open(path) if not ln.startswith("#")]
        assert rows and all(len(r) == 4 and r[0] == "4" and r[3] in ("1", "2", "4", "8", "16", "32") for r in rows)
        sq.load_tuning(path)
        p = grid_problem(64, 64, 1, "u12", 0)
        an = sq.Analysis(p.dims, 6)
        for prec in ("mixed", "fp64"):
            g = sq.SpaQR(p, an, eps=1e-4, precision=prec)
            x = g.solve(p.b)
            A = p.to_scipy()
            assert np.linalg.norm(A.T @ (A @ x - p.b)) < 1e-10 * np.linalg.norm(A.T @ p.b)
        o = OracleSpaQR(p, 6, 1e-4).factor()
        _, info = o.solve(p.b)
        g = sq.SpaQR(p, an, eps=1e-4)
        g.solve(p.b)
        assert abs(g.last_info["iters"] - info["iters"]) <= max(1, int(np.ceil(0.1 * info["iters"])))
    finally:
        sq.load_tuning(None)


def test_load_tuning_rejects_malformed(tmp_path):
    import paper_2102_09878_gb300 as sq
    from paper_2102_09878_gb300 import SpaqrError

    bad = tmp_path / "bad.txt"
    bad.write_text("4 7 7 3\n")
    with pytest.raises(SpaqrError):
        sq.load_tuning(str(bad))
    with pytest.raises(SpaqrError):
        sq.load_tuning(str(tmp_path / "missing.txt"))
    sq.load_tuning(None)
