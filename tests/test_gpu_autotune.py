"""The autotuner (lane width W and inner-CG product kernel) and its on-disk
cache, through the C ABI.

The autotuner times a truncated solve for every (W, kernel) candidate and
keeps the pair with the smallest estimated time of the column set; with
GSK_TUNE_CACHE set, the pick is written to that file and a later call with
the same pencil, request and GPU reads it back without measuring. The tuned
pair is what gsk_solve then runs with batch_w = 0 and the kernel on auto.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402


@pytest.fixture(scope="module")
def gsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk as g
    return g


def test_autotune_pick_cache_and_use(gsk, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("GSK_TUNE_CACHE", str(cache))
    s = syn.make_system(1000, 1.0 / 3.0, 0)
    eps = syn.energy_grid(32)
    z = eps.astype(np.complex128) + 1j
    cols = syn.column_subset(s.M, 96, 3).astype(np.int32)
    eta = syn.eta_per_column(cols.size, 3)
    solver = gsk.from_system(s)
    w = solver.autotune(z, cols, eta=eta, precision="mixed_df")
    r = solver.autotune_result("mixed_df")
    assert not r["from_cache"] and r["W"] == w
    # every (W, kernel) pair was measured, and the pick minimises the estimate
    pairs = {(c["W"], c["kernel"]) for c in r["candidates"]}
    assert pairs == {(W, k) for W in (32, 64, 128) for k in ("gather", "staged")}
    est = {(c["W"], c["kernel"]): c["ms_per_step"] * max(cols.size / c["W"], 2.0) for c in r["candidates"]}
    assert est[(r["W"], r["kernel"])] == min(est.values())
    # the pick is never worse than the untuned default (staged kernel, 128 lanes for more than 64 columns)
    assert est[(r["W"], r["kernel"])] <= est[(128, "gather")]
    lines = cache.read_text().splitlines()
    kcode = {"gather": gsk.GSK_SPMM_GATHER, "staged": gsk.GSK_SPMM_STAGED}[r["kernel"]]
    assert len(lines) == 1 and f"M={s.M} " in lines[0] and lines[0].endswith(f"W={r['W']} kernel={kcode}")
    # gsk_solve with batch_w = 0 and the kernel on auto runs the tuned pair
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * z.size, dtype=torch.complex128, device="cuda")
    _, st, _ = solver.solve(z, cols, G, eta=eta, precision="mixed_df", tol=1e-8)
    torch.cuda.synchronize()
    stt = solver.last_stats()
    assert (st == gsk.GSK_CONVERGED).all()
    assert stt["batch_w"] == r["W"]
    assert stt["spmm_kernel"] == {"gather": gsk.GSK_SPMM_GATHER, "staged": gsk.GSK_SPMM_STAGED}[r["kernel"]]
    solver.close()
    # a new handle of the same pencil: the cache answers, nothing is measured or appended
    solver2 = gsk.from_system(s)
    w2 = solver2.autotune(z, cols, eta=eta, precision="mixed_df")
    r2 = solver2.autotune_result("mixed_df")
    assert r2["from_cache"] and w2 == r["W"] and r2["kernel"] == r["kernel"] and not r2["candidates"]
    assert len(cache.read_text().splitlines()) == 1
    # another request (FP64: no staged kernel, W up to 64) is a miss and appends a line
    solver2.autotune(z, cols, eta=eta, precision="fp64")
    r3 = solver2.autotune_result("fp64")
    assert not r3["from_cache"] and {c["kernel"] for c in r3["candidates"]} == {"gather"}
    assert {c["W"] for c in r3["candidates"]} == {32, 64}
    assert len(cache.read_text().splitlines()) == 2
    solver2.close()
