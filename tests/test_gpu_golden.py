"""Full-size parity: sampled columns of the 20,000- and 100,000-atom workloads.

The stored references (tests/golden/*.json) were written by
tests/golden/make_golden.py, which calls only the CPU oracle (naive FP64
B-Lanczos run to a 1e-10 residual). The solver runs here in the bench's
configuration (double-float mixed precision, tol 1e-8, 128 shifts) and must
meet |Delta G| / max |G| <= 1e-8 on every stored shift; its step count must
agree with the oracle's step count at the 1e-8 level (the oracle checks the
residual every 10 steps).
"""

import glob
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    out = []
    for p in sorted(glob.glob(os.path.join(HERE, "golden", f"{name}_col*.json"))):
        out.append(json.load(open(p)))
    return out


@pytest.mark.parametrize("name,prec", [("ch20k", "mixed_df"), ("ch20k", "fp64"), ("ch100k", "mixed_df")])
def test_golden_columns(name, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    refs = _golden(name)
    if not refs:
        pytest.skip(f"no stored oracle columns for {name}")
    if prec == "fp64":
        refs = refs[-2:]          # the two shortest-running columns are enough for the FP64 path
    from paper_1609_08377_gb300 import gsk

    wl = syn.WORKLOADS[name]
    s = syn.make_system(wl.n_atoms, wl.c_fraction, refs[0]["seed"])
    solver = gsk.from_system(s)
    cols = np.array([r["column"] for r in refs], dtype=np.int32)
    eta = np.array([r["eta"] for r in refs])
    eps = syn.energy_grid(wl.n_shifts)
    z = eps.astype(np.complex128) + 1j
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * wl.n_shifts, dtype=torch.complex128, device="cuda")
    it, st, _ = solver.solve(z, cols, G, eta=eta, precision=prec, tol=1e-8, batch_w=32)
    torch.cuda.synchronize()
    Gh = G.cpu().numpy().reshape(int(off[-1]), wl.n_shifts)
    assert (st == gsk.GSK_CONVERGED).all()
    for c, r in enumerate(refs):
        R = np.array(r["G_re"]) + 1j * np.array(r["G_im"])
        got = Gh[off[c]:off[c + 1], ::r["shift_stride"]]
        err = np.abs(got - R).max() / np.abs(R).max()
        assert err <= 1e-8, (r["column"], err)
        n_or = r["iters_1e-8"]
        # an inexact inner solve (FP32 passes to 3e-6 in the mixed modes) delays
        # convergence by about 1-2 %; the FP64 inner solve (1e-12) tracks the oracle
        slack = 0.02 if prec == "fp64" else 0.04
        assert abs(it[c] - n_or) <= slack * n_or + 10, (r["column"], it[c], n_or)
    solver.close()
