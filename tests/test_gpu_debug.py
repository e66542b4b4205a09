"""The bounds-checked build (libgsk_debug.so, -DGSK_DEBUG) on the GPU.

Its kernels test every block-layout, tile and work-queue index before use
and record the first failure instead of faulting (include/gsk.h lists the
checks). Here it runs, in a child process with GSK_DEBUG=1:
- the self-test, one deliberately failing check that guards no access;
- FP64, staged and gather solves and both inner-CG products on valid inputs,
  where no check may fail.
The results must equal the normal build's results.
"""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUNS = textwrap.dedent('''
    import sys
    import numpy as np, torch
    sys.path.insert(0, ROOT)
    from paper_1609_08377_gb300 import gsk, synthetic as syn

    def runs():
        out = {}
        for name, n_at, frac in (("c64", 64, 1.0), ("ch1k", 1000, 1.0 / 3.0)):
            s = syn.make_system(n_at, frac, 0)
            h = gsk.from_system(s)
            cols = syn.column_subset(s.M, 24, 1).astype(np.int32)
            eta = syn.eta_per_column(cols.size, 1)
            z = syn.energy_grid(16).astype(np.complex128) + 1j
            off = h.pattern_offsets(cols)
            for tag, kw in (("fp64", dict(precision="fp64", batch_w=32)),
                            ("staged", dict(precision="mixed_df", batch_w=32, spmm_kernel="staged")),
                            ("gather", dict(precision="mixed_df", batch_w=64, spmm_kernel="gather"))):
                G = torch.zeros(int(off[-1]) * z.size, dtype=torch.complex128, device="cuda")
                it, st, _ = h.solve(z, cols, G, eta=eta, tol=1e-10, **kw)
                torch.cuda.synchronize()
                stats = h.last_stats()
                assert stats["debug_code"] == 0, (name, tag, stats)
                out[f"{name}_{tag}_G"] = G.cpu().numpy()
                out[f"{name}_{tag}_it"] = it
            g = torch.Generator().manual_seed(3)
            X = torch.randn(s.M * 32, generator=g, dtype=torch.float32).to("cuda")
            for which in (1, 2):
                Y = torch.zeros_like(X)
                h.spmm(which, gsk.GSK_MIXED, 32, X, Y, n_rep=1)
                torch.cuda.synchronize()
                assert h.last_stats()["debug_code"] == 0, (name, which)
                out[f"{name}_spmm{which}"] = Y.cpu().numpy()
            h.close()
        return out
''')


def test_bounds_checked_build(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import build

    build.build(debug=True)
    child = f"ROOT = {ROOT!r}\n" + _RUNS + textwrap.dedent(f'''
        assert gsk.DEBUG_BUILD and gsk.LIB_PATH.endswith("libgsk_debug.so")
        assert gsk.debug_selftest() == (gsk.GSK_OK, 99, 12345678901)
        np.savez({str(tmp_path / "debug.npz")!r}, **runs())
        print("debug build ok")
    ''')
    env = dict(os.environ, GSK_DEBUG="1")
    res = subprocess.run([sys.executable, "-c", child], env=env, capture_output=True, text=True, timeout=1200)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    # the same runs through the normal library in this process
    ns = {"ROOT": ROOT}
    exec(_RUNS, ns)
    want = ns["runs"]()
    got = np.load(tmp_path / "debug.npz")
    # The checks add branches, which may change where the compiler contracts a
    # product and a sum into an FMA, so rounding (and with it the step at which
    # a column converges) may differ: G is held to the parity bar, the step
    # counts to 2% + 10, the FP32 products to their rounding.
    bitwise = True
    for k, v in want.items():
        g = got[k]
        assert g.shape == v.shape, k
        bitwise = bitwise and bool(np.array_equal(g, v))
        if k.endswith("_it"):
            assert (np.abs(g.astype(np.int64) - v) <= 0.02 * v + 10).all(), k
        else:
            scale = max(float(np.abs(v).max()), 1e-300)
            bar = 1e-5 if "spmm" in k else 1e-8
            assert float(np.abs(g - v).max()) <= bar * scale, (k, float(np.abs(g - v).max()) / scale)
    print("bounds-checked build: results bitwise equal to the normal build:", bitwise)
