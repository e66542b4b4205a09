"""gsk_density_noalloc: the density matrix for callers that cannot allocate.

Some callers of this library cannot call cudaMalloc (their device memory
belongs to their own pool allocator, or allocation is forbidden after
start-up because it can stall the device). gsk_density_noalloc serves them
with a fixed device array inside libgsk instead of handle-owned scratch. This
test calls it through the C ABI twice in a row, with different inputs, and
compares each result with gsk_density's on the same inputs. The file is
named so that pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_density_matches_handle_density_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk
    from paper_1609_08377_gb300 import synthetic as syn

    s = syn.make_system(64, 1.0, 0)
    solver = gsk.from_system(s)
    rng = np.random.default_rng(7)
    calls = [(16, -10.0, 0.1), (64, -8.5, 0.05)]   # second call: more shifts, other mu and kT
    for S, mu, kT in calls:
        eps = syn.energy_grid(S)
        w = syn.trapezoid_weights(eps)
        n_elem = 5000
        Gh = rng.standard_normal((n_elem, S)) + 1j * rng.standard_normal((n_elem, S))
        G = torch.from_numpy(Gh.ravel()).cuda()
        rho_ref = torch.full((n_elem,), np.nan, dtype=torch.float64, device="cuda")
        rho_new = torch.full((n_elem,), np.nan, dtype=torch.float64, device="cuda")
        solver.density(G, eps, w, mu, kT, rho_ref, n_elem)
        gsk.density_noalloc(G, eps, w, mu, kT, rho_new, n_elem)
        torch.cuda.synchronize()
        a, b = rho_ref.cpu().numpy(), rho_new.cpu().numpy()
        assert np.isfinite(b).all()
        assert np.abs(a - b).max() <= 1e-8 * max(1.0, np.abs(a).max())
    # sizes beyond the fixed array are refused with a clear error
    with pytest.raises(gsk.GskError) as ei:
        eps = syn.energy_grid(2048)
        gsk.density_noalloc(G, eps, syn.trapezoid_weights(eps), -10.0, 0.1, rho_new, 10)
    assert ei.value.code == gsk.GSK_EINVAL
    solver.close()
