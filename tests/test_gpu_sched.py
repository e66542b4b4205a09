"""Learned column scheduler on the GPU: features, forward pass, gradients and
Adam against the FP64 CPU oracle, and the queue-order gain over FIFO."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import features as ofeat  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402


@pytest.fixture(scope="module")
def gsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk as g
    return g


@pytest.fixture(scope="module")
def ch1k():
    return syn.make_system(1000, 1.0 / 3.0, 0)


def test_features_match_oracle(gsk, ch1k):
    cols = syn.column_subset(ch1k.M, 300, 0)
    eta = syn.eta_per_column(cols.size, 0)
    s = gsk.from_system(ch1k)
    feat = torch.empty((cols.size, 16), dtype=torch.float32, device="cuda")
    s.features(cols, eta, feat)
    got = feat.cpu().numpy().astype(np.float64)
    want = ofeat.raw_features(ch1k.A, ch1k.B, ch1k.orb_offset, ch1k.orb_count, cols, eta)
    assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max())


def _rand_problem(n=300, seed=0):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, 16)) * 2 + 1
    t = rng.standard_normal(n)
    p = omlp.init_params(seed) + 0.1 * rng.standard_normal(omlp.N_PARAM)
    mean, std = F.mean(0), F.std(0)
    return F, t, p, mean, std


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_matches_oracle(gsk):
    F, t, p, mean, std = _rand_problem()
    y = torch.empty(F.shape[0], dtype=torch.float32, device="cuda")
    gsk.mlp_forward(F.shape[0], _dev(F), _dev(np.concatenate([mean, std])), _dev(p), y)
    torch.cuda.synchronize()
    want, _ = omlp.forward(p, (F - mean) / std)
    assert np.abs(y.cpu().numpy() - want).max() <= 1e-4 * max(1.0, np.abs(want).max())


def test_gradient_matches_oracle(gsk):
    F, t, p, mean, std = _rand_problem(n=1000, seed=1)
    n = F.shape[0]
    params = _dev(p)
    grad = torch.empty(omlp.N_PARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(gsk.mlp_workspace_bytes(n) // 4 + 1, dtype=torch.float32, device="cuda")
    gsk.mlp_train_step(n, _dev(F), _dev(np.concatenate([mean, std])), _dev(t), params, None, None, 0, 0.0,
                       work, grad=grad, loss=loss)
    torch.cuda.synchronize()
    X = (F - mean) / std
    g = omlp.grad(p, X, t)
    got = grad.cpu().numpy()
    assert np.abs(got - g).max() <= 2e-4 * np.abs(g).max()
    assert abs(loss.item() - omlp.loss(p, X, t)) <= 1e-4 * omlp.loss(p, X, t)
    # t = 0 leaves the parameters untouched
    assert np.array_equal(params.cpu().numpy(), p.astype(np.float32))


def test_adam_steps_match_oracle(gsk):
    F, t, p, mean, std = _rand_problem(n=500, seed=2)
    n = F.shape[0]
    X = (F - mean) / std
    params = _dev(p)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    work = torch.empty(gsk.mlp_workspace_bytes(n) // 4 + 1, dtype=torch.float32, device="cuda")
    po, mo, vo = p.copy(), np.zeros_like(p), np.zeros_like(p)
    for it in (1, 2, 3):
        gsk.mlp_train_step(n, _dev(F), _dev(np.concatenate([mean, std])), _dev(t), params, m, v, it, 1e-3, work)
        po, mo, vo = omlp.adam_step(po, omlp.grad(po, X, t), mo, vo, it, lr=1e-3)
    torch.cuda.synchronize()
    assert np.abs(params.cpu().numpy() - po).max() <= 5e-6


def test_training_on_gpu_reduces_loss(gsk):
    rng = np.random.default_rng(5)
    F = rng.standard_normal((2000, 16))
    t = np.tanh(F[:, 0]) + 0.5 * F[:, 1] - 0.3 * F[:, 2] ** 2
    from paper_1609_08377_gb300 import scheduler
    model = scheduler.fit(F, np.exp(t), epochs=600, lr=3e-3, log=lambda *a: None)
    hist = model["loss_history"]
    assert hist[-1][1] < 0.1 * hist[0][1]


def test_learned_order_beats_fifo(gsk, ch1k):
    """Same columns and damping mix, FIFO queue vs longest-predicted-first.

    Each column's arithmetic does not depend on its lane or its place in the
    queue, so both runs give identical G and step counts per column; only the
    number of lock-step outer steps (the makespan of the batch) changes.
    """
    from paper_1609_08377_gb300 import scheduler
    if not os.path.exists(scheduler.MODEL_PATH):
        pytest.skip("no trained scheduler model")
    model = scheduler.load()
    cols = syn.column_subset(ch1k.M, 384, 0)
    eta = syn.eta_per_column(cols.size, 0)
    s = gsk.from_system(ch1k)
    scheduler.install(s, model)
    z = syn.energy_grid(64).astype(np.complex128) + 1j
    off = s.pattern_offsets(cols)
    out = {}
    for sched in ("fifo", "learned"):
        G = torch.empty(int(off[-1]) * 64, dtype=torch.complex128, device="cuda")
        it, st, _ = s.solve(z, cols, G, eta=eta, precision="mixed_df", tol=1e-8, batch_w=64, sched=sched)
        torch.cuda.synchronize()
        out[sched] = (G.cpu().numpy(), it, s.last_stats()["outer_steps"])
    assert np.array_equal(out["fifo"][1], out["learned"][1])
    assert np.array_equal(out["fifo"][0], out["learned"][0])
    steps_fifo, steps_learned = out["fifo"][2], out["learned"][2]
    lower = int(np.ceil(out["fifo"][1].sum() / 64))
    print(f"outer steps: fifo {steps_fifo}, learned {steps_learned}, lower bound {lower}")
    assert steps_learned < steps_fifo
