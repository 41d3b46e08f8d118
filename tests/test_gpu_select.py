"""GPU GKTL weights / resampling and AMS selection against the oracle: indices
bit-exact given identical weights or scores and the same seed."""
import numpy as np
import pytest
import torch

from tests import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2005_09323_gb300 import build, lbmrare
    build.build()
    lbmrare.lib()
    return lbmrare


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("n,spread", [(1, 1.0), (7, 0.5), (64, 2.0), (1000, 1.0), (4096, 3.0)])
def test_gktl_weights_match_oracle(L, orc, n, spread):
    s = si.log_weights(n, n + 1, spread)
    W = torch.zeros(n, dtype=torch.float64, device="cuda")
    logR = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.gktl_weights(dev(s), W, logR)
    W_ref, logR_ref = orc.gktl_weights(s)
    assert np.allclose(W.cpu().numpy(), W_ref, rtol=1e-13, atol=0)
    assert abs(logR.item() - logR_ref) < 1e-12 * max(1.0, abs(logR_ref))
    assert abs(W.sum().item() - n) < 1e-10 * n


@pytest.mark.parametrize("n", [1, 2, 7, 64, 333, 1024, 4096])
def test_gktl_select_bit_exact(L, orc, n):
    parent = torch.zeros(n, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for seed in range(6):
        W = si.normalised_weights(n, 100 * n + seed, spread=0.3 + seed * 0.4)
        for it in (0, 1, 12345):
            L.gktl_select(dev(W), seed, it, parent, status)
            torch.cuda.synchronize()
            assert status.item() == 0
            assert np.array_equal(parent.cpu().numpy(), orc.gktl_select(W, seed, it))


def test_gktl_select_special_cases(L, orc):
    parent = torch.zeros(8, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    W = np.array([2.0, 0.0, 1.0, 0.0, 3.0, 1.0, 0.0, 1.0])
    L.gktl_select(dev(W), 1, 0, parent, status)
    assert list(parent.cpu().numpy()) == [0, 0, 2, 4, 4, 5, 4, 7]
    L.gktl_select(dev(np.ones(8)), 1, 3, parent, status)
    assert list(parent.cpu().numpy()) == list(range(8))
    # rejected inputs: a NaN weight, weights not summing to N
    bad = np.ones(8)
    bad[3] = np.nan
    L.gktl_select(dev(bad), 1, 0, parent, status)
    assert status.item() == L.LBM_ERR_NONFINITE and np.all(parent.cpu().numpy() == -1)
    L.gktl_select(dev(np.full(8, 1.5)), 1, 0, parent, status)
    assert status.item() == L.LBM_ERR_ARG and np.all(parent.cpu().numpy() == -1)


def test_gktl_weights_nonfinite_poisons(L):
    W = torch.zeros(4, dtype=torch.float64, device="cuda")
    logR = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.gktl_weights(dev([0.0, np.inf, 1.0, 2.0]), W, logR)
    assert torch.isnan(W).all() and torch.isnan(logR).all()


@pytest.mark.parametrize("n,ties", [(2, 0), (32, 0), (256, 0), (256, 3), (4096, 5)])
def test_ams_select_bit_exact(L, orc, n, ties):
    killed = torch.zeros(n, dtype=torch.int32, device="cuda")
    nk = torch.zeros(1, dtype=torch.int32, device="cuda")
    surv = torch.zeros(n, dtype=torch.int32, device="cuda")
    lvl = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in range(4):
        Q = si.scores(n, 7 * n + seed, n_ties=ties)
        for it in (1, 2, 499):
            L.ams_select(dev(Q), seed, it, killed, nk, surv, lvl)
            torch.cuda.synchronize()
            k_ref, s_ref, z_ref = orc.ams_select(Q, seed, it)
            k = nk.item()
            assert k == len(k_ref)
            assert lvl.item() == z_ref
            assert np.array_equal(killed.cpu().numpy()[:k], k_ref)
            assert np.array_equal(surv.cpu().numpy()[:k], s_ref)


def test_ams_select_degenerate(L):
    n = 6
    killed = torch.zeros(n, dtype=torch.int32, device="cuda")
    nk = torch.zeros(1, dtype=torch.int32, device="cuda")
    surv = torch.zeros(n, dtype=torch.int32, device="cuda")
    lvl = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.ams_select(dev(np.full(n, -np.inf)), 0, 1, killed, nk, surv, lvl)
    assert nk.item() == n
    q = np.arange(n, dtype=float)
    q[2] = np.nan
    L.ams_select(dev(q), 0, 1, killed, nk, surv, lvl)
    assert nk.item() == -1
