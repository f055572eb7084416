"""S(k, w) at k != 0 on the GPU (tgba_dsf_k: cross-sector Pfaffians of the contraction table, then
the Eq. 9 weights and the FP32 Lorentzian sum) against exact diagonalisation on a complete basis
and against the oracle on a truncated one."""
import numpy as np
import pytest
import torch

from oracle import ed
from oracle import tgba as otgba
from paper_2410_04204_gb300 import tgba
from tests.test_oracle_dsf_k import _multiplets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _run(b, s, s0, hx, n_w=256, w=(0.0, 8.0), eta=0.05):
    n = sum(tgba.tgba_sector_sizes(b)[s])
    S = torch.empty(n_w, dtype=torch.float32, device="cuda")
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    dE = torch.empty(n, dtype=torch.float64, device="cuda")
    tgba.tgba_dsf_k(b, s, s0, hx, w[0], w[1], n_w, eta, S, None, 0, wt, dE)
    return S.cpu().numpy(), wt.cpu().numpy(), dE.cpu().numpy()


def test_dsf_k_complete_basis_equals_ed():
    """L = 12, all states of sectors m = 0, 3, 6: levels and weights of S(k, w) at k = pi/2 and pi
    equal exact diagonalisation (weights summed over degenerate multiplets)."""
    L, h, hx = 12, 1.0, 0.1
    b = tgba.tgba_build_basis(L, h, [0, 3, 6], L)
    try:
        tgba.tgba_compute_x(b)
        for s, m in ((1, 3), (2, 6)):
            _, w, dE = _run(b, s, 0, hx)
            dE_ed, w_ed = ed.sector_dsf_weights(L, h, hx, m)
            assert np.abs(np.sort(dE) - np.sort(dE_ed)).max() < 1e-9
            a, c = _multiplets(dE, w), _multiplets(dE_ed, w_ed)
            assert a.shape == c.shape and np.abs(a - c).max() < 1e-9
    finally:
        tgba.tgba_basis_free(b)


def test_dsf_k_truncated_against_oracle():
    """L = 12, M <= 4, sectors m = 0 and 2: S(k, w) on 256 points against the oracle's direct
    Pfaffians (FP32 Lorentzian sum: 1e-5 of the peak)."""
    L, h, hx, mq = 12, 1.0, 0.1, 4
    b = tgba.tgba_build_basis(L, h, [0, 2], mq)
    try:
        tgba.tgba_compute_x(b)
        S, w, dE = _run(b, 1, 0, hx)
        dE_o, w_o, S_o = otgba.dsf_k(L, h, hx, 2, mq, None, 0.0, 8.0, 256, 0.05)
        assert np.abs(S - S_o).max() <= 1e-5 * S_o.max()
        a, c = _multiplets(dE, w), _multiplets(dE_o, w_o)
        assert a.shape == c.shape and np.abs(a - c).max() < 1e-10 * max(1.0, c[:, 1].max())
    finally:
        tgba.tgba_basis_free(b)


def test_dsf_k_at_k0_equals_dsf_and_rejects_bad_reference():
    L, h, hx, mq = 10, 1.0, 0.1, 4
    b = tgba.tgba_build_basis(L, h, [0, 1], mq)
    try:
        tgba.tgba_compute_x(b)
        S1, w1, _ = _run(b, 0, 0, hx)
        S0 = torch.empty(256, dtype=torch.float32, device="cuda")
        tgba.tgba_dsf(b, 0, hx, 0.0, 8.0, 256, 0.05, S0)
        assert np.abs(S1 - S0.cpu().numpy()).max() <= 1e-6 * S1.max()
        with pytest.raises(tgba.TgbaError) as e:             # the reference must be the k = 0 sector
            _run(b, 0, 1, hx)
        assert e.value.code == tgba.TGBA_EINVAL
    finally:
        tgba.tgba_basis_free(b)
