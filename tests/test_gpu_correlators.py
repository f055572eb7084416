"""Equal-time connected correlators after the quench (tgba_quench_correlators: Majorana-string
elements in the reduced form, then Re(B^H Z B)) against exact diagonalisation on a complete
basis and against the oracle (direct Pfaffians of the whole string) on truncated ones, up to
the paper's L = 60."""
import numpy as np
import pytest
import torch

from oracle import ed
from oracle import tgba as otgba
from paper_2410_04204_gb300 import tgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _run(b, h0, hx, trunc, order, t_max, n_t, j_max):
    mx = torch.empty(n_t, dtype=torch.float64, device="cuda")
    corr = torch.empty(j_max * n_t, dtype=torch.float64, device="cuda")
    chi = tgba.tgba_quench_correlators(b, 0, h0, hx, trunc, order, t_max, n_t, j_max, mx, corr)
    return chi, mx.cpu().numpy(), corr.cpu().numpy().reshape(j_max, n_t)


def test_complete_basis_equals_ed():
    L, h, h0, hx, j_max, t_max, n_t = 8, 1.0, 0.5, 0.2, 4, 5.0, 21
    b = tgba.tgba_build_basis(L, h, [0], L)
    try:
        tgba.tgba_compute_x(b)
        n = sum(tgba.tgba_sector_sizes(b)[0])
        chi, mx, corr = _run(b, h0, hx, float(n), 1, t_max, n_t, j_max)
        t = np.linspace(0.0, t_max, n_t)
        assert chi == n
        assert np.abs(mx - ed.quench_magnetisation(L, h0, h, hx, t)).max() < 1e-9
        assert np.abs(corr - ed.quench_correlators(L, h0, h, hx, t, j_max)).max() < 1e-9
    finally:
        tgba.tgba_basis_free(b)


@pytest.mark.parametrize("L,mq,cut,trunc,order,j_max", [(12, 6, None, 80, 1, 3), (10, 10, None, 6.0, 0, 3),
                                                       (60, 4, 3.0, 40, 1, 8)])
def test_truncated_against_oracle(L, mq, cut, trunc, order, j_max):
    h, h0, hx, t_max, n_t = 1.0, 0.5, 0.1, 8.0, 33
    b = tgba.tgba_build_basis(L, h, [0], mq, -1.0 if cut is None else cut)
    try:
        tgba.tgba_compute_x(b)
        chi, mx, corr = _run(b, h0, hx, float(trunc), order, t_max, n_t, j_max)
        if order == 1:
            size = trunc
        else:
            from oracle import basis as obs
            from oracle import modes as md
            ns, r = obs.sector_basis(L, h, 0, mq, cut)
            E = np.array([x.E for x in ns] + [x.E for x in r])
            size = int(np.sum(E <= md.vacuum_energy(L, md.NS, h) + trunc + 1e-9))
        assert chi == size
        t, mo, co = otgba.quench_correlators(L, h, h0, hx, mq, cut, order, size, t_max, n_t, j_max)
        assert np.abs(mx - mo).max() < 1e-9
        assert np.abs(corr - co).max() < 1e-9
    finally:
        tgba.tgba_basis_free(b)


def test_rejects_strings_that_do_not_fit():
    b = tgba.tgba_build_basis(120, 1.0, [0], 2, 1.0)     # Pfaffians of size 4 + 2 j_max = 204: too big
    try:
        tgba.tgba_compute_x(b)
        mx = torch.empty(4, dtype=torch.float64, device="cuda")
        corr = torch.empty(4 * 100, dtype=torch.float64, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_quench_correlators(b, 0, 0.5, 0.1, 4.0, 1, 1.0, 4, 100, mx, corr)
        assert e.value.code == tgba.TGBA_EINVAL
    finally:
        tgba.tgba_basis_free(b)
