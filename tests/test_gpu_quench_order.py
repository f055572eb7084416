"""The quench with overlap- and energy-ordered nested truncations (the Quench section) and the
convergence metric of Eq. 11, through the C ABI, against the oracle."""
import numpy as np
import pytest
import torch

from oracle import basis as obs
from oracle import modes as md
from oracle import tgba as otgba
from paper_2410_04204_gb300 import tgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _run(b, h0, hx, trunc, order, t_max, n_t, method=0, eps=True):
    nv = len(trunc)
    mx = torch.empty(nv * n_t, dtype=torch.float64, device="cuda")
    nrm = torch.empty(nv, dtype=torch.float64, device="cuda")
    ep = torch.empty(max(1, nv - 1), dtype=torch.float64, device="cuda") if eps else None
    chi = tgba.tgba_quench_ordered(b, 0, h0, [hx] * nv, trunc, order, t_max, n_t, mx, nrm, ep, method=method)
    return (chi, mx.cpu().numpy().reshape(nv, n_t), nrm.cpu().numpy(),
            None if ep is None else ep.cpu().numpy()[:nv - 1])


@pytest.mark.parametrize("L,mq,sizes", [(12, 6, [16, 48, 120]), (10, 10, [16, 48, 100])])
def test_overlap_order_against_oracle(L, mq, sizes):
    h, h0, hx, t_max, n_t = 1.0, 0.5, 0.1, 12.0, 61
    b = tgba.tgba_build_basis(L, h, [0], mq)
    try:
        tgba.tgba_compute_x(b)
        chi, mx, nrm, eps = _run(b, h0, hx, [float(x) for x in sizes], 1, t_max, n_t)
        t, mo, no, eo = otgba.quench_ordered(L, h, h0, hx, mq, None, 1, sizes, t_max, n_t)
        assert list(chi) == sizes
        assert np.abs(nrm - no).max() < 1e-12
        assert np.abs(mx - mo).max() < 1e-9
        assert np.abs(eps - eo).max() < 1e-9
    finally:
        tgba.tgba_basis_free(b)


def test_energy_order_cutoffs_against_oracle():
    L, mq, h, h0, hx, t_max, n_t = 12, 6, 1.0, 0.5, 0.1, 10.0, 41
    cuts = [4.0, 6.0, 9.0]
    b = tgba.tgba_build_basis(L, h, [0], mq)
    try:
        tgba.tgba_compute_x(b)
        chi, mx, nrm, eps = _run(b, h0, hx, cuts, 0, t_max, n_t)
        ns, r = obs.sector_basis(L, h, 0, mq)
        e_ns = md.vacuum_energy(L, md.NS, h)
        E = np.array([s.E for s in ns] + [s.E for s in r])
        sizes = [int(np.sum(E <= e_ns + c + 1e-9)) for c in cuts]
        assert list(chi) == sizes, (chi, sizes)
        t, mo, no, eo = otgba.quench_ordered(L, h, h0, hx, mq, None, 0, sizes, t_max, n_t)
        assert np.abs(mx - mo).max() < 1e-9
        assert np.abs(eps - eo).max() < 1e-9
        # the plain entry point is order 0
        mx2 = torch.empty(len(cuts) * n_t, dtype=torch.float64, device="cuda")
        tgba.tgba_quench(b, 0, h0, [hx] * 3, cuts, t_max, n_t, mx2)
        assert np.abs(mx2.cpu().numpy().reshape(3, n_t) - mx).max() < 1e-12
    finally:
        tgba.tgba_basis_free(b)


def test_metric_needs_nested_eigen_variants():
    L, mq = 10, 4
    b = tgba.tgba_build_basis(L, 1.0, [0], mq)
    try:
        tgba.tgba_compute_x(b)
        with pytest.raises(tgba.TgbaError) as e:              # not nested
            _run(b, 0.5, 0.1, [30.0, 10.0], 1, 5.0, 11)
        assert e.value.code == tgba.TGBA_EINVAL
        with pytest.raises(tgba.TgbaError) as e:              # Chebyshev keeps no B(t)
            _run(b, 0.5, 0.1, [10.0, 30.0], 1, 5.0, 11, method=2)
        assert e.value.code == tgba.TGBA_EINVAL
        chi, mx, nrm, _ = _run(b, 0.5, 0.1, [30.0, 10.0], 1, 5.0, 11, eps=False)   # fine without the metric
        assert list(chi) == [30, 10]
    finally:
        tgba.tgba_basis_free(b)
