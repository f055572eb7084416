"""GPU parity of the hot path against the oracle on small workloads (through the C ABI)."""
import numpy as np
import pytest
import torch

from oracle import basis as obs
from oracle import elements as oel
from oracle import tgba as otgba
from paper_2410_04204_gb300 import inputs, tgba
from tests.gpu_helpers import GpuSector, x_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("L,h,m,mq,cut", [(12, 1.0, 0, 12, None), (12, 1.0, 0, 4, None), (10, 0.6, 3, 10, None),
                                          (12, 1.4, 5, 6, 9.0), (8, 1.0, 0, 8, None)])
def test_basis_and_x_match_oracle(L, h, m, mq, cut):
    b = tgba.tgba_build_basis(L, h, [m], mq, -1.0 if cut is None else cut)
    try:
        g = GpuSector(b, 0, mq)
        ns, r = obs.sector_basis(L, h, m, mq, cut)
        assert sorted(g.keys) == sorted([(0, s.modes) for s in ns] + [(1, s.modes) for s in r])
        pa, pb = g.perm_to(ns, r)
        Eo = np.array([s.E for s in ns] + [s.E for s in r])
        assert np.abs(g.E0 - Eo[np.concatenate([pa, len(ns) + pb])]).max() < 1e-12 * max(1.0, np.abs(Eo).max())
        tgba.tgba_compute_x(b)
        ok, worst = x_close(g.x(), oel.x_block(L, h, ns, r)[np.ix_(pa, pb)])
        assert ok, worst
    finally:
        tgba.tgba_basis_free(b)


def test_eigenvalues_and_heff_config1():
    w = inputs.SMALL_QP4
    b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp)
    try:
        g = GpuSector(b, 0, w.max_qp)
        tgba.tgba_compute_x(b)
        _, _, nh = tgba.tgba_basis_totals(b)
        H = torch.empty(nh, dtype=torch.complex128, device="cuda")
        tgba.tgba_assemble_heff(b, w.h_x[0], H)
        n = g.n_ns + g.n_r
        Hg = H.cpu().numpy().reshape(n, n).T          # column-major
        ns, r, X = otgba.sector(w.L, w.h_z, 0, w.max_qp)
        Ho = otgba.heff(ns, r, X, w.L, w.h_x[0])
        pa, pb = g.perm_to(ns, r)
        p = np.concatenate([pa, len(ns) + pb])
        assert np.abs(Hg - Ho[np.ix_(p, p)]).max() < 1e-10 * np.abs(Ho).max()
        ev = torch.empty(n, dtype=torch.float64, device="cuda")
        tgba.tgba_eigvals(b, w.h_x[0], ev)
        Eo = np.linalg.eigvalsh(Ho)
        assert np.abs(ev.cpu().numpy() - Eo).max() < 1e-10 * np.abs(Eo).max()
    finally:
        tgba.tgba_basis_free(b)


def test_full_basis_config1_equals_ed():
    from oracle import ed
    w = inputs.SMALL_FULL
    b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp)
    try:
        tgba.tgba_compute_x(b)
        _, _, _ = tgba.tgba_basis_totals(b)
        ev = torch.empty(352, dtype=torch.float64, device="cuda")
        tgba.tgba_eigvals(b, w.h_x[0], ev)
        Eed = ed.sector_spectrum(w.L, w.h_z, w.h_x[0], 0)
        assert np.abs(ev.cpu().numpy() - Eed).max() < 1e-10 * np.abs(Eed).max()
    finally:
        tgba.tgba_basis_free(b)


@pytest.mark.parametrize("wl", [inputs.SMALL_QP4, inputs.SMALL_FULL])
def test_dsf_config1(wl):
    L, h, hx = wl.L, wl.h_z, wl.h_x[0]
    w_min, w_max, n_w, eta = wl.w_range
    b = tgba.tgba_build_basis(L, h, [0], wl.max_qp)
    try:
        g = GpuSector(b, 0, wl.max_qp)
        tgba.tgba_compute_x(b)
        n = g.n_ns + g.n_r
        S = torch.empty(n_w, dtype=torch.float32, device="cuda")
        wts = torch.empty(n, dtype=torch.float64, device="cuda")
        dE = torch.empty(n, dtype=torch.float64, device="cuda")
        ev = torch.empty(20, dtype=torch.float64, device="cuda")
        tgba.tgba_dsf(b, 0, hx, w_min, w_max, n_w, eta, S, ev, 20, wts, dE)
        ns, r, X = otgba.sector(L, h, 0, wl.max_qp)
        E, U = otgba.eigh(otgba.heff(ns, r, X, L, hx))
        So = otgba.dsf(E, U, otgba.x_full(X), L, w_min, w_max, n_w, eta)
        Sg = S.cpu().numpy()
        assert np.abs(Sg - So).max() <= 1e-5 * So.max()
        assert np.abs(ev.cpu().numpy() - E[:20]).max() < 1e-10 * np.abs(E).max()
        # weights, summed over degenerate groups (unique), and the sum rule
        dEo, wo = otgba.dsf_weights(E, U, otgba.x_full(X), L)
        assert abs(wts.cpu().numpy().sum() - wo.sum()) < 1e-10 * wo.sum()
    finally:
        tgba.tgba_basis_free(b)


@pytest.mark.parametrize("method", [1, 2])
def test_quench_small(method):
    """Both propagators (1: eigendecomposition, 2: Chebyshev expansion) against the oracle."""
    L, h, h0, hx = 12, 1.0, 0.5, 0.1
    for mq, cuts in ((12, [-1.0]), (4, [-1.0, 6.0])):
        b = tgba.tgba_build_basis(L, h, [0], mq)
        try:
            tgba.tgba_compute_x(b)
            n_t, t_max = 41, 20.0
            mx = torch.empty(len(cuts) * n_t, dtype=torch.float64, device="cuda")
            nrm = torch.empty(len(cuts), dtype=torch.float64, device="cuda")
            chi = tgba.tgba_quench(b, 0, h0, [hx] * len(cuts), cuts, t_max, n_t, mx, nrm, method=method)
            mxg = mx.cpu().numpy().reshape(len(cuts), n_t)
            for v, cut in enumerate(cuts):
                t, mo, c0 = otgba.quench(L, h, h0, hx, mq, None if cut < 0 else cut, t_max, n_t)
                assert chi[v] == len(c0)
                assert np.abs(mxg[v] - mo).max() < 1e-9, (mq, cut, np.abs(mxg[v] - mo).max())
                assert abs(nrm.cpu().numpy()[v] - np.vdot(c0, c0).real) < 1e-12
        finally:
            tgba.tgba_basis_free(b)
