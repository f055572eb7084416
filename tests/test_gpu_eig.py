"""Native batched eigenvalue solver (Householder tridiagonalisation by thread-block clusters,
then bisection on Sturm counts) through the C ABI, against exact diagonalisation of the spin
chain (Eq. 1 on a complete basis), against LAPACK on the same H_eff (Eq. 2) and against the
library solver.  The batch size decides how many CTAs share a matrix (up to 16; a single CTA
looping over matrices when there are more matrices than SMs), so the cases below cover one,
several and more-than-CTAs batches."""
import numpy as np
import pytest
import torch

from oracle import ed
from paper_2410_04204_gb300 import inputs, tgba
from tests.gpu_helpers import GpuSector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _sizes(b):
    return [a + c for a, c in tgba.tgba_sector_sizes(b)]


def _ed_spectra(L, h, hx, sectors):
    H = ed.spin_hamiltonian(L, h, hx)
    out = {}
    for m in sectors:
        B = ed.momentum_basis(L, m)
        out[m] = np.linalg.eigvalsh(B.conj().T @ (H @ B))
    return out


def _evals(b, fields, method):
    n = sum(_sizes(b))
    ev = torch.empty(len(fields) * n, dtype=torch.float64, device="cuda")
    tgba.tgba_eigvals(b, fields, ev, method=method)
    return ev.cpu().numpy().reshape(len(fields), n)


@pytest.mark.parametrize("L,fields", [(12, [0.0, 0.3]), (4, [0.1]), (6, [0.0, 0.2, 1.5])])
def test_native_complete_basis_equals_ed(L, fields):
    """Complete basis: the spectrum of every momentum sector equals exact diagonalisation, at
    h_x = 0 (diagonal matrices, no reflection needed), small and large h_x; L = 4 and 6 give
    sectors of 1 to 12 states."""
    h = 1.0
    sectors = list(range(L))
    b = tgba.tgba_build_basis(L, h, sectors, L)
    try:
        tgba.tgba_compute_x(b)
        sizes = _sizes(b)
        off = np.concatenate([[0], np.cumsum(sizes)])
        ev = _evals(b, fields, 1)
        for f, hx in enumerate(fields):
            exact = _ed_spectra(L, h, hx, sectors)
            for s, m in enumerate(sectors):
                got = ev[f, off[s]:off[s + 1]]
                assert len(got) == len(exact[m])
                assert np.abs(got - exact[m]).max() < 1e-10 * max(1.0, np.abs(exact[m]).max()), (hx, m)
    finally:
        tgba.tgba_basis_free(b)


def test_native_single_matrix_and_full_batch_match_library():
    """One matrix (a group of 16 CTAs) and 312 matrices (more than the 304 CTAs of two per SM:
    single CTAs that loop over matrices) against cuSOLVER."""
    L, h = 12, 1.0
    b = tgba.tgba_build_basis(L, h, [0], L)
    try:
        tgba.tgba_compute_x(b)
        e1, e2 = _evals(b, [0.1], 1), _evals(b, [0.1], 2)
        assert np.abs(e1 - e2).max() < 1e-10 * np.abs(e2).max()
        exact = _ed_spectra(L, h, 0.1, [0])[0]
        assert np.abs(e1[0] - exact).max() < 1e-10 * np.abs(exact).max()
    finally:
        tgba.tgba_basis_free(b)
    b = tgba.tgba_build_basis(L, h, list(range(L)), L)
    try:
        tgba.tgba_compute_x(b)
        fields = list(np.linspace(0.02, 0.5, 26))          # 26 x 12 = 312 matrices, more than the CTAs
        e1, e2 = _evals(b, fields, 1), _evals(b, fields, 2)
        assert np.abs(e1 - e2).max() < 1e-10 * np.abs(e2).max()
    finally:
        tgba.tgba_basis_free(b)


def test_native_L24_all_sectors_against_lapack():
    """The 24-sector L = 24 workload (48 matrices of n ~ 1900: many 32 x 16 blocks and a ragged
    tail): every eigenvalue against cuSOLVER, and two sectors against LAPACK's eigvalsh of the
    same H_eff = diag(E0) - L h_x [[0, X], [X^H, 0]] built on the host from the exported X."""
    w = inputs.SECTORS_L24
    b = tgba.tgba_build_basis(w.L, w.h_z, w.sectors, w.max_qp, w.e_cut)
    try:
        tgba.tgba_compute_x(b)
        sizes = _sizes(b)
        off = np.concatenate([[0], np.cumsum(sizes)])
        e1, e2 = _evals(b, w.h_x, 1), _evals(b, w.h_x, 2)
        scale = np.abs(e2).max()
        assert np.abs(e1 - e2).max() < 1e-10 * scale
        for s in (0, 7):
            g = GpuSector(b, s, w.max_qp)
            X = g.x()
            a, r = g.n_ns, g.n_r
            for f, hx in enumerate(w.h_x):
                H = np.zeros((a + r, a + r), np.complex128)
                H[np.arange(a + r), np.arange(a + r)] = g.E0
                H[:a, a:] = -w.L * hx * X
                H[a:, :a] = H[:a, a:].conj().T
                ref = np.linalg.eigvalsh(H)
                assert np.abs(e1[f, off[s]:off[s + 1]] - ref).max() < 1e-10 * scale
    finally:
        tgba.tgba_basis_free(b)


def test_native_rejects_oversized_and_reports_overflow():
    w = inputs.DSF_L40                                    # k = 0 sector of ~1e4 states
    b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp, w.e_cut)
    try:
        tgba.tgba_compute_x(b)
        ev = torch.empty(sum(_sizes(b)), dtype=torch.float64, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_eigvals(b, 0.1, ev, method=1)
        assert e.value.code == tgba.TGBA_EINVAL
    finally:
        tgba.tgba_basis_free(b)
    b = tgba.tgba_build_basis(8, 1.0, [0], 8)
    try:
        tgba.tgba_compute_x(b)
        ev = torch.empty(sum(_sizes(b)), dtype=torch.float64, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:           # off-diagonal entries overflow to inf
            tgba.tgba_eigvals(b, 1e308, ev, method=1)
        assert e.value.code == tgba.TGBA_ENUMERIC
        tgba.tgba_eigvals(b, 0.1, ev, method=1)          # the handle stays usable
        assert np.isfinite(ev.cpu().numpy()).all()
    finally:
        tgba.tgba_basis_free(b)


def test_bounded_group_wait_times_out_and_handle_survives():
    """Failure detection without a GPU fault: one CTA of the group that shares a matrix leaves
    before its first barrier (an arrival that never comes), the group's waits give up after a
    short poll limit, and the call returns TGBA_ETIMEOUT; the same handle then solves normally
    and matches the library solver.  One L = 24 sector gives one matrix and a group of 16 CTAs."""
    w = inputs.SECTORS_L24
    b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp, w.e_cut)
    try:
        tgba.tgba_compute_x(b)
        n = sum(_sizes(b))
        ev = torch.empty(n, dtype=torch.float64, device="cuda")
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_eigvals_wait_check(b, [0.1], ev, spin_limit=1 << 12, withhold_matrix=0, withhold_rank=3)
        assert e.value.code == tgba.TGBA_ETIMEOUT
        with pytest.raises(tgba.TgbaError) as e:       # a withheld CTA outside the group
            tgba.tgba_eigvals_wait_check(b, [0.1], ev, spin_limit=1 << 12, withhold_matrix=0, withhold_rank=99)
        assert e.value.code == tgba.TGBA_EINVAL
        tgba.tgba_eigvals_wait_check(b, [0.1], ev, spin_limit=1 << 24)   # nothing withheld: normal solve
        got = ev.cpu().numpy()
        ref = _evals(b, [0.1], 2)[0]
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
        assert np.array_equal(_evals(b, [0.1], 1)[0], got)
    finally:
        tgba.tgba_basis_free(b)
