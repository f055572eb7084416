"""S(k=0, w) on the frequency grid of the L = 40 benchmark workload (4096 points in [0, 10],
eta = 0.01; Eq. 8-9) against the oracle, on the largest k = 0 basis whose direct Pfaffians the
oracle finishes in minutes: L = 18, h_z = 1, h_x = 0.1, all 2429 states with M <= 6.  The oracle's
values are stored by tests/golden/make_dsf_L18.py (X by direct Pfaffians of the whole operator
string, dense eigenpairs, an FP64 Lorentzian sum).

Compared: every excitation energy E_a - E_0 (FP64, 1e-10 of the spectral scale), the weights
w_a = L |<psi_0|sigma^x_1|psi_a>|^2 summed over each degenerate level (only those sums are
independent of the eigenvector basis inside a level; 1e-10 of the largest weight), and S(w)
element by element against the FP32 tolerance max |S32 - S64| <= 1e-4 max S64 at eta = 0.01."""
import os

import numpy as np
import pytest
import torch

from paper_2410_04204_gb300 import tgba

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dsf_L18.txt")
L, H, HX, MAX_QP = 18, 1.0, 0.1, 6
W_MIN, W_MAX, N_W, ETA = 0.0, 10.0, 4096, 0.01


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def golden():
    with open(GOLDEN) as f:
        rows = [line.split() for line in f if not line.startswith("#")]
    n = int(rows[0][1])
    dE = np.array([float(r[0]) for r in rows[1:1 + n]])
    w = np.array([float(r[1]) for r in rows[1:1 + n]])
    n_w = int(rows[1 + n][1])
    S = np.array([float(r[0]) for r in rows[2 + n:2 + n + n_w]])
    return dE, w, S


def level_sums(dE, w, tol):
    """Sums of w over clusters of dE closer than tol (dE ascending)."""
    cuts = np.flatnonzero(np.diff(dE) > tol) + 1
    return np.add.reduceat(w, np.concatenate([[0], cuts])), len(cuts) + 1


def test_dsf_against_oracle_on_the_L40_grid():
    dE_o, w_o, S_o = golden()
    b = tgba.tgba_build_basis(L, H, [0], MAX_QP)
    try:
        info = tgba.tgba_basis_info(b, 0, MAX_QP)
        n = info["n_ns"] + info["n_r"]
        assert n == len(dE_o)
        tgba.tgba_compute_x(b)
        S = torch.empty(N_W, dtype=torch.float32, device="cuda")
        wts = torch.empty(n, dtype=torch.float64, device="cuda")
        dE = torch.empty(n, dtype=torch.float64, device="cuda")
        tgba.tgba_dsf(b, 0, HX, W_MIN, W_MAX, N_W, ETA, S, None, 0, wts, dE)
        dg, wg = dE.cpu().numpy(), wts.cpu().numpy()
        order = np.argsort(dg, kind="stable")
        dg, wg = dg[order], wg[order]
        scale = max(1.0, np.abs(dE_o).max())
        assert np.abs(dg - dE_o).max() < 1e-10 * scale
        tol = 1e-7
        so, no = level_sums(dE_o, w_o, tol)
        sg, ng = level_sums(dg, wg, tol)
        assert no == ng
        assert np.abs(sg - so).max() < 1e-10 * w_o.max()
        Sg = S.cpu().numpy().astype(np.float64)
        assert np.abs(Sg - S_o).max() <= 1e-4 * S_o.max()
    finally:
        tgba.tgba_basis_free(b)
