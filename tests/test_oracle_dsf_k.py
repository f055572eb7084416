"""S(k, w) at every momentum (Eq. 8-9 with the cross-sector matrix element): the oracle's
cross-sector elements and weights pinned to exact diagonalisation of the spin chain, a sum rule,
and the k = 0 limit."""
import numpy as np
import pytest

from oracle import ed
from oracle import tgba as otgba


def _multiplets(dE, w, tol=1e-8):
    """(energy, summed weight) per group of degenerate levels: invariant under the choice of
    eigenvectors inside a degenerate subspace."""
    order = np.argsort(dE)
    out, cur_e, cur_w = [], None, 0.0
    for i in order:
        if cur_e is not None and dE[i] - cur_e > tol:
            out.append((cur_e, cur_w))
            cur_w = 0.0
        if cur_e is None or dE[i] - cur_e > tol:
            cur_e = dE[i]
        cur_w += w[i]
    out.append((cur_e, cur_w))
    return np.array(out)


@pytest.mark.parametrize("m", [0, 1, 3, 4])
def test_dsf_k_weights_equal_ed_on_complete_basis(m):
    """L = 8, complete basis (M <= 8): every level of sector m and its weight equal exact
    diagonalisation (weights summed over degenerate multiplets)."""
    L, h, hx = 8, 0.8, 0.15
    dE, w, _ = otgba.dsf_k(L, h, hx, m, L, None, 0.0, 1.0, 2, 0.1)
    dE_ed, w_ed = ed.sector_dsf_weights(L, h, hx, m)
    assert np.abs(np.sort(dE) - np.sort(dE_ed)).max() < 1e-10
    a, b = _multiplets(dE, w), _multiplets(dE_ed, w_ed)
    assert a.shape == b.shape
    assert np.abs(a - b).max() < 1e-9


def test_dsf_k_sum_rule():
    """Complete basis: sum over all momenta and levels of w_a = N <psi_0|(sigma^x_1)^2|psi_0> = N."""
    L, h, hx = 6, 1.2, 0.3
    total = sum(otgba.dsf_k(L, h, hx, m, L, None, 0.0, 1.0, 2, 0.1)[1].sum() for m in range(L))
    assert abs(total - L) < 1e-10


def test_dsf_k_at_k0_is_the_k0_dsf():
    """m = 0: the cross-sector form reduces to Eq. 9's k = 0 weights and spectrum."""
    L, h, hx, mq = 10, 1.0, 0.1, 4
    dE, w, S = otgba.dsf_k(L, h, hx, 0, mq, None, 0.0, 6.0, 64, 0.05)
    ns, r, X = otgba.sector(L, h, 0, mq)
    E, U = otgba.eigh(otgba.heff(ns, r, X, L, hx))
    S0 = otgba.dsf(E, U, otgba.x_full(X), L, 0.0, 6.0, 64, 0.05)
    assert np.abs(S - S0).max() < 1e-12 * S0.max()


def test_ed_sector_weights_match_the_k0_operator():
    """The ED pin itself: at m = 0, N |<psi_a|sigma^x_1|psi_0>|^2 equals |<psi_a|sigma^x_{k=0}|psi_0>|^2
    with sigma^x_{k=0} = N^{-1/2} sum_j sigma^x_j (translation invariance)."""
    L, h, hx = 8, 0.9, 0.2
    dE1, w1 = ed.sector_dsf_weights(L, h, hx, 0)
    dE2, w2 = ed.dsf_weights(L, h, hx)
    assert np.abs(dE1 - dE2).max() < 1e-12
    a, b = _multiplets(dE1, w1), _multiplets(dE2, w2)
    assert np.abs(a - b).max() < 1e-10
