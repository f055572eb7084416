"""Equal-time correlators <sigma^x_1 sigma^x_{j+1}>(t) after the quench (the correlation-function
passage of the appendix): the Majorana-string elements pinned by the
basis's orthonormality (j = 0) and Hermiticity, and the connected correlators by exact
diagonalisation on a complete basis."""
import numpy as np

from oracle import basis as obs
from oracle import ed
from oracle import elements as oel
from oracle import modes as md
from oracle import tgba as otgba


def test_empty_string_is_the_overlap_matrix():
    """j = 0: sigma^x_1 sigma^x_1 = 1, so Z is <phi_a|phi_b> = delta_ab in both parities."""
    L, h, mq = 8, 0.7, 4
    ns, r = obs.sector_basis(L, h, 0, mq)
    for P, states in ((md.NS, ns), (md.R, r)):
        Z = oel.z_block(L, h, P, 0, states)
        assert np.abs(Z - np.eye(len(states))).max() < 1e-12


def test_string_elements_hermitian_and_parity_blocks():
    L, h, mq = 8, 1.3, 4
    ns, r = obs.sector_basis(L, h, 0, mq)
    for j in (1, 3):
        for P, states in ((md.NS, ns), (md.R, r)):
            Z = oel.z_block(L, h, P, j, states)
            assert np.abs(Z - Z.conj().T).max() < 1e-12
            assert np.abs(Z).max() > 1e-3


def test_complete_basis_correlators_equal_ed():
    L, h, h0, hx, j_max = 8, 1.0, 0.5, 0.2, 4
    n = sum(len(x) for x in otgba.sector(L, h, 0, L)[:2])
    t, mx, corr = otgba.quench_correlators(L, h, h0, hx, L, None, 1, n, 5.0, 21, j_max)
    ref = ed.quench_correlators(L, h0, h, hx, t, j_max)
    assert np.abs(mx - ed.quench_magnetisation(L, h0, h, hx, t)).max() < 1e-9
    assert np.abs(corr - ref).max() < 1e-9
