"""Pins of the oracle's H_eff, spectra, S(k=0, w) and quench against exact diagonalisation
of the spin chain, the h_par = 0 limit and the Calabrese closed form (Eq. S6)."""
import numpy as np
import pytest

from oracle import basis as bs
from oracle import ed
from oracle import elements as el
from oracle import modes as md
from oracle import tgba
from paper_2410_04204_gb300 import inputs
from tests import pins


@pytest.mark.parametrize("N,h,hx", [(8, 1.0, 0.1), (8, 0.6, 0.3), (6, 1.5, 0.8)])
def test_untruncated_spectrum_equals_ed(N, h, hx):
    assert pins.spectrum_error(N, h, hx) < 1e-10


def test_config1_full_basis_equals_ed():
    w = inputs.SMALL_FULL
    assert pins.spectrum_error(w.L, w.h_z, w.h_x[0], sectors=[0]) < 1e-10


def test_diagonal_limit():
    N, h = 10, 1.0
    ns, r, X = tgba.sector(N, h, 0, 4)
    E = np.linalg.eigvalsh(tgba.heff(ns, r, X, N, 0.0))
    assert np.array_equal(np.sort([s.E for s in ns + r]), E) or np.abs(np.sort([s.E for s in ns + r]) - E).max() < 1e-13


@pytest.mark.parametrize("N,h,hx", [(8, 1.0, 0.2), (8, 0.8, 0.1)])
def test_dsf_equals_ed(N, h, hx):
    assert pins.dsf_error(N, h, hx) < 1e-10


def test_dsf_sum_rule_and_rotation_invariance():
    N, h, hx = 10, 1.0, 0.1
    ns, r, X = tgba.sector(N, h, 0, 4)
    E, U = tgba.eigh(tgba.heff(ns, r, X, N, hx))
    Xf = tgba.x_full(X)
    dE, w = tgba.dsf_weights(E, U, Xf, N)
    assert abs(w.sum() - N * np.linalg.norm(Xf @ U[:, 0]) ** 2) < 1e-10
    # a random unitary rotation inside each (near-)degenerate group of excited states leaves S invariant
    g = inputs.rng(5)
    U2 = U.copy()
    i = 1
    while i < len(E):
        j = i
        while j + 1 < len(E) and E[j + 1] - E[i] < 1e-9:
            j += 1
        if j > i:
            q, _ = np.linalg.qr(g.standard_normal((j - i + 1, j - i + 1)) + 1j * g.standard_normal((j - i + 1, j - i + 1)))
            U2[:, i:j + 1] = U[:, i:j + 1] @ q
        i = j + 1
    S1 = tgba.dsf(E, U, Xf, N, 0, 8, 300, 0.05)
    S2 = tgba.dsf(E, U2, Xf, N, 0, 8, 300, 0.05)
    assert np.abs(S1 - S2).max() < 1e-9 * S1.max()


@pytest.mark.parametrize("N,h0,h,hx", [(8, 0.5, 1.0, 0.1), (8, 0.3, 0.9, 0.2)])
def test_quench_equals_ed(N, h0, h, hx):
    assert pins.quench_error(N, h0, h, hx) < 1e-10


@pytest.mark.parametrize("N,h,h0", [(8, 1.0, 0.5), (10, 1.0, 0.5), (10, 0.8, 1.6)])
def test_overlaps_equal_calabrese_closed_form(N, h, h0):
    for parity in (md.NS, md.R):
        st = [s for m in range(N) for s in bs.parity_states(N, h, parity, m, N)]
        direct = el.overlaps(N, h, h0, parity, st)
        closed = pins.calabrese_overlaps(N, h, h0, parity, st)
        assert np.abs(direct - closed).max() < 1e-13
        # the full basis of the parity captures the whole vacuum (Quench section: sum |c|^2 <= 1)
        assert abs(np.sum(np.abs(direct) ** 2) - 1.0) < 1e-12


def test_quench_norm_is_time_independent():
    """||B(t)|| = ||c0|| in a truncated basis (Quench section)."""
    N, h, h0, hx = 12, 1.0, 0.5, 0.1
    ns, r, X = tgba.sector(N, h, 0, 4)
    E, U = tgba.eigh(tgba.heff(ns, r, X, N, hx))
    c0 = tgba.initial_overlaps(N, h, h0, ns, r)
    assert np.sum(np.abs(c0) ** 2) < 1.0
    B = tgba.quench_coefficients(E, U, c0, tgba.time_grid(50.0, 11))
    assert np.abs(np.linalg.norm(B, axis=0) - np.linalg.norm(c0)).max() < 1e-12
    t, mx, _ = tgba.quench(N, h, h0, hx, 4, None, 50.0, 11)
    assert mx[0] > 0
