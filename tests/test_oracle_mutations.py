"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one plausible error into the oracle and checks that a pin that passes for
the real oracle now fails by a wide margin."""
import numpy as np
import pytest

from oracle import elements as el
from oracle import modes as md
from oracle import tgba
from tests import pins


def test_wrong_bogoliubov_sign(monkeypatch):
    real = md.theta
    monkeypatch.setattr(md, "theta", lambda N, p, h: -real(N, p, h))
    assert pins.spectrum_error(6, 1.0, 0.3) > 1e-3


def test_wrong_pi_mode_energy(monkeypatch):
    monkeypatch.setattr(md, "excitation_energy", lambda N, p, h: md.eps(N, p, h))
    assert pins.spectrum_error(6, 0.5, 0.3) > 1e-3


def test_missing_vacuum_normalisation(monkeypatch):
    monkeypatch.setattr(md, "vacuum_norm", lambda N, p, h: 1.0)
    assert pins.spectrum_error(6, 1.0, 0.3) > 1e-3


def test_dropped_factor_n_in_v(monkeypatch):
    real = tgba.heff
    monkeypatch.setattr(tgba, "heff", lambda ns, r, X, N, hx: real(ns, r, X, 1, hx))
    assert pins.spectrum_error(6, 1.0, 0.3) > 1e-3


def test_wrong_sign_of_longitudinal_field(monkeypatch):
    """The spectrum cannot see the sign of h_par (spin flip); the quench can."""
    real = tgba.heff
    monkeypatch.setattr(tgba, "heff", lambda ns, r, X, N, hx: real(ns, r, X, N, -hx))
    assert pins.spectrum_error(6, 1.0, 0.3) < 1e-10
    assert pins.quench_error(6, 0.5, 1.0, 0.3) > 1e-3


def test_swapped_operator_order(monkeypatch):
    """Reversing the ket excitations flips the sign of states with M' = 2, 6: a change of
    gauge that no spectrum sees, but the element-wise Fock-space pin does."""
    from oracle import basis as bs
    from oracle import ed
    from tests import fock
    real = el._ket_excitations
    monkeypatch.setattr(el, "_ket_excitations", lambda N, p, th, sel: real(N, p, th, sel)[::-1])
    N, h = 6, 1.0
    F = ed.Fock(N)
    ns, r = bs.sector_basis(N, h, 0, N)
    brute = fock.states(N, h, md.NS, ns, F).conj().T @ (fock.sigma1(F) @ fock.states(N, h, md.R, r, F))
    assert np.abs(brute - el.x_block(N, h, ns, r)).max() > 1e-3
    assert pins.spectrum_error(N, h, 0.3, sectors=[0]) < 1e-10
