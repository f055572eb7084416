"""Pins of the oracle's direct-Pfaffian matrix elements (Appendix A) against Fock-space
brute force, plus the parity selection rule, hermiticity and the eigen-equation of the
basis states."""
import math

import numpy as np
import pytest

from oracle import basis as bs
from oracle import ed
from oracle import elements as el
from oracle import modes as md
from oracle import native as nat
from tests import fock

CASES = [(4, 0.5), (6, 1.0), (6, 1.7), (8, 0.7), (8, 1.0)]


@pytest.fixture(scope="module")
def focks():
    return {N: ed.Fock(N) for N in (4, 6, 8)}


@pytest.mark.parametrize("N,h", CASES)
def test_states_are_normalised_h0_eigenstates(N, h, focks):
    F = focks[N]
    H0 = ed.spin_hamiltonian(N, h, 0.0)
    for m in range(N):
        for parity, st in zip((md.NS, md.R), bs.sector_basis(N, h, m, N)):
            V = fock.states(N, h, parity, st, F)
            assert np.allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-12)
            E = np.array([s.E for s in st])
            assert np.abs(H0 @ V - V * E).max() < 1e-10
            # translation eigenvalue e^{-iK}, K = 2 pi m / N  (T moves site j to j+1)
            T = np.array([ed.translate(N, s) for s in range(1 << N)])
            TV = np.zeros_like(V)
            TV[T] = V
            assert np.abs(TV - np.exp(-2j * math.pi * m / N) * V).max() < 1e-10


@pytest.mark.parametrize("N,h", CASES)
def test_elements_match_fock_space(N, h, focks):
    F = focks[N]
    sig = fock.sigma1(F)
    for m in range(N):
        ns, r = bs.sector_basis(N, h, m, N)
        Vn, Vr = fock.states(N, h, md.NS, ns, F), fock.states(N, h, md.R, r, F)
        brute = Vn.conj().T @ (sig @ Vr)
        assert np.abs(brute - el.x_block(N, h, ns, r)).max() < 1e-12
        # sigma^x_1 flips the fermion parity: NS-NS and R-R blocks vanish (Appendix A)
        assert np.abs(Vn.conj().T @ (sig @ Vn)).max() < 1e-13
        assert np.abs(Vr.conj().T @ (sig @ Vr)).max() < 1e-13


def test_hermitian_conjugate_string():
    """<R|sigma|NS> evaluated as its own operator string equals conj(<NS|sigma|R>)."""
    N, h = 8, 1.0
    ns, r = bs.sector_basis(N, h, 0, 6)
    thn, thr = md.theta(N, md.NS, h), md.theta(N, md.R, h)
    nn, nr = md.momenta_n(N, md.NS), md.momenta_n(N, md.R)
    strings, want = [], []
    X = el.x_block(N, h, ns, r)
    for a in range(0, len(ns), 3):
        for b in range(0, len(r), 3):
            s = [(nat.OP_DDAG, math.pi * nr[i] / N, thr[i]) for i in range(N) if nr[i] != N]
            for i in sorted(r[b].modes, reverse=True):
                s.append((nat.OP_C, math.pi, 0.0) if nr[i] == N else (nat.OP_D, math.pi * nr[i] / N, thr[i]))
            s.append((nat.OP_SIGMA1, 0.0, 0.0))
            for i in sorted(ns[a].modes):
                s.append((nat.OP_DDAG, math.pi * nn[i] / N, thn[i]))
            s += [(nat.OP_D, math.pi * nn[i] / N, thn[i]) for i in reversed(range(N))]
            strings.append(s)
            want.append(np.conj(X[a, b]))
    got, _ = nat.wick_batch(N, strings)
    got = got * md.vacuum_norm(N, md.NS, h) * md.vacuum_norm(N, md.R, h)
    assert np.abs(got - np.array(want)).max() < 1e-13


def test_overlaps_match_fock_space(focks):
    N, h, h0 = 6, 1.0, 0.4
    F = focks[N]
    for parity in (md.NS, md.R):
        st = bs.parity_states(N, h, parity, 0, N)
        vac0 = fock.states(N, h0, parity, [bs.State(parity, (), 0.0)], F)[:, 0]
        brute = fock.states(N, h, parity, st, F).conj().T @ vac0
        assert np.abs(brute - el.overlaps(N, h, h0, parity, st)).max() < 1e-13


@pytest.mark.parametrize("L,h", [(8, 1.0), (12, 0.7), (12, 1.3)])
def test_reduced_form_equals_direct_pfaffians(L, h):
    """The oracle's second route (Schur complement of the vacuum and sigma operators, one small
    Pfaffian per element) gives the direct Pfaffians of the whole string, which the Fock-space
    tests above pin."""
    ns, r = bs.sector_basis(L, h, 0, min(L, 6))
    pairs = [(a.modes, b.modes) for a in ns[::3] for b in r[::5]][:300]
    d = el.x_elements(L, h, pairs)
    red = el.x_elements_reduced(L, h, pairs)
    assert np.abs(d - red).max() <= 1e-12 * np.abs(d).max()
