"""Pins of the oracle's single-particle data and basis enumeration.

  * the multiset of basis energies of each parity equals the exact spectrum of H0 (Eq. 3 at
    h_par = 0) restricted to that fermion parity, found by exact diagonalisation;
  * the number of states of every momentum sector equals the Burnside count
    (1/N) sum_x e^{iKx} 2^gcd(x, N) of spin configurations with momentum K;
  * the pruned depth-first enumeration equals a brute-force scan of all subsets.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import basis as bs
from oracle import ed
from oracle import modes as md


@pytest.mark.parametrize("N,h", [(6, 0.4), (8, 1.0), (8, 1.8), (10, 0.7)])
def test_energies_match_exact_h0_spectrum(N, h):
    H = ed.spin_hamiltonian(N, h, 0.0).toarray()
    Q = np.ones(1 << N)
    for j in range(1, N + 1):
        Q *= 2.0 * ((np.arange(1 << N) >> (j - 1)) & 1) - 1.0
    for parity, q in ((md.NS, 1.0), (md.R, -1.0)):
        idx = np.where(Q == q)[0]
        exact = np.linalg.eigvalsh(H[np.ix_(idx, idx)])
        ours = sorted(s.E for m in range(N) for s in bs.parity_states(N, h, parity, m, N))
        assert len(ours) == len(exact) == 1 << (N - 1)
        assert np.abs(np.array(ours) - exact).max() < 1e-11


def burnside(N, m):
    K = 2 * math.pi * m / N
    return round(sum((np.exp(1j * K * x) * 2 ** math.gcd(x, N)).real for x in range(N)) / N)


@pytest.mark.parametrize("N", [4, 6, 8, 10, 12])
def test_sector_sizes_are_burnside_counts(N):
    for m in range(N):
        ns, r = bs.sector_basis(N, 1.0, m, N)
        assert len(ns) + len(r) == burnside(N, m)
    ns, r = bs.sector_basis(12, 1.0, 0, 12)
    assert (len(ns), len(r)) == (180, 172)       # 352 binary necklaces of length 12


@pytest.mark.parametrize("N,h,m,mq,cut", [(10, 1.0, 0, 4, 9.0), (10, 1.4, 3, 6, 12.0), (12, 0.5, 5, 6, 10.0)])
def test_pruned_enumeration_equals_bruteforce(N, h, m, mq, cut):
    e_ns = md.vacuum_energy(N, md.NS, h)
    for parity in (md.NS, md.R):
        ex = md.excitation_energy(N, parity, h)
        nl = md.momenta_n(N, parity)
        brute = set()
        for M in range(0, mq + 1, 2):
            for sel in itertools.combinations(range(N), M):
                E = md.vacuum_energy(N, parity, h) + sum(ex[list(sel)])
                if (sum(nl[list(sel)]) - 2 * m) % (2 * N) == 0 and E - e_ns <= cut + 1e-9:
                    brute.add(sel)
        got = {s.modes for s in bs.parity_states(N, h, parity, m, mq, cut)}
        assert got == brute


def test_ordering_and_cap():
    ns = bs.parity_states(12, 1.0, md.NS, 0, 6, None, 40)
    keys = [(s.E, s.M, s.modes) for s in ns]
    assert keys == sorted(keys) and len(ns) == 40
    full = bs.parity_states(12, 1.0, md.NS, 0, 6)
    assert [s.modes for s in full[:40]] == [s.modes for s in ns]


def test_dispersion_closed_forms():
    # h = 0: eps = 2 for k != pi, eps_pi = -2; vacua degenerate at -N
    N = 10
    assert np.allclose(md.eps(N, md.NS, 0.0), 2.0)
    e = md.eps(N, md.R, 0.0)
    assert np.allclose(e[:-1], 2.0) and e[-1] == -2.0
    assert md.vacuum_energy(N, md.NS, 0.0) == pytest.approx(-N)
    assert md.vacuum_energy(N, md.R, 0.0) == pytest.approx(-N)
    # theta is odd in k and lies in (-pi, pi]
    th = md.theta(N, md.NS, 0.7)
    assert np.allclose(th, -th[::-1]) and np.all(np.abs(th) <= math.pi)
