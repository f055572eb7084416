"""Overlap-ordered quench truncation and the convergence metric of Eq. 11 (Quench section):
pinned to the identities the text states (norm of the truncated state fixed by the retained
overlaps, exact at t = 0) and to the complete basis."""
import math

import numpy as np

from oracle import ed
from oracle import tgba as otgba


def test_overlap_order_keeps_the_largest_overlaps_first():
    L, h, h0, mq = 10, 1.0, 0.5, 6
    ns, r, X = otgba.sector(L, h, 0, mq)
    c0 = otgba.initial_overlaps(L, h, h0, ns, r)
    rank, (first,) = otgba.ordered_subspaces(ns, r, c0, 1, [20])
    a_all = np.abs(c0)
    a = np.abs(c0[rank])
    assert np.all(np.diff(a) <= 1e-10)                  # non-increasing overlaps (to the key's quantum)
    assert a[0] > 0.5 and np.abs(c0[first]).min() >= np.abs(c0[rank[20:]]).max() - 1e-10


def test_eps_bounds_at_t0_and_norm():
    """||Psi^chi(t)|| = sqrt(sum_{a <= chi} |c0_a|^2) at every t (the text's norm statement), so
    eps(chi', chi) >= its value at t = 0, sqrt(sum_{chi < a <= chi'} |c0_a|^2), and >= the
    difference of the norms."""
    L, h, h0, hx, mq = 10, 1.0, 0.5, 0.1, 6
    sizes = [8, 16, 40]
    t, mx, nrm, eps = otgba.quench_ordered(L, h, h0, hx, mq, None, 1, sizes, 10.0, 41)
    ns, r, X = otgba.sector(L, h, 0, mq)
    c0 = otgba.initial_overlaps(L, h, h0, ns, r)
    rank, subsets = otgba.ordered_subspaces(ns, r, c0, 1, sizes)
    for v in range(len(sizes) - 1):
        extra = rank[sizes[v]:sizes[v + 1]]
        t0 = math.sqrt(float(np.sum(np.abs(c0[extra]) ** 2)))
        assert eps[v] >= t0 - 1e-12
        assert eps[v] >= abs(math.sqrt(nrm[v + 1]) - math.sqrt(nrm[v])) - 1e-12
    assert np.all(np.diff(nrm) >= -1e-15) and np.all(nrm <= 1 + 1e-12)


def test_complete_basis_is_exact_and_order_independent():
    """The whole basis (M <= L) in either order gives the exact quench: <sigma^x>(t) equals exact
    diagonalisation, and the two orders agree (eps between them is not defined; compare mx)."""
    L, h, h0, hx = 8, 1.0, 0.5, 0.2
    n = sum(len(x) for x in otgba.sector(L, h, 0, L)[:2])
    t, mx_e, nrm_e, _ = otgba.quench_ordered(L, h, h0, hx, L, None, 0, [n], 6.0, 31)
    _, mx_o, nrm_o, _ = otgba.quench_ordered(L, h, h0, hx, L, None, 1, [n], 6.0, 31)
    assert np.abs(mx_e - mx_o).max() < 1e-10
    assert abs(nrm_e[0] - 1.0) < 1e-10
    ref = ed.quench_magnetisation(L, h0, h, hx, t)
    assert np.abs(mx_e[0] - ref).max() < 1e-9


def test_eps_vanishes_between_equal_subspaces_and_shrinks_to_the_full_basis():
    L, h, h0, hx, mq = 8, 1.0, 0.5, 0.15, 8
    n = sum(len(x) for x in otgba.sector(L, h, 0, mq)[:2])
    _, _, _, eps = otgba.quench_ordered(L, h, h0, hx, mq, None, 1, [10, 10, 30, n], 8.0, 33)
    assert eps[0] == 0.0
    assert eps[2] < eps[1]
