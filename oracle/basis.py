"""Gaussian basis of one momentum sector, with truncation (Eq. 6-7 text, Method section,
Appendix B).

Test infrastructure only.

A basis state is (parity, modes): modes are ascending mode indices (see ``modes``) of the
excitation operators applied to the parity's vacuum; their number M is even.  Its energy is
E_vac + sum of the excitation energies, the sum taken over the values sorted ascending so
that states with the same multiset of energies get bit-identical E.  Its momentum is
sum k = pi (sum n) / N mod 2 pi; sector m holds the states with sum n = 2m (mod 2N).

Truncation (readings of the paper): keep M <= max_qp (Appendix B step (i)); keep
E - E_NS,vac <= e_cut + 1e-9 if a cutoff is given ("retain the lowest energy states",
Method section); order by (E, M, modes) and keep the first max_per_parity of each parity if
a cap is given.  The sector's basis lists the NS states first, then the R states.
"""
from dataclasses import dataclass

import numpy as np

from . import modes as md


@dataclass(frozen=True)
class State:
    parity: int
    modes: tuple
    E: float

    @property
    def M(self):
        return len(self.modes)


def _energy(N, parity, h, sel):
    ex = md.excitation_energy(N, parity, h)
    return md.vacuum_energy(N, parity, h) + float(sum(sorted(float(ex[i]) for i in sel)))


def parity_states(N, h, parity, m, max_qp, e_cut=None, max_per_parity=None):
    """All kept states of one parity in sector m, sorted by (E, M, modes)."""
    ex = md.excitation_energy(N, parity, h)
    nlab = md.momenta_n(N, parity)
    e_ns = md.vacuum_energy(N, md.NS, h)
    e_vac = md.vacuum_energy(N, parity, h)
    cut = np.inf if e_cut is None else e_ns + e_cut + 1e-9
    order = sorted(range(N), key=lambda i: (ex[i], i))
    neg_suffix = np.zeros(N + 1)
    for t in range(N - 1, -1, -1):
        neg_suffix[t] = neg_suffix[t + 1] + min(0.0, ex[order[t]])
    found = []

    def dfs(t, chosen, e_part):
        # every completion of `chosen` by modes order[t:] has energy >= e_part + neg_suffix[t]
        if e_vac + e_part + neg_suffix[t] > cut + 1e-6:
            return
        if len(chosen) % 2 == 0 and (int(np.sum(nlab[list(chosen)])) - 2 * m) % (2 * N) == 0:
            found.append(tuple(sorted(chosen)))
        if len(chosen) == max_qp:
            return
        for u in range(t, N):
            i = order[u]
            chosen.append(i)
            dfs(u + 1, chosen, e_part + ex[i])
            chosen.pop()

    dfs(0, [], 0.0)
    states = []
    for sel in found:
        E = _energy(N, parity, h, sel)
        if E <= cut:
            states.append(State(parity, sel, E))
    states.sort(key=lambda s: (s.E, s.M, s.modes))
    if max_per_parity is not None:
        states = states[:max_per_parity]
    return states


def sector_basis(N, h, m, max_qp, e_cut=None, max_per_parity=None):
    """(NS states, R states) of sector m."""
    return (parity_states(N, h, md.NS, m, max_qp, e_cut, max_per_parity),
            parity_states(N, h, md.R, m, max_qp, e_cut, max_per_parity))
