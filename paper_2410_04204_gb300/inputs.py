"""Seeded, synthetic input recipes shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: only parameters of the workloads (chain
length, fields, truncation, frequency and time grids, seeds) and seeded random draws.  It
imports nothing else from the package, so the oracle side may use it too.

Workloads follow the paper's own setups: the critical chain h_perp = 1 with a weak
longitudinal field (Fig. 1, Table 1: N = 60, h_par = 0.05), the quench (0.5, 0) -> (1, h_par)
(Fig. 2), truncation by an energy cutoff and by quasiparticle number (Method section,
Appendix B).  Sizes are those of the five benchmark configurations.
"""
from dataclasses import dataclass, field

import numpy as np

SEED = 2410


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    h_z: float
    h_x: tuple
    max_qp: int
    e_cut: float = None            # above the NS vacuum; None = no energy cutoff
    max_per_parity: int = None
    sectors: tuple = (0,)
    w_range: tuple = None          # (w_min, w_max, n_w, eta) for S(k=0, w)
    quench: dict = field(default_factory=dict)


# Config 1: L = 12, all Gaussian states of the k = 0 sector (exact), then <= 4 quasiparticles.
SMALL_FULL = Workload("L12_k0_full", 12, 1.0, (0.1,), 12, None, None, (0,), (0.0, 8.0, 1024, 0.05))
SMALL_QP4 = Workload("L12_k0_qp4", 12, 1.0, (0.1,), 4, None, None, (0,), (0.0, 8.0, 1024, 0.05))
# Config 2: L = 24, every momentum sector, M <= 6, cutoff leaving ~2000 states per sector.
SECTORS_L24 = Workload("L24_all_sectors", 24, 1.0, (0.05, 0.1), 6, 11.925, None, tuple(range(24)))
# Config 3: L = 40, k = 0, ~1e4 states, S(k=0, w) on 4096 points in [0, 10], eta = 0.01.
DSF_L40 = Workload("L40_k0_dsf", 40, 1.0, (0.1,), 6, 10.325, None, (0,), (0.0, 10.0, 4096, 0.01))
# Config 4: L = 60, k = 0, ~3e4 states (screening).
SCREEN_L60 = Workload("L60_k0_screen", 60, 1.0, (0.05,), 6, 8.984, None, (0,))
# Config 5: L = 80, k = 0, M <= 10, cutoff capped at 2e4 states per parity (quench).
QUENCH_L80 = Workload("L80_k0_quench", 80, 1.0, (0.1,), 10, 6.551, 20000, (0,),
                      quench=dict(h_z0=0.5, t_max=100.0, n_t=2000))

# Config 5 variants: 8 longitudinal fields x 8 nested energy cutoffs; cutoff i keeps the
# 5000 i lowest states of the basis (about 2500 i per parity), the last one the whole capped basis.
QUENCH_L80_HX = (0.025, 0.05, 0.075, 0.1, 0.125, 0.15, 0.175, 0.2)
QUENCH_L80_KEEP = tuple(5000 * i for i in range(1, 9))

SCREEN_TAUS = (1e-12, 1e-11, 1e-10, 1e-9, 1e-8)


def rng(tag=0):
    return np.random.default_rng([SEED, int(tag)])


def random_skew(n, count, tag=0, complex_=False):
    """Dense skew-symmetric matrices with standard-normal entries (real or complex)."""
    g = rng(tag)
    a = g.standard_normal((count, n, n))
    if complex_:
        a = a + 1j * g.standard_normal((count, n, n))
    return a - np.swapaxes(a, 1, 2)


def nested_cutoffs(energies, keep):
    """Energy cutoffs (above the NS vacuum) that keep the keep[i] lowest of the given state
    energies: midpoints between consecutive distinct levels; -1 (keep all) where keep[i] is at
    least the number of states."""
    e = np.sort(np.asarray(energies, dtype=np.float64))
    out = []
    for k in keep:
        if k >= len(e):
            out.append(-1.0)
            continue
        lo = k
        while lo > 0 and e[lo] - e[lo - 1] < 1e-6:      # not inside a degenerate level
            lo -= 1
        out.append(float(0.5 * (e[lo - 1] + e[lo])))
    return out


def sample_pairs(n_a, n_b, count, tag=0):
    """Seeded (a, b) index pairs into two lists of lengths n_a and n_b."""
    g = rng(tag)
    return np.stack([g.integers(0, n_a, count), g.integers(0, n_b, count)], axis=1)
