"""Gaussian basis states built as explicit 2^N vectors in Fock space (test helper).

The states are made exactly as the paper writes them (Eq. 6 text and Eq. S3): Bogoliubov
operators applied, as sparse matrices, to the Jordan-Wigner vacuum, with the product order
and the normalisation stated in ``oracle.modes``.  No Wick contraction or Pfaffian is used,
so these vectors pin the oracle's Pfaffian route.
"""
import math

import numpy as np

from oracle import ed
from oracle import modes as md


def states(N, h, parity, st, F):
    n = md.momenta_n(N, parity)
    th = md.theta(N, parity, h)
    v = F.vacuum_c()
    for i in range(N):                 # |0>_P = n_P d_{k_N} ... d_{k_1} |0>_c: d_{k_1} acts first
        if n[i] != N:
            v = F.dk(math.pi * n[i] / N, th[i]) @ v
    v = v * md.vacuum_norm(N, parity, h)
    out = []
    for s in st:
        w = v.copy()
        for i in reversed(s.modes):    # e_{q_1} ... e_{q_M} |0>: the last operator acts first
            w = (F.ckd(math.pi) if n[i] == N else F.dkd(math.pi * n[i] / N, th[i])) @ w
        out.append(w)
    return np.array(out).T if out else np.zeros((1 << N, 0), complex)


def sigma1(F):
    return F.c[1] + F.cd[1]
