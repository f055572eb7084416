"""Matrix elements between Gaussian basis states by direct Pfaffians (Appendix A).

Test infrastructure only.

X_ab = <phi_a^NS| (c_1 + c_1^dag) |phi_b^R> is evaluated exactly as Appendix A describes:
both states are written as products of Bogoliubov operators on the Jordan-Wigner vacuum
(Eq. S3), so the element is one vacuum expectation of 2N + M + M' linear operators, i.e.
one Pfaffian of that size (Eq. S1-S2).  The operator string, left to right, is

    d_k^dag for all NS k ascending        (the bra <0|_NS)
    d_p for p in phi_a, descending        (the bra excitations)
    c_1 + c_1^dag                         (sigma^x_1)
    e_q for q in phi_b, ascending         (the ket excitations; e_q = d_q^dag, e_pi = c_pi^dag)
    d_k for all R k != pi, descending     (the ket |0>_R)

times n_NS n_R.  By translation invariance <phi|V|phi'> = -N h_x X (Eq. S4); X vanishes
between states of equal parity.
"""
import math

import numpy as np

from . import modes as md
from . import native as nat


def _k(N, parity, i):
    return math.pi * float(md.momenta_n(N, parity)[i]) / N


def _bra_vacuum(N, parity, th):
    n = md.momenta_n(N, parity)
    return [(nat.OP_DDAG, math.pi * n[i] / N, th[i]) for i in range(N) if n[i] != N]


def _ket_vacuum(N, parity, th):
    n = md.momenta_n(N, parity)
    return [(nat.OP_D, math.pi * n[i] / N, th[i]) for i in reversed(range(N)) if n[i] != N]


def _bra_excitations(N, parity, th, sel):
    n = md.momenta_n(N, parity)
    out = []
    for i in sorted(sel, reverse=True):
        if n[i] == N:
            out.append((nat.OP_C, math.pi, 0.0))         # (c_pi^dag)^dag
        else:
            out.append((nat.OP_D, math.pi * n[i] / N, th[i]))
    return out


def _ket_excitations(N, parity, th, sel):
    n = md.momenta_n(N, parity)
    out = []
    for i in sorted(sel):
        if n[i] == N:
            out.append((nat.OP_CDAG, math.pi, 0.0))
        else:
            out.append((nat.OP_DDAG, math.pi * n[i] / N, th[i]))
    return out


def x_string(N, h, sel_ns, sel_r):
    th_ns = md.theta(N, md.NS, h)
    th_r = md.theta(N, md.R, h)
    return (_bra_vacuum(N, md.NS, th_ns) + _bra_excitations(N, md.NS, th_ns, sel_ns)
            + [(nat.OP_SIGMA1, 0.0, 0.0)]
            + _ket_excitations(N, md.R, th_r, sel_r) + _ket_vacuum(N, md.R, th_r))


def x_elements(N, h, pairs, n_threads=0, return_threads=False):
    """X for a list of (NS modes, R modes) pairs."""
    strings = [x_string(N, h, a, b) for a, b in pairs]
    vals, used = nat.wick_batch(N, strings, n_threads)
    vals = vals * (md.vacuum_norm(N, md.NS, h) * md.vacuum_norm(N, md.R, h))
    return (vals, used) if return_threads else vals


def x_elements_reduced(N, h, pairs, n_threads=0, return_threads=False):
    """X for a list of (NS modes, R modes) pairs by the reduced form (a second CPU route, used
    as the faster CPU baseline): the string of every element keeps the same vacuum and sigma
    operators F and adds its excitation operators, so with the Schur complement S of the
    contraction matrix of the string that holds ALL excitation operators (NS d_p for every NS
    mode, descending; R ones for every R mode, ascending), X = n_NS n_R Pf(A_FF) Pf(S[sel, sel]).
    Pinned to x_elements in the tests."""
    th_ns = md.theta(N, md.NS, h)
    th_r = md.theta(N, md.R, h)
    all_ns = list(range(N))
    string = (_bra_vacuum(N, md.NS, th_ns) + _bra_excitations(N, md.NS, th_ns, all_ns)
              + [(nat.OP_SIGMA1, 0.0, 0.0)]
              + _ket_excitations(N, md.R, th_r, list(range(N))) + _ket_vacuum(N, md.R, th_r))
    n_vac_ns = len(_bra_vacuum(N, md.NS, th_ns))
    is_f = [1] * n_vac_ns + [0] * N + [1] + [0] * N + [1] * (len(string) - n_vac_ns - 2 * N - 1)
    S, pf = nat.reduced_table(N, string, is_f)
    # E positions: NS mode i sits at N - 1 - i (descending block), R mode j at N + j
    sels = [[N - 1 - i for i in sorted(a, reverse=True)] + [N + j for j in sorted(b)] for a, b in pairs]
    scale = md.vacuum_norm(N, md.NS, h) * md.vacuum_norm(N, md.R, h)
    vals, used = nat.reduced_batch(S, pf, scale, sels, n_threads)
    return (vals, used) if return_threads else vals


def x_block(N, h, ns_states, r_states, n_threads=0):
    """Dense X[a, b] over two lists of basis states."""
    pairs = [(a.modes, b.modes) for a in ns_states for b in r_states]
    if not pairs:
        return np.zeros((len(ns_states), len(r_states)), dtype=np.complex128)
    return x_elements(N, h, pairs, n_threads).reshape(len(ns_states), len(r_states))


def sxsx_middle(j):
    """sigma^x_1 sigma^x_{j+1} after the Jordan-Wigner map: with A_l = c_l^dag + c_l and
    B_l = c_l^dag - c_l (so 1 - 2 n_l = A_l B_l and sigma^x_1 = A_1),
    sigma^x_1 sigma^x_{j+1} = A_1 (A_1 B_1)(A_2 B_2)...(A_j B_j) A_{j+1} = B_1 A_2 B_2 ... B_j A_{j+1}."""
    out = []
    for l in range(1, j + 1):
        out.append((nat.OP_MAJ_B, float(l), 0.0))
        out.append((nat.OP_MAJ_A, float(l + 1), 0.0))
    return out


def z_string(N, h, parity, sel_a, sel_b, j):
    """<phi_a| sigma^x_1 sigma^x_{j+1} |phi_b> between two states of the same parity: the
    string of X with the bra and ket vacua of that parity and the 2j Majoranas of
    sxsx_middle(j) in place of sigma^x_1."""
    th = md.theta(N, parity, h)
    return (_bra_vacuum(N, parity, th) + _bra_excitations(N, parity, th, sel_a) + sxsx_middle(j)
            + _ket_excitations(N, parity, th, sel_b) + _ket_vacuum(N, parity, th))


def z_elements(N, h, parity, j, pairs, n_threads=0):
    """<phi_a|sigma^x_1 sigma^x_{j+1}|phi_b> for a list of (modes_a, modes_b) pairs of one parity."""
    strings = [z_string(N, h, parity, a, b, j) for a, b in pairs]
    vals, _ = nat.wick_batch(N, strings, n_threads)
    return vals * md.vacuum_norm(N, parity, h) ** 2


def z_block(N, h, parity, j, states, n_threads=0):
    """Dense Z[a, b] over one list of basis states of one parity."""
    pairs = [(a.modes, b.modes) for a in states for b in states]
    if not pairs:
        return np.zeros((len(states), len(states)), dtype=np.complex128)
    return z_elements(N, h, parity, j, pairs, n_threads).reshape(len(states), len(states))


def vacuum_sigma(N, h):
    """<0_NS(h)| sigma^x_1 |0_R(h)>."""
    return x_elements(N, h, [((), ())])[0]


def overlaps(N, h, h0, parity, states, n_threads=0):
    """<phi(h)| 0_parity(h0)> for basis states of the post-quench field h, by direct Pfaffians
    (Appendix B: overlaps of eigenstates of different Hamiltonians by the Pfaffian formula)."""
    th = md.theta(N, parity, h)
    th0 = md.theta(N, parity, h0)
    strings = [_bra_vacuum(N, parity, th) + _bra_excitations(N, parity, th, s.modes) + _ket_vacuum(N, parity, th0)
               for s in states]
    if not strings:
        return np.zeros(0, dtype=np.complex128)
    vals, _ = nat.wick_batch(N, strings, n_threads)
    return vals * (md.vacuum_norm(N, parity, h) * md.vacuum_norm(N, parity, h0))
