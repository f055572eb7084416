"""Effective Hamiltonian, eigenpairs and the spectral sums (Eq. 2, 8-10, S4, S6).

Test infrastructure only.  Everything in float64 / complex128 with numpy/LAPACK.
"""
import math

import numpy as np

from . import basis as bs
from . import elements as el
from . import modes as md


def heff(ns, r, X, N, h_x):
    """H = diag(E^(0)) + <phi|V|phi'> with <V> = -N h_x X between NS and R states (Eq. 2, S4).
    Basis order: NS states, then R states."""
    a, b = len(ns), len(r)
    H = np.zeros((a + b, a + b), dtype=np.complex128)
    H[np.arange(a + b), np.arange(a + b)] = [s.E for s in ns] + [s.E for s in r]
    H[:a, a:] = -N * h_x * X
    H[a:, :a] = np.conj(H[:a, a:]).T
    return H


def x_full(X):
    """<phi|sigma^x_1|phi'> over the whole sector basis: [[0, X], [X^H, 0]]."""
    a, b = X.shape
    Y = np.zeros((a + b, a + b), dtype=np.complex128)
    Y[:a, a:] = X
    Y[a:, :a] = np.conj(X).T
    return Y


def eigh(H):
    """Eigenpairs, ascending; columns of U are the eigenvectors (U = M^T in Eq. 1's notation)."""
    return np.linalg.eigh(H)


def lorentzian(x, eta):
    return (eta / math.pi) / (x * x + eta * eta)


def omega_grid(w_min, w_max, n_w):
    """w_i = w_min + i (w_max - w_min)/(n_w - 1)."""
    if n_w == 1:
        return np.array([float(w_min)])
    return w_min + (w_max - w_min) * np.arange(n_w) / (n_w - 1)


def dsf_weights(E, U, Xf, N):
    """Eq. 9 at k = 0 with the matrix element of the Dynamic-structure-factor section:
    <psi_0|sigma^x_{k=0}|psi_a> = sqrt(N) sum M(0)^*_{0mu} <phi_mu|sigma^x_1|phi_nu> M_{a nu}.
    Returns (E_a - E_0, w_a = N |u_0^H Xf u_a|^2) for every eigenstate a (elastic term included)."""
    u0 = U[:, 0]
    amp = np.conj(U).T @ (Xf.conj().T @ u0)      # amp_a = u_a^H Xf^H u_0 = conj(u_0^H Xf u_a)
    w = N * np.abs(amp) ** 2
    return E - E[0], w


def dsf(E, U, Xf, N, w_min, w_max, n_w, eta):
    """S(k=0, w) = 2 pi sum_a w_a L_eta(w - (E_a - E_0)), L_eta the normalised Lorentzian."""
    dE, w = dsf_weights(E, U, Xf, N)
    om = omega_grid(w_min, w_max, n_w)
    return 2.0 * math.pi * (lorentzian(om[:, None] - dE[None, :], eta) @ w)


def x_cross(X_k0, X_0k):
    """<phi_mu|sigma^x_1|phi_nu> from the basis of sector k (rows: NS states, then R states) to
    the basis of the K = 0 sector (columns: NS, then R).  sigma^x_1 flips the fermion parity, so
    only NS_k x R_0 (X_k0 = X(NS_k, R_0)) and R_k x NS_0 (the adjoint of X_0k = X(NS_0, R_k))
    are non-zero.  For k = 0 it is x_full(X)."""
    a, b = X_k0.shape
    c, d = X_0k.shape
    Y = np.zeros((a + d, c + b), dtype=np.complex128)
    Y[:a, c:] = X_k0
    Y[a:, :c] = np.conj(X_0k).T
    return Y


def dsf_k_weights(E_k, U_k, E_0, u0, Y, N):
    """Weights of S(k, w) (Eq. 9 with the matrix element sqrt(N) e^{-ik} <psi_a|sigma^x_1|psi_0>
    that follows it): (E_a - E_0, w_a = N |u_a^H Y u_0|^2) for every eigenstate a of sector k;
    E_0, u_0: ground-state energy and vector of the K = 0 sector."""
    amp = np.conj(U_k).T @ (Y @ u0)
    return E_k - E_0, N * np.abs(amp) ** 2


def dsf_k(N, h, h_x, m, max_qp, e_cut, w_min, w_max, n_w, eta, n_threads=0):
    """S(k, w) = 2 pi sum_a w_a L_eta(w - (E_a - E_0)) at the momentum of sector m.  Returns
    (E_a - E_0, w_a, S on the w grid)."""
    ns0, r0, X0 = sector(N, h, 0, max_qp, e_cut, None, n_threads)
    E0, U0 = eigh(heff(ns0, r0, X0, N, h_x))
    nsk, rk, Xk = sector(N, h, m, max_qp, e_cut, None, n_threads)
    Ek, Uk = eigh(heff(nsk, rk, Xk, N, h_x))
    Y = x_cross(el.x_block(N, h, nsk, r0, n_threads), el.x_block(N, h, ns0, rk, n_threads))
    dE, w = dsf_k_weights(Ek, Uk, E0[0], U0[:, 0], Y, N)
    om = omega_grid(w_min, w_max, n_w)
    S = 2.0 * math.pi * (lorentzian(om[:, None] - dE[None, :], eta) @ w)
    return dE, w, S


def vacuum_phase(N, h0):
    """s with |s| = 1 that makes <Phi0|sigma^x_1|Phi0> = Re(s z) > 0, z = <0_NS|sigma_1|0_R>
    at the initial field (Fig. 2 caption: the superposition with positive magnetisation)."""
    z = el.vacuum_sigma(N, h0)
    return np.conj(z) / abs(z)


def initial_overlaps(N, h, h0, ns, r, n_threads=0):
    """c0 = <phi(h)|Phi0> with Phi0 = (|0_NS(h0)> + s |0_R(h0)>)/sqrt(2), by direct Pfaffians."""
    s = vacuum_phase(N, h0)
    c_ns = el.overlaps(N, h, h0, md.NS, ns, n_threads) / math.sqrt(2.0)
    c_r = s * el.overlaps(N, h, h0, md.R, r, n_threads) / math.sqrt(2.0)
    return np.concatenate([c_ns, c_r])


def time_grid(t_max, n_t):
    """t_i = i t_max / (n_t - 1)."""
    if n_t == 1:
        return np.zeros(1)
    return t_max * np.arange(n_t) / (n_t - 1)


def quench_coefficients(E, U, c0, t):
    """B(t) = M^T e^{-iEt} M^* c0 = U e^{-iEt} U^H c0 (Eq. 10); columns indexed by t."""
    a = np.conj(U).T @ c0
    return U @ (np.exp(-1j * np.outer(E, t)) * a[:, None])


def magnetisation(B, Xf, c0):
    """<sigma^x>(t) = B^H Xf B / ||c0||^2 (normalised by the retained weight, Quench section)."""
    val = np.einsum("it,ij,jt->t", np.conj(B), Xf, B)
    return val.real / float(np.vdot(c0, c0).real)


def sector(N, h, m, max_qp, e_cut=None, max_per_parity=None, n_threads=0):
    """Basis and X block of sector m at transverse field h."""
    ns, r = bs.sector_basis(N, h, m, max_qp, e_cut, max_per_parity)
    X = el.x_block(N, h, ns, r, n_threads)
    return ns, r, X


def quench(N, h, h0, h_x, max_qp, e_cut, t_max, n_t, max_per_parity=None, n_threads=0):
    """<sigma^x>(t) after the quench (h0, 0) -> (h, h_x) in the k = 0 sector."""
    ns, r, X = sector(N, h, 0, max_qp, e_cut, max_per_parity, n_threads)
    H = heff(ns, r, X, N, h_x)
    E, U = eigh(H)
    c0 = initial_overlaps(N, h, h0, ns, r, n_threads)
    t = time_grid(t_max, n_t)
    B = quench_coefficients(E, U, c0, t)
    return t, magnetisation(B, x_full(X), c0), c0


def ranking_key(state, c0_abs, e_ref, order):
    """Sort key of a basis state for the truncated subspace (the Quench section).  order 1:
    |<phi|Phi0>| largest first, then energy; order 0: energy.  The values are quantised
    (|c0| to 1e-10, E - e_ref to 1e-9) so that exact ties (zero overlaps of states whose momenta
    are not (-k, k) pairs, degenerate energies) do not depend on rounding; they are broken by
    (parity, M, modes)."""
    a = int(round(c0_abs * 1e10))
    e = int(round((state.E - e_ref) * 1e9))
    tail = (state.parity, state.M, tuple(state.modes))
    return ((-a, e) if order == 1 else (e,)) + tail


def ordered_subspaces(ns, r, c0, order, sizes, e_ref=0.0):
    """Nested truncated subspaces of one sector.  Returns the state ranking (NS indices
    0..len(ns)-1, R indices len(ns)..) by ranking_key and, for each size chi, the first chi
    states of it."""
    states = list(ns) + list(r)
    rank = np.array(sorted(range(len(states)), key=lambda i: ranking_key(states[i], abs(c0[i]), e_ref, order)),
                    dtype=np.int64)
    return rank, [rank[:chi] for chi in sizes]


def quench_ordered(N, h, h0, h_x, max_qp, e_cut, order, sizes, t_max, n_t, n_threads=0):
    """<sigma^x>(t), the retained weight sum |c0|^2 and the convergence metric of Eq. 11,
    eps(chi', chi) = max_t || Psi^chi(t) - Psi^chi'(t) ||, for successive nested truncations
    chi_1 < chi_2 < ... of the k = 0 sector (basis: M <= max_qp, E below e_cut), ordered by
    energy (order 0) or by the overlap with the initial state (order 1).  Returns
    (t, mx [len(sizes)][n_t], norm2 [len(sizes)], eps [len(sizes) - 1])."""
    ns, r, X = sector(N, h, 0, max_qp, e_cut, None, n_threads)
    c0 = initial_overlaps(N, h, h0, ns, r, n_threads)
    Hf = heff(ns, r, X, N, h_x)
    Xf = x_full(X)
    t = time_grid(t_max, n_t)
    _, subsets = ordered_subspaces(ns, r, c0, order, sizes, md.vacuum_energy(N, md.NS, h))
    mx, nrm, Bs = [], [], []
    for keep in subsets:
        E, U = eigh(Hf[np.ix_(keep, keep)])
        c = c0[keep]
        B = quench_coefficients(E, U, c, t)
        mx.append(magnetisation(B, Xf[np.ix_(keep, keep)], c))
        nrm.append(float(np.vdot(c, c).real))
        full = np.zeros((len(c0), len(t)), dtype=np.complex128)    # B in the whole candidate basis
        full[keep] = B
        Bs.append(full)
    eps = [float(np.sqrt((np.abs(Bs[v + 1] - Bs[v]) ** 2).sum(axis=0)).max()) for v in range(len(sizes) - 1)]
    return t, np.array(mx), np.array(nrm), np.array(eps)


def quench_correlators(N, h, h0, h_x, max_qp, e_cut, order, chi, t_max, n_t, j_max, n_threads=0):
    """Equal-time connected correlators <sigma^x_1(t) sigma^x_{j+1}(t)> - <sigma^x(t)>^2,
    j = 1..j_max, in the truncated subspace of the first chi states (order as quench_ordered),
    with the state normalised by its time-independent norm (the Quench section); translation
    invariance of the k = 0 state makes <sigma^x_{j+1}> = <sigma^x_1>.  The NS-NS and R-R
    blocks of sigma^x_1 sigma^x_{j+1} are direct Pfaffians (elements.z_block).  Returns
    (t, mx [n_t], corr [j_max][n_t])."""
    ns, r, X = sector(N, h, 0, max_qp, e_cut, None, n_threads)
    c0 = initial_overlaps(N, h, h0, ns, r, n_threads)
    _, (keep,) = ordered_subspaces(ns, r, c0, order, [chi], md.vacuum_energy(N, md.NS, h))
    Hf = heff(ns, r, X, N, h_x)
    E, U = eigh(Hf[np.ix_(keep, keep)])
    c = c0[keep]
    t = time_grid(t_max, n_t)
    B = quench_coefficients(E, U, c, t)
    nrm = float(np.vdot(c, c).real)
    mx = magnetisation(B, x_full(X)[np.ix_(keep, keep)], c)
    kns = [i for i in keep if i < len(ns)]
    kr = [i - len(ns) for i in keep if i >= len(ns)]
    pos_ns = [k for k, i in enumerate(keep) if i < len(ns)]
    pos_r = [k for k, i in enumerate(keep) if i >= len(ns)]
    corr = np.zeros((j_max, n_t))
    for j in range(1, j_max + 1):
        Zn = el.z_block(N, h, md.NS, j, [ns[i] for i in kns], n_threads)
        Zr = el.z_block(N, h, md.R, j, [r[i] for i in kr], n_threads)
        Bn, Br = B[pos_ns], B[pos_r]
        val = (np.einsum("it,ij,jt->t", np.conj(Bn), Zn, Bn) + np.einsum("it,ij,jt->t", np.conj(Br), Zr, Br)).real
        corr[j - 1] = val / nrm - mx ** 2
    return t, mx, corr

