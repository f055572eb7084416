"""Exact diagonalisation and Fock-space brute force for small chains.

Test infrastructure only: these routines pin the rest of the oracle to the spin model itself
(Eq. 3) without any Gaussian-state machinery.

Occupation/spin basis: integer s, bit j-1 is site j; bit set <-> sigma^z_j = +1 <-> the
Jordan-Wigner fermion n_j = 1 (sigma^z = 2 c^dag c - 1).
"""
import math

import numpy as np
import scipy.sparse as sp


def _bit(s, j):
    return (s >> (j - 1)) & 1


def pauli_x(N, j):
    d = 1 << N
    s = np.arange(d)
    return sp.csr_matrix((np.ones(d), (s ^ (1 << (j - 1)), s)), shape=(d, d))


def pauli_z(N, j):
    d = 1 << N
    s = np.arange(d)
    return sp.diags(2.0 * ((s >> (j - 1)) & 1) - 1.0).tocsr()


def spin_hamiltonian(N, h, h_x):
    """H = -sum sx_j sx_{j+1} - h sum sz_j - h_x sum sx_j, periodic (Eq. 3)."""
    d = 1 << N
    H = sp.csr_matrix((d, d))
    for j in range(1, N + 1):
        jn = j % N + 1
        H = H - pauli_x(N, j) @ pauli_x(N, jn) - h * pauli_z(N, j) - h_x * pauli_x(N, j)
    return H.tocsr()


def magnetisation_op(N):
    """(1/N) sum_j sigma^x_j."""
    d = 1 << N
    M = sp.csr_matrix((d, d))
    for j in range(1, N + 1):
        M = M + pauli_x(N, j)
    return (M / N).tocsr()


def translate(N, s):
    """T moves the spin on site j to site j+1 (cyclically)."""
    top = (s >> (N - 1)) & 1
    return ((s << 1) & ((1 << N) - 1)) | top


def momentum_basis(N, m):
    """Orthonormal columns spanning T-eigenstates with T|v> = e^{-iK}|v>, K = 2 pi m / N."""
    K = 2 * math.pi * m / N
    d = 1 << N
    seen = np.zeros(d, dtype=bool)
    cols = []
    for s0 in range(d):
        if seen[s0]:
            continue
        orbit = [s0]
        s = translate(N, s0)
        while s != s0:
            orbit.append(s)
            s = translate(N, s)
        for s in orbit:
            seen[s] = True
        v = np.zeros(d, dtype=np.complex128)
        for x in range(N):                       # sum_x e^{-iKx} T^x |s0>, T^x|s0> = orbit[x mod P]
            v[orbit[x % len(orbit)]] += np.exp(-1j * K * x)
        nv = np.linalg.norm(v)
        if nv > 1e-9:
            cols.append(v / nv)
    return np.array(cols).T


def sector_spectrum(N, h, h_x, m):
    B = momentum_basis(N, m)
    Hk = B.conj().T @ (spin_hamiltonian(N, h, h_x) @ B)
    return np.linalg.eigvalsh(Hk)


def dsf_weights(N, h, h_x):
    """Exact (E_a - E_0, |<psi_a| sigma^x_{k=0} |psi_0>|^2) in the k = 0 sector,
    sigma^x_{k=0} = N^{-1/2} sum_j sigma^x_j (Eq. 8-9)."""
    B = momentum_basis(N, 0)
    Hk = B.conj().T @ (spin_hamiltonian(N, h, h_x) @ B)
    E, V = np.linalg.eigh(Hk)
    Sx = B.conj().T @ (magnetisation_op(N) @ B) * math.sqrt(N)
    amp = V.conj().T @ (Sx @ V[:, 0])
    return E - E[0], np.abs(amp) ** 2


def sector_dsf_weights(N, h, h_x, m):
    """Exact (E_a - E_0, N |<psi_a| sigma^x_1 |psi_0>|^2) for every eigenstate a of momentum
    sector m, with psi_0 the ground state of the K = 0 sector.  Translation invariance makes
    this |<psi_a| sigma^x_k |psi_0>|^2 with sigma^x_k = N^{-1/2} sum_j e^{-ikj} sigma^x_j at the
    momentum k of sector m (the weights of S(k, w), Eq. 8-9); written with sigma^x_1 so that no
    Fourier sign convention enters."""
    H = spin_hamiltonian(N, h, h_x)
    B0 = momentum_basis(N, 0)
    E0, V0 = np.linalg.eigh(B0.conj().T @ (H @ B0))
    psi0 = B0 @ V0[:, 0]
    Bm = momentum_basis(N, m)
    Em, Vm = np.linalg.eigh(Bm.conj().T @ (H @ Bm))
    amp = Vm.conj().T @ (Bm.conj().T @ (pauli_x(N, 1) @ psi0))
    return Em - E0[0], N * np.abs(amp) ** 2


def quench_magnetisation(N, h0, h, h_x, t):
    """Exact <sigma^x>(t) from (|GS_Q=+1(h0)> + s|GS_Q=-1(h0)>)/sqrt 2 in the k = 0 sector,
    s chosen to make <sigma^x>(0) > 0, evolved with H(h, h_x)."""
    B = momentum_basis(N, 0)
    Q = np.ones(1 << N)
    for j in range(1, N + 1):
        Q = Q * (2.0 * ((np.arange(1 << N) >> (j - 1)) & 1) - 1.0)
    Mx = B.conj().T @ (magnetisation_op(N) @ B)
    H0 = B.conj().T @ (spin_hamiltonian(N, h0, 0.0) @ B)
    E0, V0 = np.linalg.eigh(H0)
    qv = np.einsum("ia,i,ia->a", np.conj(B @ V0), Q, B @ V0).real
    ns = V0[:, np.where(qv > 0.5)[0][0]]
    r = V0[:, np.where(qv < -0.5)[0][0]]
    z = np.vdot(ns, Mx @ r)
    phi0 = (ns + (np.conj(z) / abs(z)) * r) / math.sqrt(2.0)
    Hk = B.conj().T @ (spin_hamiltonian(N, h, h_x) @ B)
    E, V = np.linalg.eigh(Hk)
    a = V.conj().T @ phi0
    psi = V @ (np.exp(-1j * np.outer(E, t)) * a[:, None])
    return np.einsum("it,ij,jt->t", np.conj(psi), Mx, psi).real


def quench_correlators(N, h0, h, h_x, t, j_max):
    """Exact connected <sigma^x_1 sigma^x_{j+1}>(t) - <sigma^x_1>(t) <sigma^x_{j+1}>(t) for
    j = 1..j_max after the quench of quench_magnetisation (rows: j; columns: t)."""
    B = momentum_basis(N, 0)
    Q = np.ones(1 << N)
    for j in range(1, N + 1):
        Q = Q * (2.0 * ((np.arange(1 << N) >> (j - 1)) & 1) - 1.0)
    Mx = B.conj().T @ (magnetisation_op(N) @ B)
    H0 = B.conj().T @ (spin_hamiltonian(N, h0, 0.0) @ B)
    E0, V0 = np.linalg.eigh(H0)
    qv = np.einsum("ia,i,ia->a", np.conj(B @ V0), Q, B @ V0).real
    ns = V0[:, np.where(qv > 0.5)[0][0]]
    r = V0[:, np.where(qv < -0.5)[0][0]]
    z = np.vdot(ns, Mx @ r)
    phi0 = (ns + (np.conj(z) / abs(z)) * r) / math.sqrt(2.0)
    Hk = B.conj().T @ (spin_hamiltonian(N, h, h_x) @ B)
    E, V = np.linalg.eigh(Hk)
    psi = B @ (V @ (np.exp(-1j * np.outer(E, t)) * (V.conj().T @ phi0)[:, None]))   # full space
    s1 = pauli_x(N, 1)
    m1 = np.einsum("it,it->t", np.conj(psi), s1 @ psi).real
    out = np.zeros((j_max, len(t)))
    for j in range(1, j_max + 1):
        op = s1 @ pauli_x(N, j + 1)
        mj = np.einsum("it,it->t", np.conj(psi), pauli_x(N, j + 1) @ psi).real
        out[j - 1] = np.einsum("it,it->t", np.conj(psi), op @ psi).real - m1 * mj
    return out


# ---------------------------------------------------------------- Fock-space brute force

def fermion_c(N, j):
    """c_j with the Jordan-Wigner sign (-1)^{sum_{l<j} n_l}."""
    d = 1 << N
    rows, cols, vals = [], [], []
    for s in range(d):
        if _bit(s, j):
            sign = (-1) ** bin(s & ((1 << (j - 1)) - 1)).count("1")
            rows.append(s ^ (1 << (j - 1)))
            cols.append(s)
            vals.append(sign)
    return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(d, d))


class Fock:
    """Fermion operators of an N-site chain as explicit 2^N x 2^N matrices."""

    def __init__(self, N):
        self.N = N
        self.c = [None] + [fermion_c(N, j) for j in range(1, N + 1)]
        self.cd = [None] + [cj.conj().T.tocsr() for cj in self.c[1:]]

    def ck(self, k):
        return sum(np.exp(-1j * k * j) * self.c[j] for j in range(1, self.N + 1)) / math.sqrt(self.N)

    def ckd(self, k):
        return sum(np.exp(1j * k * j) * self.cd[j] for j in range(1, self.N + 1)) / math.sqrt(self.N)

    def dk(self, k, th):
        return math.sin(th / 2) * self.ck(k) - 1j * math.cos(th / 2) * self.ckd(-k)

    def dkd(self, k, th):
        return math.sin(th / 2) * self.ckd(k) + 1j * math.cos(th / 2) * self.ck(-k)

    def vacuum_c(self):
        v = np.zeros(1 << self.N, dtype=np.complex128)
        v[0] = 1.0
        return v
