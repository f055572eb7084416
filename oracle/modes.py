"""Single-particle data of the transverse-field Ising chain (Eq. 4-7 and Eq. S3).

Test infrastructure only.

Conventions (each a reading of the paper, stated once here):
  * N even, sites j = 1..N, c_j = N^{-1/2} sum_k e^{ikj} c_k (Eq. 6 text).
  * Momentum k = pi n / N.  NS (Q = +1): n odd in [-(N-1), N-1].  R (Q = -1): n even in
    [-(N-2), N], n = N being k = pi.  Modes are indexed in ascending n.
  * eps_k = 2 sqrt((h-1)^2 + 4 h cos^2(k/2)) for k != pi and eps_pi = 2(h-1), signed (Eq. 7).
  * theta_k = sign(k) arccos(2(h + cos k)/eps_k), sign(0) = 0, and theta_pi = 0 (the value
    of the formula for h != 1, also taken at h = 1 where it reads 0/0).
  * |0>_NS = n_NS d_{k_N}...d_{k_1}|0>_c, the product in descending k from the left
    (k_1 < ... < k_N), n_NS = prod_{0<k} 1/cos(theta_k/2) (Eq. S3).  |0>_R the same over R
    modes without pi.
  * With theta_pi = 0, d_pi = -i c_pi^dag, so |0>_R has the d_pi quasiparticle present.  The
    R "excitation" at pi is therefore c_pi^dag (removing that quasiparticle); it costs
    -eps_pi = 2(1-h).  All other excitations are d_k^dag and cost eps_k.
  * E_NS,vac = -1/2 sum_{k in NS} eps_k,  E_R,vac = -1/2 sum_{k in R, k != pi} eps_k + eps_pi/2.
  * A general coupling J > 0 enters by the exact rescaling H(J, h, h_x) = J H(1, h/J, h_x/J).
"""
import math

import numpy as np

NS, R = 0, 1


def momenta_n(N, parity):
    """Integer labels n (k = pi n / N) of the modes of one parity sector, ascending."""
    if N < 2 or N % 2:
        raise ValueError("N must be even and >= 2")
    if parity == NS:
        return np.arange(-(N - 1), N, 2, dtype=np.int64)
    return np.arange(-(N - 2), N + 1, 2, dtype=np.int64)


def eps(N, parity, h):
    """eps_k per Eq. 7, eps_pi signed."""
    n = momenta_n(N, parity)
    k = math.pi * n / N
    e = 2.0 * np.sqrt((h - 1.0) ** 2 + 4.0 * h * np.cos(k / 2.0) ** 2)
    e[n == N] = 2.0 * (h - 1.0)
    return e


def theta(N, parity, h):
    """Bogoliubov angles theta_k = sign(k) arccos(2(h + cos k)/eps_k); theta_pi = 0."""
    n = momenta_n(N, parity)
    k = math.pi * n / N
    e = eps(N, parity, h)
    out = np.zeros(len(n))
    for i in range(len(n)):
        if n[i] == N or n[i] == 0:
            continue
        x = 2.0 * (h + math.cos(k[i])) / e[i]
        x = min(1.0, max(-1.0, x))
        out[i] = math.copysign(math.acos(x), k[i])
    return out


def excitation_energy(N, parity, h):
    """Energy cost of each excitation operator (eps_k; -eps_pi for the R mode at pi)."""
    e = eps(N, parity, h).copy()
    n = momenta_n(N, parity)
    e[n == N] = -e[n == N]
    return e


def vacuum_energy(N, parity, h):
    n = momenta_n(N, parity)
    e = eps(N, parity, h)
    if parity == NS:
        return -0.5 * float(np.sum(e))
    return -0.5 * float(np.sum(e[n != N])) + 0.5 * float(e[n == N][0])


def vacuum_norm(N, parity, h):
    """n_P = prod_{0<k in P} 1/cos(theta_k/2)  (Eq. S3; the k = pi factor is 1)."""
    n = momenta_n(N, parity)
    th = theta(N, parity, h)
    return float(np.prod(1.0 / np.cos(th[n > 0] / 2.0)))
