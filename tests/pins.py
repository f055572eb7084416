"""Pin checks of the oracle against exact diagonalisation (test helper).

Each function returns an error measure; the tests assert it is tiny for the oracle as it
stands and large for the oracle with a planted mistake."""
import math

import numpy as np

from oracle import basis as bs
from oracle import ed
from oracle import elements as el
from oracle import modes as md
from oracle import tgba


def spectrum_error(N, h, h_x, sectors=None):
    """max |TGBA eigenvalues - ED eigenvalues| over sectors with the untruncated basis (Method section:
    without truncation the method is exact)."""
    worst = 0.0
    for m in (range(N) if sectors is None else sectors):
        ns, r, X = tgba.sector(N, h, m, N)
        e1 = np.linalg.eigvalsh(tgba.heff(ns, r, X, N, h_x))
        e2 = ed.sector_spectrum(N, h, h_x, m)
        if len(e1) != len(e2):
            return np.inf
        worst = max(worst, float(np.abs(e1 - e2).max()))
    return worst


def dsf_error(N, h, h_x, eta=0.05):
    ns, r, X = tgba.sector(N, h, 0, N)
    E, U = tgba.eigh(tgba.heff(ns, r, X, N, h_x))
    dE, w = tgba.dsf_weights(E, U, tgba.x_full(X), N)
    dE2, w2 = ed.dsf_weights(N, h, h_x)
    om = tgba.omega_grid(0.0, 8.0, 400)
    S1 = 2 * math.pi * (tgba.lorentzian(om[:, None] - dE[None, :], eta) @ w)
    S2 = 2 * math.pi * (tgba.lorentzian(om[:, None] - dE2[None, :], eta) @ w2)
    return float(np.abs(S1 - S2).max() / np.abs(S2).max())


def quench_error(N, h0, h, h_x, t_max=12.0, n_t=25):
    t, mx, c0 = tgba.quench(N, h, h0, h_x, N, None, t_max, n_t)
    return float(np.abs(mx - ed.quench_magnetisation(N, h0, h, h_x, t)).max())


def calabrese_overlaps(N, h, h0, parity, states):
    """Eq. S6: |0(h0)> = prod_{0<k<pi} cos(D_k/2) [1 + i tan(D_k/2) d^dag_{-k} d^dag_k] |0(h)>,
    D_k = theta_k(h) - theta_k(h0).  A state overlaps only if its momenta form (-k, k) pairs
    (none at 0 or pi); the coefficient is prod cos(D/2) times i tan(D_k/2) per pair."""
    n = md.momenta_n(N, parity)
    th, th0 = md.theta(N, parity, h), md.theta(N, parity, h0)
    pos = [i for i in range(N) if 0 < n[i] < N]
    base = float(np.prod([math.cos((th[i] - th0[i]) / 2) for i in pos]))
    index = {int(n[i]): i for i in range(N)}
    out = []
    for s in states:
        labs = sorted(int(n[i]) for i in s.modes)
        if any(-l not in labs for l in labs) or 0 in labs or N in labs:
            out.append(0.0)
            continue
        v = complex(base)
        for l in labs:
            if l > 0:
                i = index[l]
                v *= 1j * math.tan((th[i] - th0[i]) / 2)
        out.append(v)
    return np.array(out, dtype=complex)
