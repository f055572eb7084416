"""Writes dsf_L18.txt: the oracle's S(k=0, w) on the frequency grid of the L = 40 benchmark
workload (4096 points in [0, 10], Lorentzian eta = 0.01) for the largest k = 0 basis its direct
Pfaffians finish in minutes: L = 18, h_z = 1, h_x = 0.1, every state with M <= 6 (2429 states).

Calls only the oracle: X by direct Pfaffians of the whole operator string (Appendix A,
Eq. S1-S2), H_eff (Eq. 2, S4), dense eigenpairs, the weights w_a = L |<psi_0|sigma^x_1|psi_a>|^2
and S(w) = 2 pi sum_a w_a L_eta(w - (E_a - E_0)) (Eq. 8-9), summed in FP64.

    python tests/golden/make_dsf_L18.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import native                # noqa: E402
from oracle import tgba as otgba         # noqa: E402

L, H, HX, MAX_QP = 18, 1.0, 0.1, 6
W_MIN, W_MAX, N_W, ETA = 0.0, 10.0, 4096, 0.01
OUT = os.path.join(HERE, "dsf_L18.txt")


def main():
    native.build()
    ns, r, X = otgba.sector(L, H, 0, MAX_QP)
    E, U = otgba.eigh(otgba.heff(ns, r, X, L, HX))
    Xf = otgba.x_full(X)
    dE, w = otgba.dsf_weights(E, U, Xf, L)
    S = otgba.dsf(E, U, Xf, L, W_MIN, W_MAX, N_W, ETA)
    lines = ["# oracle S(k=0,w), L=%d h_z=%g h_x=%g max_qp=%d, %d states; w in [%g, %g], n_w=%d, eta=%g "
             "(tests/golden/make_dsf_L18.py)" % (L, H, HX, MAX_QP, len(E), W_MIN, W_MAX, N_W, ETA),
             "# 'states n', then n lines 'E_a - E_0  w_a' (ascending E_a), then 'S n_w' and the n_w values of S"]
    lines.append("states %d" % len(E))
    lines.extend("%.17g %.17g" % (a, b) for a, b in zip(dE, w))
    lines.append("S %d" % N_W)
    lines.extend("%.17g" % v for v in S)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
