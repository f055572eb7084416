"""Writes quench_L80.txt: the oracle's quench at L = 80 (the size of the quench benchmark
workload: M <= 10, h_z = 1, initial state the h_x = 0 ground states at h_z0 = 0.5, 2000 times
in [0, 100]) on the nested energy cutoffs 3.0, 3.5 and 3.74 above the NS vacuum (338, 760 and
1018 states of the k = 0 sector; no level lies within 1e-4 of a cutoff) for h_x = 0.05 and 0.1.

Calls only the oracle: X by direct Pfaffians of the whole operator string (Appendix A,
Eq. S1-S2), H_eff (Eq. 2, S4), dense eigenpairs, the Eq. S6 overlaps by direct Pfaffians and
B(t) = U e^{-iEt} U^H c0 (Eq. 10), <sigma^x>(t) = B^H X B / ||c0||^2.  The direct Pfaffians
take several minutes on a few cores, which is why the values are stored.

    python tests/golden/make_quench_L80.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import basis as obs          # noqa: E402
from oracle import modes as md           # noqa: E402
from oracle import native                # noqa: E402
from oracle import tgba as otgba         # noqa: E402

L, H, H0, MAX_QP = 80, 1.0, 0.5, 10
CUTS = (3.0, 3.5, 3.74)
HXS = (0.05, 0.1)
T_MAX, N_T = 100.0, 2000
OUT = os.path.join(HERE, "quench_L80.txt")


def main():
    native.build()
    ns, r, X = otgba.sector(L, H, 0, MAX_QP, CUTS[-1])
    c0 = otgba.initial_overlaps(L, H, H0, ns, r)
    e_vac = md.vacuum_energy(L, md.NS, H)
    t = otgba.time_grid(T_MAX, N_T)
    lines = ["# oracle quench, L=%d h_z=%g h_z0=%g max_qp=%d t_max=%g n_t=%d (tests/golden/make_quench_L80.py)"
             % (L, H, H0, MAX_QP, T_MAX, N_T),
             "# per case: 'case e_cut h_x chi norm2' then the n_t values of <sigma^x>(t_i), t_i = i t_max/(n_t-1)"]
    for cut in CUTS:
        kn = [i for i, s in enumerate(ns) if s.E <= e_vac + cut + 1e-9]
        kr = [j for j, s in enumerate(r) if s.E <= e_vac + cut + 1e-9]
        ns_c, r_c = [ns[i] for i in kn], [r[j] for j in kr]
        Xc = X[np.ix_(kn, kr)]
        c = np.concatenate([c0[kn], c0[len(ns) + np.array(kr, dtype=np.int64)]])
        for hx in HXS:
            E, U = otgba.eigh(otgba.heff(ns_c, r_c, Xc, L, hx))
            B = otgba.quench_coefficients(E, U, c, t)
            mx = otgba.magnetisation(B, otgba.x_full(Xc), c)
            lines.append("case %.17g %.17g %d %.17g" % (cut, hx, len(c), float(np.vdot(c, c).real)))
            lines.extend("%.17g" % v for v in mx)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
