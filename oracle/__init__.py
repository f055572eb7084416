"""TGBA oracle: a plain, slow, FP64 CPU implementation of what the GPU path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The product package never imports it and shares no code,
table or constant with it; the only thing both sides use is ``paper_2410_04204_gb300/inputs.py`` (seeded input
recipes that hold none of the method's arithmetic).

Modules
  modes     single-particle momenta, dispersion, Bogoliubov angles, vacua (Eq. 4-7, S3)
  basis     enumeration and truncation of the Gaussian basis per momentum sector
  elements  <phi_a|c_1 + c_1^dag|phi_b> and initial-state overlaps by direct Pfaffians
            of size 2N+M+M' (Eq. S1-S2, S4), through the C file ``tgba_oracle.c``
  tgba      H_eff (Eq. 2, S4), eigenpairs, S(k=0, w) (Eq. 9), quench <sigma^x>(t) (Eq. 10)
  ed        exact diagonalisation of the spin chain (Eq. 3) and Fock-space brute force,
            used only to pin the rest
  mlp       forward/backward/Adam of the pair-screening MLP, in float64 numpy
"""
