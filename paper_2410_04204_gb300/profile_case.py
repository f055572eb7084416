"""Run one stage of the path on a small seeded case, for kernel profilers (ncu -k ... -c ...).

    python -m paper_2410_04204_gb300.profile_case eig --sectors 0 1 2 3
    python -m paper_2410_04204_gb300.profile_case pfaffian --sectors 0 1 2 3
    python -m paper_2410_04204_gb300.profile_case direct --sectors 7 --pairs 20000

eig: the native batched eigenvalue solver (one fill per matrix, one tridiagonalisation launch,
one bisection launch) on sectors of the L = 24, h_z = 1, M <= 6 basis with its cutoff;
pfaffian: the Pfaffian stage of the same basis; direct: the paper-literal X (tgba_x_direct) of
--pairs seeded pairs of the first listed sector, with its algorithmic FP64 flops per element
(the operator-string matrix, 4 m (m - 1) L, plus the complex Parlett-Reid elimination,
sum over j = m - 2, m - 4, ..., 2 of 8 j (j - 1) + 6 j, for the string length m = 2L + M_a + M_b).  The stage runs --reps times; the eigenvalues
are checked to be finite.  Prints one line of CUDA-event timings (not benchmark numbers when
run under a profiler).
"""
import argparse
import sys


def main(argv=None):
    import torch

    from . import tgba
    from .inputs import SECTORS_L24

    p = argparse.ArgumentParser()
    p.add_argument("stage", choices=["eig", "pfaffian", "direct"])
    p.add_argument("--pairs", type=int, default=20000)
    p.add_argument("--L", type=int, default=SECTORS_L24.L)
    p.add_argument("--sectors", type=int, nargs="+", default=[0, 1, 2, 3])
    p.add_argument("--max-qp", type=int, default=SECTORS_L24.max_qp)
    p.add_argument("--e-cut", type=float, default=SECTORS_L24.e_cut)
    p.add_argument("--hx", type=float, nargs="+", default=[SECTORS_L24.h_x[0]])
    p.add_argument("--reps", type=int, default=1)
    a = p.parse_args(argv)
    torch.cuda.set_device(0)
    b = tgba.tgba_build_basis(a.L, SECTORS_L24.h_z, a.sectors, a.max_qp, a.e_cut)
    try:
        tgba.tgba_compute_x(b)
        n_states = sum(x + y for x, y in tgba.tgba_sector_sizes(b))
        if a.stage == "direct":
            return _direct(tgba, b, a, torch)
        ev = torch.empty(len(a.hx) * n_states, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(a.reps):
            torch.cuda.synchronize()
            e0.record()
            if a.stage == "eig":
                tgba.tgba_eigvals(b, a.hx, ev, method=1)
            else:
                tgba.tgba_compute_x(b)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = tgba.tgba_profile(b)
        if a.stage == "eig":
            assert torch.isfinite(ev).all()
        print("stage=%s L=%d sectors=%s states=%d ms=%s tridiag_ms=%.3f bisect_ms=%.3f pfaffian_ms=%.3f"
              % (a.stage, a.L, a.sectors, n_states, [round(t, 3) for t in times], prof["tridiag_ms"],
                 prof["bisect_ms"], prof["pfaffian_ms"]))
    finally:
        tgba.tgba_basis_free(b)
    return 0


def _direct(tgba, b, a, torch):
    import numpy as np

    from .inputs import sample_pairs
    info = tgba.tgba_basis_info(b, 0)
    n_ns, n_r = info["n_ns"], info["n_r"]
    pairs = sample_pairs(n_ns, n_r, a.pairs, tag=a.L)
    M = info["nqp"]
    m = 2 * a.L + M[pairs[:, 0]].astype(np.int64) + M[n_ns + pairs[:, 1]].astype(np.int64)

    def pf_flops(mm):
        return sum(8 * j * (j - 1) + 6 * j for j in range(int(mm) - 2, 0, -2))

    flops = float(sum(4 * mm * (mm - 1) * a.L + pf_flops(mm) for mm in m))
    p = torch.tensor(pairs, dtype=torch.int32, device="cuda")
    out = torch.empty(len(pairs), dtype=torch.complex128, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(max(1, a.reps)):
        torch.cuda.synchronize()
        e0.record()
        tgba.tgba_x_direct(b, 0, p, out)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    assert torch.isfinite(torch.view_as_real(out)).all()
    best = min(times)
    print("stage=direct L=%d sector=%d pairs=%d mean_string=%.1f ms=%s elements_per_s=%.3e gflops=%.1f"
          % (a.L, a.sectors[0], len(pairs), float(m.mean()), [round(t, 3) for t in times], len(pairs) / best * 1e3,
             flops / best / 1e6))
    return 0


if __name__ == "__main__":
    sys.exit(main())
