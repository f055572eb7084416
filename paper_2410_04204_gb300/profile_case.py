"""Run one stage of the path on a small seeded case, for kernel profilers (ncu -k ... -c ...).

    python -m paper_2410_04204_gb300.profile_case eig --sectors 0 1 2 3
    python -m paper_2410_04204_gb300.profile_case pfaffian --sectors 0 1 2 3

eig: the native batched eigenvalue solver (one fill per matrix, one tridiagonalisation launch,
one bisection launch) on sectors of the L = 24, h_z = 1, M <= 6 basis with its cutoff;
pfaffian: the Pfaffian stage of the same basis.  The stage runs --reps times; the eigenvalues
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
    p.add_argument("stage", choices=["eig", "pfaffian"])
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


if __name__ == "__main__":
    sys.exit(main())
