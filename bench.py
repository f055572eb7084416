#!/usr/bin/env python
"""Benchmark of the TGBA hot path on GB300 (one JSON line on stdout).

Workload (default): every momentum sector of the L = 24 chain at h_z = 1, M <= 6
quasiparticles, energy cutoff 11.925 above the NS vacuum (~900 x 900 NS x R states per
sector), longitudinal fields h_x = 0.05 and 0.1.  One step = the whole hot path on it:
contraction table, Pfaffians of all NS x R pairs of all sectors (one X serves both h_x), then
for each h_x the dense complex H_eff of every sector and all its eigenvalues.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

value = H_eff (Pfaffian) elements of the step, summed over ranks, per second of the step
time (CUDA events on the launching stream, max over ranks); pfaffian_elements_per_s = the same
elements per second of the Pfaffian stage alone.  Under torchrun every rank runs its own copy of
the workload (weak scaling, no data-path collective).  --impl reference times the CPU oracle
(the reduced form: one Schur complement of the vacuum operators per sector, then a Pfaffian of
size M+M' per element; the direct Pfaffians of size 2N+M+M' as a context row; numpy
eigensolver) on the host cores on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_eff elements/sec (FP64 Pfaffian) and % FP64 peak; screened vs plain speedup @1e-6"
UNIT = "H_eff elements/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="L24_all_sectors", choices=["L24_all_sectors", "L80_k0_quench"],
                   help="L24_all_sectors: every sector of L = 24, H_eff and all eigenvalues for two h_x; "
                        "L80_k0_quench: the L = 80 quench, 64 (h_x, cutoff) variants, 2000 times")
    p.add_argument("--e2e-steps", type=int, default=2, help="end-to-end steps (0: skip, for profiler runs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-budget-s", type=float, default=12.0)
    p.add_argument("--no-screening", action="store_true")
    p.add_argument("--no-solver-comparison", action="store_true",
                   help="skip the one-off native vs cuSOLVER eigen-solver timing after the timed steps")
    g = p.add_argument_group("single stage on a small seeded case (for kernel profilers: ncu -k ... -c ...)")
    g.add_argument("--stage", choices=["eig", "pfaffian", "direct", "dgemm", "screen"],
                   help="run one stage --reps times and print its CUDA-event timings instead of the benchmark")
    g.add_argument("--sectors", type=int, nargs="+", default=[0, 1, 2, 3])
    g.add_argument("--pairs", type=int, default=20000)
    g.add_argument("--L", type=int, default=None)
    g.add_argument("--hx", type=float, nargs="+", default=None)
    g.add_argument("--reps", type=int, default=1)
    g.add_argument("--mnk", type=int, nargs=3, default=[8192, 128, 20000],
                   help="dgemm stage: C (M x N) = A (M x K) B^T (N x K) on the tensor cores")
    return p.parse_args()


def measured_peaks():
    """The measured peaks the driver writes (MEASURED_PEAKS.json), or {} when absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def workload_config(w, n_elements=None, n_states=None):
    cfg = {"workload": w.name, "L": w.L, "h_z": w.h_z, "h_x": list(w.h_x), "sectors": len(w.sectors),
           "max_qp": w.max_qp, "e_cut": w.e_cut}
    if n_elements is not None:
        cfg["elements"] = n_elements
        cfg["states"] = n_states
    return cfg


# ------------------------------------------------------------------ clocks during the timed region
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ the oracle on the host cores
def oracle_sample(w, budget_s, tag=0):
    """Time the oracle on a bounded, seeded sample of the workload and extrapolate to one step.

    Sample: pairs drawn uniformly from the oracle's own basis of a few sectors, evaluated by
    both of the oracle's routes: the direct Pfaffian of size 2N+M+M' per element (Appendix A as
    written) and the reduced form (one Schur complement of the vacuum operators, then a Pfaffian
    of size M+M' per element), each on all host cores and on one thread; and one complex128
    numpy eigvalsh of a sector-sized Hermitian matrix.  Step estimate = elements x (time per
    pair) + 2 h_x x sum over sectors of the eigensolve time scaled by (n / n_ref)^3."""
    import numpy as np

    from oracle import basis as obs
    from oracle import elements as oel
    from paper_2410_04204_gb300 import inputs

    g = inputs.rng(100 + tag)
    sectors = sorted(g.choice(w.sectors, size=min(3, len(w.sectors)), replace=False).tolist())
    bases = {m: obs.sector_basis(w.L, w.h_z, m, w.max_qp, w.e_cut, w.max_per_parity) for m in sectors}
    sizes = {m: (len(ns), len(r)) for m, (ns, r) in bases.items()}

    def time_pairs(fn, budget, threads, per_sector, cap):
        t, n, used, rnd = 0.0, 0, 1, 0
        while t < budget and n < cap:
            batch = []
            for m in sectors:
                ns, r = bases[m]
                if ns and r:
                    for a, bb in inputs.sample_pairs(len(ns), len(r), per_sector, tag=1000 * tag + 97 * rnd + m):
                        batch.append((ns[a].modes, r[bb].modes))
            t0 = time.perf_counter()
            _, used = fn(w.L, w.h_z, batch, n_threads=threads, return_threads=True)
            t += time.perf_counter() - t0
            n += len(batch)
            rnd += 1
        return t / max(n, 1), n, used

    rows = {}
    for name, fn, share, per_sector, cap in (("direct", oel.x_elements, 0.35, 256, 65536),
                                             ("reduced", oel.x_elements_reduced, 0.25, 20000, 4_000_000)):
        t_all, n_all, threads = time_pairs(fn, share * budget_s, 0, per_sector, cap)
        t_one, n_one, _ = time_pairs(fn, 0.1 * budget_s, 1, max(64, per_sector // 8), cap)
        rows[name] = dict(t_pair=t_all, n_pairs=n_all, threads=threads, t_pair_1thread=t_one, n_pairs_1thread=n_one)
    n_ref = max(a + b for a, b in sizes.values())
    h = g.standard_normal((n_ref, n_ref)) + 1j * g.standard_normal((n_ref, n_ref))
    h = h + h.conj().T
    t0 = time.perf_counter()
    np.linalg.eigvalsh(h)
    t_eig = time.perf_counter() - t0
    return dict(rows=rows, t_eig=t_eig, n_ref=n_ref, threads=rows["reduced"]["threads"], sectors=sectors)


def oracle_step_seconds(w, s, sector_sizes, form="reduced", one_thread=False):
    n_el = sum(a * b for a, b in sector_sizes)
    row = s["rows"][form]
    t = n_el * (row["t_pair_1thread"] if one_thread else row["t_pair"])
    for a, b in sector_sizes:
        t += len(w.h_x) * s["t_eig"] * ((a + b) / s["n_ref"]) ** 3
    return t, n_el


def oracle_sector_sizes(w):
    from oracle import basis as obs
    out = []
    for m in w.sectors:
        ns, r = obs.sector_basis(w.L, w.h_z, m, w.max_qp, w.e_cut, w.max_per_parity)
        out.append((len(ns), len(r)))
    return out


def sample_text(s):
    r = s["rows"]
    return ("seeded pairs from sectors %s: %d by the reduced form (Schur complement, Pfaffian of size M+M' per "
            "element; value), %d by direct Pfaffians of size 2N+M+M'; %d threads; one complex128 eigvalsh of "
            "n=%d (numpy threads); extrapolated to the full step"
            % (s["sectors"], r["reduced"]["n_pairs"], r["direct"]["n_pairs"], s["threads"], s["n_ref"]))


def cpu_rows(w, s, sizes):
    """Elements/s of the step for each oracle route, all host cores and one thread (the
    eigensolves always with numpy's threads)."""
    out = {}
    for form in ("reduced", "direct"):
        for one, tag in ((False, "all_cores"), (True, "1_thread")):
            t, n_el = oracle_step_seconds(w, s, sizes, form, one)
            out["%s_%s" % (form, tag)] = n_el / t
    out["pfaffian_pairs_per_s"] = {f: 1.0 / s["rows"][f]["t_pair"] for f in ("reduced", "direct")}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from paper_2410_04204_gb300 import inputs
    w = inputs.SECTORS_L24
    sizes = oracle_sector_sizes(w)
    budget = max(2.0, args.cpu_budget_s / 2)
    for k in range(args.warmup):
        oracle_sample(w, 0.2 * budget, tag=k)
    vals, secs = [], []
    for k in range(args.steps):
        s = oracle_sample(w, budget, tag=100 + k)
        t, n_el = oracle_step_seconds(w, s, sizes)
        vals.append(n_el / t)
        secs.append(t)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, sum(a * b for a, b in sizes), sum(a + b for a, b in sizes)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": s["threads"], "kind": "oracle", "sample": sample_text(s),
                             "rows": cpu_rows(w, s, sizes)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate(ms_local, n_elements, world, dist=None, device=None):
    """Whole-job throughput under weak scaling: every rank processes its own copy of the
    workload, the step time is the slowest rank's, value = world * elements / time."""
    ms = float(ms_local)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * n_elements / (ms * 1e-3)


def screening_leg(b24, tgba, inputs, torch, bf16_peak_tflops):
    """Learned screening: train on 2e6 exact pairs of the L = 24 sectors (this workload), then,
    at L = 60 (k = 0, M <= 6, 2.25e8 pairs) and L = 80 (k = 0, M <= 10, 3.8e8 pairs), time the
    Pfaffian stage with and without screening for each tau, time the inference alone
    (tgba_screen_predict), and bound what any screener could gain: the share of Pfaffian work
    (F(n)-weighted) on pairs with |V| = L h_x |X| < tau (a perfect screener's saving, from the
    exact X) against the inference's own floor (2 * 256 * 256 FLOP per pair at the BF16 tensor
    peak).  Also the relative error of the lowest 20 eigenvalues at L = 40 (k = 0, n ~ 1e4)."""
    s, st = tgba.tgba_screen_train([b24], 2_000_000, inputs.SEED, 10)
    out = {"trained_on": "2e6 pairs of L24_all_sectors", "train": {k: round(v, 4) for k, v in st.items()}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(f, reps=2):
        best = 1e30
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def F(n):
        return sum(2 * m * (m - 1) + m for m in range(n - 2, 0, -2))

    for name, w in (("L60_k0", inputs.SCREEN_L60), ("L80_k0", inputs.QUENCH_L80)):
        b = tgba.tgba_build_basis(w.L, w.h_z, [0], w.max_qp, w.e_cut, w.max_per_parity)
        hx = w.h_x[0]
        t_exact = timed(lambda: tgba.tgba_compute_x(b))
        pf_exact = tgba.tgba_profile(b)["pfaffian_ms"]
        info = tgba.tgba_basis_info(b, 0, w.max_qp)
        nns, nr = info["n_ns"], info["n_r"]
        x = torch.empty(nns * nr, dtype=torch.complex128, device="cuda")
        tgba.tgba_x_export(b, 0, x)
        absv = (x.abs() * (w.L * hx)).view(nns, nr)
        del x
        M = torch.tensor(info["nqp"].astype("int64"), device="cuda")
        fl = torch.tensor([float(F(k)) for k in range(0, 41)], dtype=torch.float64, device="cuda")
        flw = fl[M[:nns, None] + M[None, nns:]]
        tot = flw.sum().item()
        perfect = {str(tau): (flw * (absv < tau)).sum().item() / tot for tau in inputs.SCREEN_TAUS}
        del flw
        pred = torch.empty(nns * nr, dtype=torch.float32, device="cuda")
        t_inf = timed(lambda: tgba.tgba_screen_predict(s, b, 0, pred))
        del pred
        rows = []
        xs = torch.empty(nns * nr, dtype=torch.complex128, device="cuda")
        for tau in inputs.SCREEN_TAUS:
            t_scr = timed(lambda: tgba.tgba_compute_x(b, s, tau, hx))
            ev, sc = tgba.tgba_x_stats(b)
            tgba.tgba_x_export(b, 0, xs)
            # pairs the network dropped although |V| >= tau (wrong drops: the error it makes)
            wrong = ((xs.view(nns, nr) == 0) & (absv >= tau)).sum().item()
            rows.append({"tau": tau, "screened_fraction": sc / (ev + sc), "wrongly_dropped_fraction": wrong / (ev + sc),
                         "ms": round(t_scr, 2), "speedup": t_exact / t_scr})
        del xs, absv
        floor_ms = nns * nr * 2.0 * 256 * 256 / (bf16_peak_tflops * 1e12) * 1e3
        best_saving = max(perfect.values()) * pf_exact
        out[name] = {"pairs": nns * nr, "exact_ms": round(t_exact, 2), "pfaffian_ms": round(pf_exact, 2),
                     "inference_ms": round(t_inf, 2), "inference_floor_ms": round(floor_ms, 2),
                     "perfect_screener_work_fraction": perfect,
                     "perfect_screener_max_saving_ms": round(best_saving, 2),
                     "screening_can_pay": floor_ms < best_saving, "taus": rows}
        tgba.tgba_basis_free(b)
    w3 = inputs.DSF_L40
    hx = w3.h_x[0]
    b = tgba.tgba_build_basis(w3.L, w3.h_z, [0], w3.max_qp, w3.e_cut)
    info = tgba.tgba_basis_info(b, 0, w3.max_qp)
    n = info["n_ns"] + info["n_r"]
    ev = torch.empty(n, dtype=torch.float64, device="cuda")
    tgba.tgba_compute_x(b)
    tgba.tgba_eigvals(b, hx, ev)
    exact = ev[:20].clone()
    tau = inputs.SCREEN_TAUS[-1]
    tgba.tgba_compute_x(b, s, tau, hx)
    tgba.tgba_eigvals(b, hx, ev)
    err = ((ev[:20] - exact).abs() / exact.abs()).max().item()
    _, sc = tgba.tgba_x_stats(b)
    out["L40_k0_eigen_check"] = {"tau": tau, "screened_fraction": sc / (info["n_ns"] * info["n_r"]),
                                 "max_rel_err_lowest20": err}
    tgba.tgba_basis_free(b)
    tgba.tgba_screen_free(s)
    return out


# DRAM bytes of one sytrd_groups launch on the L = 24 all-sector workload, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum); None until measured for the current kernel.
SYTRD_TRAFFIC = 487853093632 + 493968308224
# DRAM bytes (read + write) of the Pfaffian stage's one launch on this workload, from one ncu
# capture (profiles/pf_reg_queue_L24_all_sectors.md)
PF_TRAFFIC = 966912 + 116337664


def eigen_solver_leg(b, w, evs, tgba, torch):
    """Outside the timed steps: the native eigen-solver against cuSOLVER's batched one on the
    same matrices (time of one call each, and the largest eigenvalue difference)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out, res = {}, {}
    for name, method in (("cusolver_batched_ms", 2), ("native_ms", 1)):
        torch.cuda.synchronize()
        e0.record()
        tgba.tgba_eigvals(b, list(w.h_x), evs, method=method)
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1), 2)
        res[method] = evs.clone()
    out["max_abs_diff"] = (res[1] - res[2]).abs().max().item()
    return out


# ------------------------------------------------------------------ the GPU path
def run_gb300(args):
    import torch

    from paper_2410_04204_gb300 import build as libbuild
    from paper_2410_04204_gb300 import inputs, tgba

    rank, local_rank, world = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if not os.path.exists(libbuild.LIB):
        libbuild.build()
    w = inputs.SECTORS_L24
    stream = torch.cuda.current_stream()
    peak_gflops = tgba.tgba_fp64_peak(5)
    b = tgba.tgba_build_basis(w.L, w.h_z, w.sectors, w.max_qp, w.e_cut)
    n_sec, n_el, n_heff = tgba.tgba_basis_totals(b)
    sizes = [(tgba.tgba_basis_info(b, s, w.max_qp)["n_ns"], tgba.tgba_basis_info(b, s, w.max_qp)["n_r"]) for s in range(n_sec)]
    n_states = sum(a + c for a, c in sizes)
    H = torch.empty(n_heff, dtype=torch.complex128, device="cuda")
    evs = torch.empty(len(w.h_x) * n_states, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    def step():
        tgba.tgba_compute_x(b)
        for hx in w.h_x:
            tgba.tgba_assemble_heff(b, hx, H)
        tgba.tgba_eigvals(b, list(w.h_x), evs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    step_ms, pf_ms, tab_ms, tri_ms, bis_ms = [], [], [], [], []
    launches0 = tgba.tgba_profile(b)["kernel_launches"]
    clocks = Clocks(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()                      # evict the L2 between steps (outside the step events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        prof = tgba.tgba_profile(b)
        pf_ms.append(prof["pfaffian_ms"])
        tab_ms.append(prof["table_ms"])
        tri_ms.append(prof["tridiag_ms"])
        bis_ms.append(prof["bisect_ms"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = tgba.tgba_profile(b)["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(c) for a, c in ev]
    ms, value = aggregate(statistics.mean(step_ms), n_el, world, dist, "cuda")
    prof = tgba.tgba_profile(b)
    pf_mean, tab_mean = statistics.mean(pf_ms), statistics.mean(tab_ms)
    tri_mean, bis_mean = statistics.mean(tri_ms), statistics.mean(bis_ms)
    pf_gflops = prof["pfaffian_flops"] / (pf_mean * 1e-3) / 1e9
    peak_src = "live FP64 DFMA-chain kernel (tgba_fp64_peak); MEASURED_PEAKS.json has no FP64 entry"
    pf_roof = {"bound": "alu", "kernel": "pf_reg_queue / pf_tiles (FP64 Parlett-Reid Pfaffians)",
               "achieved": pf_gflops, "peak": peak_gflops, "unit": "GFLOP/s", "frac": pf_gflops / peak_gflops,
               "traffic": PF_TRAFFIC if prof["pfaffian_launches"] == 1 else None,
               "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of the stage's one launch on this "
                                 "workload (one ncu capture)",
               "peak_source": peak_src, "flops_per_launch": prof["pfaffian_flops"],
               "ms": pf_mean, "launches_per_stage": prof["pfaffian_launches"],
               "autotune": {"mode": prof["tune_mode"], "threads": prof["tune_threads"],
                            "candidates_ms": [round(x, 3) for x in prof["tune_ms"]]}}
    if tri_mean > pf_mean:
        # the dominant kernel of the step: the cluster tridiagonalisation of the native solver
        tri_gflops = prof["tridiag_flops"] / (tri_mean * 1e-3) / 1e9
        roofline = {"bound": "alu", "kernel": "sytrd_groups (FP64 Householder tridiagonalisation)",
                    "achieved": tri_gflops, "peak": peak_gflops, "unit": "GFLOP/s",
                    "frac": tri_gflops / peak_gflops, "traffic": SYTRD_TRAFFIC, "peak_source": peak_src,
                    "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of this kernel on this workload "
                                      "(one ncu capture of the warm-up launch; 1.11x the algorithmic 8 n^3/3 B per "
                                      "matrix)",
                    "flops_per_launch": prof["tridiag_flops"], "ms": tri_mean,
                    "matrices": prof["eig_matrices"], "ctas_per_matrix": prof["eig_cluster"]}
    else:
        roofline = pf_roof

    # end to end through the public API with host buffers: host enumeration and upload of the
    # state tables, the step, and the eigenvalues read back to pinned host memory
    host_ev = torch.empty(len(w.h_x) * n_states, dtype=torch.float64, pin_memory=True)
    e2e_s, h2d = [], 0
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2 = tgba.tgba_build_basis(w.L, w.h_z, w.sectors, w.max_qp, w.e_cut)
        tgba.tgba_compute_x(b2)
        for hx in w.h_x:
            tgba.tgba_assemble_heff(b2, hx, H)
        tgba.tgba_eigvals(b2, list(w.h_x), evs)
        host_ev.copy_(evs, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s.append(time.perf_counter() - t0)
        h2d = tgba.tgba_profile(b2)["upload_bytes"]
        tgba.tgba_basis_free(b2)
    e2e_value = world * n_el / statistics.mean(e2e_s) if e2e_s else None

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w, n_el, n_states),
                           l2="256 MiB buffer written between steps, outside the step events"),
            "pfaffian_elements_per_s": n_el / (pf_mean * 1e-3) * world,
            "roofline": roofline,
            "stages_ms": {"table": tab_mean, "pfaffian": pf_mean, "tridiag": tri_mean, "bisect": bis_mean,
                          "heff_fill_and_other": ms - tab_mean - pf_mean - tri_mean - bis_mean},
            "pfaffian_stage": dict(pf_roof, elements_per_s=n_el / (pf_mean * 1e-3),
                                   elements_per_s_with_table=n_el / ((pf_mean + tab_mean) * 1e-3)),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": n_states * 8 * len(w.h_x)},
            "gpu_launches": launches}
    if not args.no_solver_comparison:
        line["eigen_solver"] = eigen_solver_leg(b, w, evs, tgba, torch)
    if not args.no_screening:
        line["screening"] = screening_leg(b, tgba, inputs, torch, measured_peaks().get("bf16_tflops", 1945.0))
    tgba.tgba_basis_free(b)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample(w, args.cpu_budget_s)
        sizes_o = oracle_sector_sizes(w)
        t_cpu, _ = oracle_step_seconds(w, s, sizes_o)
        line["cpu_baseline"] = {"value": n_el / t_cpu, "unit": UNIT, "cores": s["threads"], "kind": "oracle",
                                "sample": sample_text(s), "rows": cpu_rows(w, s, sizes_o)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ the L = 80 quench workload
def quench_variants(tgba, inputs, b, w):
    """The 64 (h_x, cutoff) variants: the nested cutoffs keep 5000 i of the basis' lowest
    states (i = 1..8), each with the 8 fields."""
    info = tgba.tgba_basis_info(b, 0, w.max_qp)
    E = info["E0"]
    e_vac = E[:info["n_ns"]].min()
    cuts = inputs.nested_cutoffs(E - e_vac, inputs.QUENCH_L80_KEEP)
    hxs = [hx for _ in cuts for hx in inputs.QUENCH_L80_HX]
    ecs = [c for c in cuts for _ in inputs.QUENCH_L80_HX]
    return hxs, ecs, cuts


def run_gb300_quench(args):
    """One step = the Pfaffian stage of the L = 80, M <= 10 basis (3.8e8 elements, one X for
    every variant) and the quench of all 64 variants (batched Chebyshev propagation, one graph),
    2000 times in [0, 100]."""
    import torch

    from paper_2410_04204_gb300 import build as libbuild
    from paper_2410_04204_gb300 import inputs, tgba

    rank, local_rank, world = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if not os.path.exists(libbuild.LIB):
        libbuild.build()
    w = inputs.QUENCH_L80
    q = w.quench
    stream = torch.cuda.current_stream()
    peak_gflops = tgba.tgba_fp64_peak(5)
    b = tgba.tgba_build_basis(w.L, w.h_z, w.sectors, w.max_qp, w.e_cut, w.max_per_parity)
    _, n_el, _ = tgba.tgba_basis_totals(b)
    hxs, ecs, cuts = quench_variants(tgba, inputs, b, w)
    nv, n_t = len(hxs), q["n_t"]
    mx = torch.empty(nv * n_t, dtype=torch.float64, device="cuda")
    nrm = torch.empty(nv, dtype=torch.float64, device="cuda")
    chi = None

    def step():
        nonlocal chi
        tgba.tgba_compute_x(b)
        chi = tgba.tgba_quench(b, 0, q["h_z0"], hxs, ecs, q["t_max"], n_t, mx, nrm, method=2)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = tgba.tgba_profile(b)["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    profs = []
    clocks = Clocks(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        profs.append(tgba.tgba_profile(b))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = tgba.tgba_profile(b)["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(c) for a, c in ev]
    ms, value = aggregate(statistics.mean(step_ms), n_el, world, dist, "cuda")
    pf_ms = statistics.mean(p["pfaffian_ms"] for p in profs)
    tab_ms = statistics.mean(p["table_ms"] for p in profs)
    q_ms = statistics.mean(p["quench_ms"] for p in profs)
    prof = profs[-1]
    q_gflops = prof["quench_flops"] / (q_ms * 1e-3) / 1e9
    # The propagation's products run on the tensor cores as 21 BF16 slice-pair products per FP64
    # product (digit diagonals p + q <= 5 of six slices), so its roofline is the BF16 tensor peak:
    # achieved = 21 x the useful FP64 flops of the off-diagonal products (8 K kn kr per variant)
    # / the propagation's time; peak = the measured sustained BF16 rate (a kernel inside a
    # seconds-long step).
    peaks = measured_peaks()
    tc_peak = peaks.get("bf16_tflops_sustained")
    tc_src = "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    if tc_peak is None:
        tc_peak, tc_src = 1700.0, "profiling recipe's sustained fallback (of fallback)"
    tc_tflops = 21.0 * prof["quench_flops"] / (q_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "kernel": "Chebyshev propagation: FP64 products with the X block on the tensor "
                                             "cores (dgemm_tc_kernel, BF16 slices) + cheb_step + vector slicing",
                "achieved": tc_tflops, "peak": tc_peak, "unit": "TFLOP/s", "frac": tc_tflops / tc_peak,
                "traffic": None, "peak_source": tc_src, "slice_products_per_fp64_product": 21,
                "fp64_equivalent_gflops": q_gflops, "fp64_pipe_peak_gflops": peak_gflops,
                "fp64_flops_per_step": prof["quench_flops"], "ms": q_ms, "terms_K": prof["quench_terms"]}
    host_mx = torch.empty(nv * n_t, dtype=torch.float64, pin_memory=True)
    e2e_s, h2d = [], 0
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2 = tgba.tgba_build_basis(w.L, w.h_z, w.sectors, w.max_qp, w.e_cut, w.max_per_parity)
        tgba.tgba_compute_x(b2)
        tgba.tgba_quench(b2, 0, q["h_z0"], hxs, ecs, q["t_max"], n_t, mx, nrm, method=2)
        host_mx.copy_(mx, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s.append(time.perf_counter() - t0)
        h2d = tgba.tgba_profile(b2)["upload_bytes"]
        tgba.tgba_basis_free(b2)
    tgba.tgba_basis_free(b)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "L": w.L, "h_z": w.h_z, "h_z0": q["h_z0"], "max_qp": w.max_qp,
                       "e_cut": w.e_cut, "max_per_parity": w.max_per_parity, "elements": n_el,
                       "variants": nv, "h_x": list(inputs.QUENCH_L80_HX), "cutoffs": cuts,
                       "chi": [int(c) for c in chi[::len(inputs.QUENCH_L80_HX)]], "t_max": q["t_max"], "n_t": n_t,
                       "l2": "inputs larger than L2 (3.2 GB X block per step)"},
            "roofline": roofline,
            "stages_ms": {"table": tab_ms, "pfaffian": pf_ms,
                          "quench_slicing_and_bounds": statistics.mean(p["quench_prep_ms"] for p in profs),
                          "quench_propagation": q_ms,
                          "quench_moments": statistics.mean(p["quench_gram_ms"] for p in profs),
                          "quench_time_sums": statistics.mean(p["quench_eval_ms"] for p in profs),
                          "quench_rest": ms - tab_ms - pf_ms - q_ms},
            "pfaffian_stage": {"ms": pf_ms, "elements_per_s": n_el / (pf_ms * 1e-3),
                               "gflops": prof["pfaffian_flops"] / (pf_ms * 1e-3) / 1e9,
                               "frac": prof["pfaffian_flops"] / (pf_ms * 1e-3) / 1e9 / peak_gflops},
            "clocks": clk,
            "e2e": {"value": world * n_el / statistics.mean(e2e_s) if e2e_s else None, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": nv * n_t * 8},
            "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ one stage, for profilers
def run_stage(args):
    """One stage of the path on sectors of the L = 24, h_z = 1, M <= 6 basis with its cutoff:
    eig = the native batched eigenvalue solver (one fill per matrix, one tridiagonalisation
    launch, one bisection launch); pfaffian = the Pfaffian stage; direct = the paper-literal X
    (tgba_x_direct) of --pairs seeded pairs of the first listed sector, with its algorithmic FP64
    flops per element (the operator-string matrix, 4 m (m - 1) L, plus the complex Parlett-Reid
    elimination, sum over j = m - 2, m - 4, ..., 2 of 8 j (j - 1) + 6 j, for the string length
    m = 2L + M_a + M_b).  Prints one line of CUDA-event timings (not benchmark numbers when run
    under a profiler)."""
    import numpy as np
    import torch

    from paper_2410_04204_gb300 import inputs, tgba

    w = inputs.SECTORS_L24
    L = args.L or w.L
    hx = args.hx or [w.h_x[0]]
    torch.cuda.set_device(0)
    if args.stage == "screen":
        # screener inference (tensor cores) on every pair of the L = 40, k = 0 basis, with a
        # seeded untrained network: prediction, then the screened Pfaffian stage
        w3 = inputs.DSF_L40
        b = tgba.tgba_build_basis(w3.L, w3.h_z, [0], w3.max_qp, w3.e_cut)
        s = tgba.tgba_screen_create(256, None, inputs.SEED)
        try:
            tgba.tgba_compute_x(b)
            info = tgba.tgba_basis_info(b, 0, w3.max_qp)
            pred = torch.empty(info["n_ns"] * info["n_r"], dtype=torch.float32, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            times = []
            for _ in range(max(1, args.reps)):
                torch.cuda.synchronize()
                e0.record()
                tgba.tgba_screen_predict(s, b, 0, pred)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            tgba.tgba_compute_x(b, s, 1e-8, w3.h_x[0])
            torch.cuda.synchronize()
            assert torch.isfinite(pred).all()
            print("stage=screen L=%d pairs=%d predict_ms=%s" % (w3.L, pred.numel(), [round(t, 3) for t in times]))
        finally:
            tgba.tgba_screen_free(s)
            tgba.tgba_basis_free(b)
        return 0
    if args.stage == "dgemm":
        # FP64 product on the tensor cores: 2 M N K FP64 flops, 21 BF16 slice products of each
        M, N, K = args.mnk
        g = torch.Generator(device="cuda").manual_seed(inputs.SEED)
        A = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn(N, K, dtype=torch.float64, device="cuda", generator=g)
        C = torch.empty(N, M, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(max(1, args.reps)):
            torch.cuda.synchronize()
            e0.record()
            tgba.tgba_dgemm_tc(M, N, K, A, K, B, K, C, M)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        err = ((C.T - A @ B.T).abs().max() / (A.abs() @ B.abs().T).max()).item()
        best = min(times)
        print("stage=dgemm M=%d N=%d K=%d ms=%s fp64_equiv_tflops=%.2f max_rel_err=%.2e"
              % (M, N, K, [round(t, 3) for t in times], 2.0 * M * N * K / best / 1e9, err))
        return 0
    b = tgba.tgba_build_basis(L, w.h_z, args.sectors, w.max_qp, w.e_cut)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        tgba.tgba_compute_x(b)
        n_states = sum(x + y for x, y in tgba.tgba_sector_sizes(b))
        if args.stage == "direct":
            info = tgba.tgba_basis_info(b, 0)
            n_ns, n_r = info["n_ns"], info["n_r"]
            pairs = inputs.sample_pairs(n_ns, n_r, args.pairs, tag=L)
            M = info["nqp"]
            m = 2 * L + M[pairs[:, 0]].astype(np.int64) + M[n_ns + pairs[:, 1]].astype(np.int64)
            # per element: the string matrix, two complex products per entry of its strict upper
            # triangle (the site sums come from per-launch tables), and the complex Parlett-Reid
            flops = float(sum(12 * mm * (mm - 1) // 2 + sum(8 * j * (j - 1) + 6 * j for j in range(int(mm) - 2, 0, -2))
                              for mm in m))
            p = torch.tensor(pairs, dtype=torch.int32, device="cuda")
            out = torch.empty(len(pairs), dtype=torch.complex128, device="cuda")
            times = []
            for _ in range(max(1, args.reps)):
                torch.cuda.synchronize()
                e0.record()
                tgba.tgba_x_direct(b, 0, p, out)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            assert torch.isfinite(torch.view_as_real(out)).all()
            best = min(times)
            print("stage=direct L=%d sector=%d pairs=%d mean_string=%.1f ms=%s elements_per_s=%.3e gflops=%.1f"
                  % (L, args.sectors[0], len(pairs), float(m.mean()), [round(t, 3) for t in times],
                     len(pairs) / best * 1e3, flops / best / 1e6))
            return 0
        ev = torch.empty(len(hx) * n_states, dtype=torch.float64, device="cuda")
        times = []
        for _ in range(max(1, args.reps)):
            torch.cuda.synchronize()
            e0.record()
            if args.stage == "eig":
                tgba.tgba_eigvals(b, hx, ev, method=1)
            else:
                tgba.tgba_compute_x(b)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = tgba.tgba_profile(b)
        if args.stage == "eig":
            assert torch.isfinite(ev).all()
        print("stage=%s L=%d sectors=%s states=%d ms=%s tridiag_ms=%.3f bisect_ms=%.3f pfaffian_ms=%.3f"
              % (args.stage, L, args.sectors, n_states, [round(t, 3) for t in times], prof["tridiag_ms"],
                 prof["bisect_ms"], prof["pfaffian_ms"]))
    finally:
        tgba.tgba_basis_free(b)
    return 0


def main():
    args = parse()
    if args.stage:
        return run_stage(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "L80_k0_quench":
        return run_gb300_quench(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
