"""Benchmark of the HI-NQS subspace-diagonalisation hot path on B300.

One step = one pass of the whole hot path over the synthetic "precision"
workload (n_orb = 16, n_alpha = n_beta = 5, 2000 x 2000 HF-weighted strings,
4.0e6 determinants): Hamiltonian preparation, subspace build (filter, sort,
dedupe), alpha and beta string links, Davidson to 1e-6 Ha (mixed precision:
FP32 sigma bulk + FP64 refinement), 1-/2-RDMs with the Hellmann-Feynman
backward, and the spin-marginal teacher weights.

value = determinants through the whole path per second (N / step time), summed
over ranks.  Also reported: sigma determinants per second of one sigma product
in FP64 and FP32, and Davidson time-to-1e-6 Ha for the mixed and the FP64 solver
on the same GPU.

--impl reference runs the CPU oracle (FP64, plain C with OpenMP) on a bounded
sample of the same workload on the host cores.

nvidia-smi clock samples taken during the timed region go to
$HINQS_CLOCK_LOG_DIR/hinqs_clocks_rank<i>.csv (default: the temp directory); their
summary is the line's "clocks" entry.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sigma dets/s and Davidson time-to-1e-6 Ha: mixed vs FP64 on the same B300"
kNumSMs_B300 = 148
SM_MAX_MHZ = 2032
# DRAM bytes (read + write) per launch from one ncu capture of the current kernels on
# this workload: the two row-product launches of the same-spin half, and the
# tensor-core opposite-spin kernel
PROFILED_TRAFFIC = {"same": 63.29e6, "opposite": 33.10e6}
WORKLOAD = "precision"


def sig3(x):
    """x rounded to four significant digits (None stays None), for a compact line."""
    if x is None:
        return None
    return float(f"{x:.4g}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-ref", action="store_true",
                    help="large workload: also the FP64 Davidson to a 1e-8 residual as E_ref")
    ap.add_argument("--detail", action="store_true", help="per-component timings to stderr")
    ap.add_argument("--probe", default=None,
                    help="PART:PREC[:tune] -- run one sigma product (PART sigma|same|opposite, "
                         "PREC fp64|fp32|bf16ab|bf16x3ab|bf16c|fp64dfab) on the workload, untimed, and exit "
                         "(the target of kernel-level ncu captures); ':tune' autotunes first; "
                         "'pt2' -- one classical expansion and PT2 scoring on the converged "
                         "eigenvector")
    ap.add_argument("--tuning", default=None,
                    help="R,CH,ST -- pin the sigma tiles (rows per warp, CUDA-core chunk, "
                         "tensor-core stages) instead of autotuning: under a profiler the "
                         "autotuner's timings are distorted, so profiled runs pin the tiles "
                         "it keeps outside one")
    ap.add_argument("--profile", action="store_true",
                    help="run only the warm-up and timed steps (for a profiler's launch list)")
    return ap.parse_args()


def count_launches(fn, torch):
    """Kernels of this library (namespace hinqs) launched by one call of fn,
    counted from the CUDA activity records of torch.profiler, outside any timed
    region; None when the profiler cannot record CUDA activity."""
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events() if "hinqs::" in e.name]
        return len(names)
    except Exception:  # noqa: BLE001 - the count is a report, not a result
        return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw nvidia-smi samples: $HINQS_CLOCK_LOG_DIR if set, else the temp directory
        out_dir = os.environ.get("HINQS_CLOCK_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"hinqs_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- rooflines --

def rooflines(hq, sub, la, lb, n, nb, t_same, t_opp, t_sig, results):
    """Roofline of the step's dominant sigma kernel and of the other half.

    Algorithmic work per launch (the scope table's per-unit figures times the units):
      same-spin half (row products, BF16 operand, FP32 sums): read C + write sigma = 2 N 4 B, plus the
        link records read once (8 B per record of both spins and per alpha-self x
        beta-single record), the per-string tables (4 n^2 B per alpha string, 8 B of
        diagonal per string); bound: HBM, against the measured copy bandwidth.  A
        secondary figure gives the bytes the kernel moves between L1 and registers
        (2 B per link and column, 6 B per alpha-self x beta-single and column) against
        the L1 data path derived from unit counts and clocks.
      opposite-spin half (tensor cores, BF16): the MMA FLOPs executed on 128-row tiles
        over the padded folded K, and the useful share 2 sum (singles_a)(singles_b +
        n_b); bound: tensor, against the measured BF16 burst rate (the kernel is timed
        alone).
      FP64 sigma: 2 FLOPs per FMA of the algorithmic FMA count, against the FP64 FMA
        rate measured live by the library's probe kernel."""
    import json as _json
    N = sub.N
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        mp = _json.load(f)
    hbm = mp["hbm_gbs"]
    bf16_burst = mp["bf16_tflops"]
    fp64_peak = hq.probe_fma_rate(hq.PREC_FP64)
    fp32_peak = hq.probe_fma_rate(hq.PREC_FP32)
    alg_same = (2.0 * N * 4 + 8.0 * (la.n_links + lb.n_links + lb.n_singles)
                + 4.0 * n * n * sub.Na + 8.0 * (sub.Na + sub.Nb))
    # operand bytes per link and column: 2 (the BF16 copy of C); the alpha-self x
    # beta-single term also reads its FP32 table entry
    l1_same = 2.0 * (la.n_links * sub.Nb + lb.n_links * sub.Na) + 6.0 * lb.n_singles * sub.Na
    fma_same = N + sub.Na * (lb.n_links + lb.n_singles) + sub.Nb * la.n_links
    fma_opp_useful = la.n_singles * (lb.n_singles + sub.Nb * nb)
    mma_flops = tc_executed_flops(n, sub, la)
    l1_peak = kNumSMs_B300 * 128 * SM_MAX_MHZ * 1e6 / 1e9
    same_line = {
        "bound": "hbm", "kernel": "same-spin half, row products on the BF16 copy of C (FP32 sums)",
        "achieved": sig3(alg_same / t_same / 1e9), "peak": hbm, "unit": "GB/s",
        "frac": sig3(alg_same / t_same / 1e9 / hbm), "traffic": PROFILED_TRAFFIC.get("same"),
        "alg_bytes": alg_same, "ms": sig3(1e3 * t_same),
        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
        "l1_secondary": {"bytes": l1_same, "achieved_gbs": sig3(l1_same / t_same / 1e9),
                         "peak_gbs": l1_peak, "frac": sig3(l1_same / t_same / 1e9 / l1_peak),
                         "peak_source": "derived: 148 SMs x 128 B/cycle x 2032 MHz"}}
    opp_line = {
        "bound": "tensor", "kernel": "opposite-spin half, BF16 tcgen05",
        "achieved": sig3(mma_flops / t_opp / 1e12), "peak": bf16_burst, "unit": "TFLOP/s",
        "frac": sig3(mma_flops / t_opp / 1e12 / bf16_burst),
        "traffic": PROFILED_TRAFFIC.get("opposite"), "flops": mma_flops,
        "useful_flops": 2.0 * fma_opp_useful,
        "useful_frac": sig3(2.0 * fma_opp_useful / t_opp / 1e12 / bf16_burst),
        "ms": sig3(1e3 * t_opp), "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; "
                                              "of measured)"}
    n_inner = sum(r.n_sigma_fp32 for r in results) / len(results)
    same_dominant = n_inner * t_same >= n_inner * t_opp
    roof = dict(same_line if same_dominant else opp_line)
    roof["other_half"] = opp_line if same_dominant else same_line
    roof["fp64_sigma"] = {"bound": "alu", "achieved": sig3(2 * (fma_same + fma_opp_useful)
                                                           / t_sig["fp64"] / 1e12),
                          "peak": sig3(fp64_peak), "unit": "TFLOP/s",
                          "frac": sig3(2 * (fma_same + fma_opp_useful) / t_sig["fp64"] / 1e12
                                       / fp64_peak),
                          "peak_source": "FP64 FMA rate measured live (hinqs_probe_fma_rate)"}
    roof["fp32_fma_peak_tflops"] = sig3(fp32_peak)
    return roof


def tc_executed_flops(n, sub, la):
    """MMA FLOPs the tensor-core opposite-spin kernel executes per launch: for every
    alpha string, its singles in chunks of 64 (128 when a string has more than 64)
    against 128-row beta tiles over the folded K = n(n+1)/2 padded to 16."""
    K = n * (n + 1) // 2
    Kp = -(-K // 16) * 16
    NW = 64 if la.max_srow <= 64 else 128
    n_tiles = -(-sub.Nb // 128)
    return 2.0 * 128 * NW * Kp * n_tiles * sub.Na * (-(-la.max_srow // NW))



# ------------------------------------------------------------- reference --

def run_reference(args):
    """The CPU oracle, as it stands, on a bounded sample of the workload (host cores).

    One step = the same whole path as the GPU arm's step (subspace, ground state to a
    1e-6 residual, 1-/2-RDMs, spin marginals) on the sub-problem spanned by the first
    30 alpha and 30 beta strings of the workload (the HF-weighted sampler draws the
    important strings first): the oracle's subspace build, Lanczos with full
    reorthogonalisation on its matrix-free sigma, operator-expectation RDMs and plain
    marginal sums.  value = determinants of the sample per second of a step, the GPU
    arm's unit.  Also reported: the oracle's sigma rate on 4000 random rows of the
    full workload."""
    import numpy as np

    import oracle
    import synth
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = synth.workload(args.workload)
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    H = oracle.Ham(w["h"], w["eri"], w["e_nuc"], na, nb)
    k = 30
    a_s, b_s = w["alpha"][:k], w["beta"][:k]

    def step():
        sa, sb = oracle.build_subspace(a_s, b_s, na, nb)
        E, c, res = oracle.lanczos(H, sa, sb, tol=1e-6)
        g1, g2 = oracle.rdm(n, sa, sb, c)
        oracle.marginals(c, len(sa), len(sb))
        return len(sa) * len(sb), E

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        n_det, _ = step()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    dets_s = n_det / t
    # the oracle's sigma rows per second on the full workload, for reference
    sa, sb = oracle.build_subspace(w["alpha"], w["beta"], na, nb)
    N = len(sa) * len(sb)
    rows = np.sort(np.random.default_rng(0).choice(N, 4000, replace=False))
    t0 = time.perf_counter()
    oracle.sigma(H, sa, sb, synth.random_vector(N, 3), rows=rows)
    sigma_rate = len(rows) / (time.perf_counter() - t0)
    threads = oracle.max_threads()
    sample = (f"whole path (subspace, Lanczos to a 1e-6 residual, RDMs, marginals) on the "
              f"first {k} x {k} strings ({n_det} determinants) of the {N}-determinant workload")
    line = {
        "impl": "reference", "metric": METRIC, "value": dets_s, "unit": "dets/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} sub-problem, N={n_det} determinants (the first "
                               f"{k} x {k} strings of the N={N} workload): n_orb={n} "
                               f"n_alpha={na} n_beta={nb}",
                   "sample": sample,
                   "note": f"value is dets/s at N={n_det}, not at N={N}: per-determinant cost "
                           "grows with N, so compare it with the GPU arm's "
                           "same_sample_as_reference, not with its value"},
        "cpu_baseline": {"value": dets_s, "unit": "dets/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "sigma_rows_per_s": sigma_rate,
                         "sigma_sample": f"4000 random rows of one sigma of the {N}-determinant workload"},
        "e2e": {"value": dets_s, "unit": "dets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline_detail(oracle, synth, np, H_o, sa_o, sb_o, c_h):
    """More of the CPU oracle as it stands, on bounded samples (about ten seconds):
    one host core on the precision workload; the full 3136-determinant space (n_orb 8,
    3/3): a whole sigma product and the oracle's Lanczos solve with its
    time-to-1e-6 Ha against dense eigh; 500 rows of the 2.5e7-determinant
    differentiation workload."""
    out = {"cpu_model": cpu_model()}
    N = len(sa_o) * len(sb_o)
    rows = np.sort(np.random.default_rng(1).choice(N, 400, replace=False))
    t0 = time.perf_counter()
    oracle.sigma(H_o, sa_o, sb_o, c_h, rows=rows, n_threads=1)
    out["single_core"] = {"value": len(rows) / (time.perf_counter() - t0), "unit": "sigma dets/s",
                          "sample": f"{len(rows)} rows of the precision workload, 1 thread"}
    ws = synth.workload("fp64_small")
    Hs = oracle.Ham(ws["h"], ws["eri"], ws["e_nuc"], ws["n_alpha"], ws["n_beta"])
    sa, sb = oracle.build_subspace(ws["alpha"], ws["beta"], ws["n_alpha"], ws["n_beta"])
    Ns = len(sa) * len(sb)
    E_ref, _ = oracle.ground_state_dense(Hs, sa, sb)
    cs = synth.random_vector(Ns, 3)
    t0 = time.perf_counter()
    oracle.sigma(Hs, sa, sb, cs)
    t_sig = time.perf_counter() - t0
    trace = []
    t0 = time.perf_counter()
    E_l, _, res = oracle.lanczos(Hs, sa, sb, tol=1e-4, trace=trace)
    t_solve = time.perf_counter() - t0
    hit = next((t for th, t in trace if abs(th - E_ref) <= 1e-6), None)
    out["small"] = {"workload": f"fp64_small: full space, N={Ns}", "sigma_dets_per_s": Ns / t_sig,
                    "lanczos_iterations": len(trace), "solve_s": t_solve,
                    "time_to_1e-6_Ha_s": None if hit is None else hit - t0,
                    "energy_error_Ha": abs(E_l - E_ref), "residual": res,
                    "solver": "oracle Lanczos (full reorthogonalisation) to a 1e-4 residual, "
                              "E_ref from dense eigh"}
    wd = synth.workload("differentiation")
    Hd = oracle.Ham(wd["h"], wd["eri"], wd["e_nuc"], wd["n_alpha"], wd["n_beta"])
    da, db = oracle.build_subspace(wd["alpha"], wd["beta"], wd["n_alpha"], wd["n_beta"])
    Nd = len(da) * len(db)
    cd = synth.random_vector(Nd, 4)
    rows = np.sort(np.random.default_rng(2).choice(Nd, 500, replace=False))
    t0 = time.perf_counter()
    oracle.sigma(Hd, da, db, cd, rows=rows)
    out["differentiation"] = {"sigma_dets_per_s": len(rows) / (time.perf_counter() - t0),
                              "sample": f"500 rows of the {Nd}-determinant workload"}
    return out


# ------------------------------------------------------- bond scan (batch) --

def run_bond_scan(args):
    """24 geometries of the synthetic 16-orbital (5,5) bond scan with 500..4000
    strings per spin: one step = Hamiltonians, subspaces and links of every
    geometry + the batched mixed solve in lockstep (one batched launch per sigma
    stage per round, BF16 tensor-core inner sigma, FP64 refinement) to a 1e-6
    residual.  Compared, untimed by the step loop but on the same GPU: the worker-
    stream batch, the same solves one after another on one stream, and the plain
    FP64 Davidson one after another."""
    import numpy as np
    import torch

    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2606_26760_b300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    import paper_2606_26760_b300 as hq
    from paper_2606_26760_b300 import sharding
    import synth

    dev = torch.device("cuda", local)
    ws_all = synth.bond_scan_workload()
    n, ne = ws_all[0]["n_orb"], ws_all[0]["n_alpha"]
    # geometries are independent: each rank takes its longest-first share, no exchange
    costs = [sharding.geometry_cost(len(w["alpha"]), len(w["beta"])) for w in ws_all]
    mine = sharding.lpt_assign(costs, world)[rank]
    ws = [ws_all[g] for g in mine]
    N_all = int(sum(len(w["alpha"]) * len(w["beta"]) for w in ws_all))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(t):
        if world == 1:
            return t
        x = torch.tensor([t], device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        return float(x)
    host = [(torch.tensor(w["h"]).pin_memory(), torch.tensor(w["eri"]).pin_memory(),
             torch.from_numpy(w["alpha"].view(np.int64).copy()).pin_memory(),
             torch.from_numpy(w["beta"].view(np.int64).copy()).pin_memory()) for w in ws]
    resident = [tuple(x.to(dev) for x in hw) for hw in host]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mixed = dict(precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32_BF16C, inner_tol=3e-2,
                 tol_residual=1e-6, tol_energy=1e-8, max_subspace=16, max_iter=600)

    def prepare(inputs):
        probs = []
        for (h, eri, a, b), w in zip(inputs, ws):
            ham = hq.Hamiltonian(h, eri, ne, ne, w["e_nuc"])
            sub = hq.build_subspace(a, b, n, ne, ne)
            probs.append((ham, sub, hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)))
        return probs

    def step(inputs):
        probs = prepare(inputs)
        return probs, hq.davidson_batch(probs, autotune=True, n_streams=0, **mixed)

    for _ in range(args.warmup):
        step(resident)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        ev0.record(stream)
        probs, res = step(resident)
        ev1.record(stream)
        barrier()
        times.append(max_over_ranks(ev0.elapsed_time(ev1) / 1e3))
    e2e = []
    for _ in range(max(1, args.steps // 2)):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        _, r2 = step([tuple(x.to(dev, non_blocking=True) for x in hw) for hw in host])
        en = torch.tensor([x.energy for x in r2])  # energies come back with the call
        cs = [x.c.cpu() for x in r2]
        barrier()
        e2e.append(max_over_ranks(time.perf_counter() - t0))
    clk = clocks.stop()
    launches = count_launches(lambda: step(resident), torch)
    Ntot = N_all
    if world > 1:
        # the one collective: every rank's energies and statuses for the final check
        parts = [None] * world
        dist.all_gather_object(parts, {g: (r.energy, int(r.status)) for g, r in zip(mine, res)})
        statuses = sorted({st for part in parts for (_, st) in part.values()})
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": Ntot / (sum(times) / len(times)),
                              "unit": "dets/s", "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup,
                              "ms_per_step": 1e3 * sum(times) / len(times),
                              "higher_is_better": True, "scaling": "strong",
                              "vs_baseline": None, "dtype": "f32+bf16+f64", "data": "synthetic",
                              "config": {"workload": f"bond_scan: 24 geometries, {Ntot} "
                                                     "determinants in all",
                                         "parallelism": f"geometries sharded over {world} "
                                                        "ranks, longest first"},
                              "e2e": {"value": Ntot / (sum(e2e) / len(e2e)), "unit": "dets/s",
                                      "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
                              "gpu_launches": None if launches is None else launches * args.steps,
                              "energy": {"statuses": statuses}, "clocks": clk}), flush=True)
        dist.destroy_process_group()
        return
    h2d = sum(x.numel() * x.element_size() for hw in host for x in hw)
    d2h = sum(c.numel() * c.element_size() for c in cs) + en.numel() * 8

    # the solve alone: batched vs one-after-another, mixed vs FP64 (links already built)
    def solve_time(fn):
        flush.zero_()
        torch.cuda.synchronize()
        ev0.record(stream)
        out = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3, out

    t_batch, rb = solve_time(lambda: hq.davidson_batch(probs, n_streams=0, **mixed))
    t_workers, _ = solve_time(lambda: hq.davidson_batch(probs, n_streams=4, **mixed))
    t_seq_mixed, rs = solve_time(lambda: [hq.davidson(*p, **mixed) for p in probs])
    t_seq_fp64, rf = solve_time(lambda: [hq.davidson(*p, precision=hq.DAVIDSON_FP64,
                                                     tol_residual=1e-6, tol_energy=1e-8,
                                                     max_subspace=16, max_iter=600)
                                         for p in probs])
    err = max(abs(a.energy - b.energy) for a, b in zip(rb, rf))
    # the same scan with small subspaces (60..400 strings per spin), where every sigma
    # is launch-bound and the lockstep rounds batch all 24 geometries
    small = []
    for w in synth.bond_scan_workload(lo=60, hi=400):
        ham = hq.Hamiltonian(torch.tensor(w["h"], device=dev), torch.tensor(w["eri"], device=dev),
                             ne, ne, w["e_nuc"])
        sub = hq.build_subspace(torch.from_numpy(w["alpha"].view(np.int64).copy()).to(dev),
                                torch.from_numpy(w["beta"].view(np.int64).copy()).to(dev), n, ne, ne)
        small.append((ham, sub, hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)))
    hq.davidson_batch(small, autotune=True, n_streams=0, **mixed)
    ts_batch, rsb = solve_time(lambda: hq.davidson_batch(small, n_streams=0, **mixed))
    ts_workers, _ = solve_time(lambda: hq.davidson_batch(small, n_streams=4, **mixed))
    ts_seq, rss = solve_time(lambda: [hq.davidson(*p, **mixed) for p in small])
    t_mean = sum(times) / len(times)
    line = {
        "metric": METRIC,
        "value": Ntot / t_mean,
        "unit": "dets/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_mean,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f32+bf16+f64",
        "data": "synthetic",
        "config": {"workload": f"bond_scan: 24 geometries, n_orb={n} n_alpha=n_beta={ne}, "
                               f"500..4000 strings per spin, {Ntot} determinants in all",
                   "step": "24 x (ham+subspace+links) + batched mixed Davidson to 1e-6 residual",
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": "lockstep: one batched launch per sigma stage per round"},
        "e2e": {"value": Ntot / (sum(e2e) / len(e2e)), "unit": "dets/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": None if launches is None else launches * args.steps,
        "solve_s": {"batch_mixed_bf16": t_batch, "worker_streams_mixed_bf16": t_workers,
                    "sequential_mixed_bf16": t_seq_mixed, "sequential_fp64": t_seq_fp64,
                    "speedup_batch_vs_fp64": t_seq_fp64 / t_batch,
                    "speedup_batch_vs_sequential_mixed": t_seq_mixed / t_batch},
        "solve_s_small_scan": {"subspaces": "60..400 strings per spin, "
                                            f"{sum(p[1].N for p in small)} determinants in all",
                               "batch_mixed_bf16": ts_batch, "worker_streams_mixed_bf16": ts_workers,
                               "sequential_mixed_bf16": ts_seq,
                               "max_abs_diff_batch_vs_sequential_Ha":
                                   max(abs(a.energy - b.energy) for a, b in zip(rsb, rss))},
        "energy": {"max_abs_diff_batch_mixed_vs_fp64_Ha": err,
                   "statuses": sorted(set(int(x.status) for x in rb + rf))},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- large space --

def run_large(args):
    """n_orb = 26, (7,7), 20000 x 20000 strings (4e8 determinants): one step =
    Hamiltonian, subspace, links, mixed Davidson (BF16-operand inner sigma, double-float
    refinement, subspace of 16) to a 1e-5 residual, RDMs with the backward and the
    marginals.  The FP64 Davidson (about 340 FP64 products of ~2.8 s) runs only with
    --fp64-ref, as E_ref for both solvers' time-to-1e-6 Ha; one FP64 sigma is timed."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2606_26760_b300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    import paper_2606_26760_b300 as hq
    import synth

    w = synth.workload("large")
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    dev = torch.device("cuda", local)
    h_d = torch.tensor(w["h"], device=dev)
    eri_d = torch.tensor(w["eri"], device=dev)
    a_d = torch.from_numpy(w["alpha"].view(np.int64)).to(dev)
    b_d = torch.from_numpy(w["beta"].view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    opts = dict(precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32_BF16C, inner_tol=3e-2,
                tol_residual=1e-5, tol_energy=1e-7, max_subspace=16, max_iter=800)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    parts = {}

    def step():
        t = {}
        ev0.record(stream)
        ham = hq.Hamiltonian(h_d, eri_d, na, nb, w["e_nuc"])
        sub = hq.build_subspace(a_d, b_d, n, na, nb)
        la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
        hq.autotune(ham, sub, la, lb, hq.PREC_FP32_BF16C)
        ev1.record(stream)
        torch.cuda.synchronize()
        t["setup_s"] = ev0.elapsed_time(ev1) / 1e3
        ev0.record(stream)
        res = hq.davidson(ham, sub, la, lb, **opts)
        ev1.record(stream)
        torch.cuda.synchronize()
        t["solve_s"] = ev0.elapsed_time(ev1) / 1e3
        ev0.record(stream)
        g1, g2 = hq.rdm(sub, la, lb, res.c)
        gh, ge = hq.energy_backward(n, 1.0, g1, g2)
        pa, pb = hq.spin_marginals(sub, res.c)
        ev1.record(stream)
        torch.cuda.synchronize()
        t["rdm_backward_marginals_s"] = ev0.elapsed_time(ev1) / 1e3
        parts.update(t)
        return ham, sub, la, lb, res, g1, g2

    for _ in range(args.warmup):
        step()
    times = []
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ham, sub, la, lb, res, g1, g2 = step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    e_id = float((h_d * g1).sum() + 0.5 * (eri_d * g2).sum()) + w["e_nuc"]
    sig = {}
    for name, p in (("fp32_bf16c", hq.PREC_FP32_BF16C), ("fp32_bf16ab", hq.PREC_FP32_BF16AB),
                    ("fp32", hq.PREC_FP32),
                    ("fp64", hq.PREC_FP64)):
        x = torch.rand(sub.N, device=dev, dtype=torch.float64 if p == hq.PREC_FP64 else torch.float32)
        y = torch.empty_like(x)
        hq.sigma(ham, sub, la, lb, x, out=y, precision=p)
        torch.cuda.synchronize()
        ev0.record(stream)
        hq.sigma(ham, sub, la, lb, x, out=y, precision=p)
        ev1.record(stream)
        torch.cuda.synchronize()
        sig[name] = ev0.elapsed_time(ev1)
        del x, y
    ref = None
    if args.fp64_ref:
        # E_ref: the FP64 Davidson at a 1e-8 residual, and the time-to-1e-6 Ha of both
        # solvers against it (trace clocks)
        del g1, g2
        torch.cuda.empty_cache()
        rf = hq.davidson(ham, sub, la, lb, precision=hq.DAVIDSON_FP64, tol_residual=1e-8,
                         tol_energy=1e-11, max_subspace=8, max_iter=1000, trace_cap=2048)
        rm = hq.davidson(ham, sub, la, lb, trace_cap=2048,
                         **dict(opts, tol_residual=1e-6, tol_energy=1e-8))

        def tt(r):
            return next((t for th, t, k in zip(r.trace["theta"], r.trace["time"], r.trace["kind"])
                         if k == 0 and abs(th - rf.energy) <= 1e-6), None)
        ref = {"E_ref_fp64": rf.energy, "E_ref_residual": rf.residual, "E_ref_status": int(rf.status),
               "fp64_solve_s": sig3(rf.seconds), "fp64_sigmas": rf.n_sigma_fp64,
               "fp64_time_to_1e-6_Ha_s": sig3(tt(rf)), "mixed_time_to_1e-6_Ha_s": sig3(tt(rm)),
               "mixed_abs_err_Ha": abs(rm.energy - rf.energy), "mixed_residual": rm.residual}
    t_mean = sum(times) / len(times)
    print(json.dumps({
        "fp64_reference": ref,
        "metric": METRIC, "value": sub.N / t_mean, "unit": "dets/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_mean,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+bf16+f64", "data": "synthetic",
        "config": {"workload": f"large: n_orb={n} n_alpha={na} n_beta={nb} {sub.Na}x{sub.Nb} "
                               f"strings, N={sub.N} determinants",
                   "step": "ham+subspace+links+mixed Davidson (m_max 16) to 1e-5 residual+RDM "
                           "backward+marginals"},
        "parts_s": parts, "sigma_ms": sig,
        "energy": {"mixed": res.energy, "residual": res.residual, "status": int(res.status),
                   "sigmas_fp64_fp32": [res.n_sigma_fp64, res.n_sigma_fp32],
                   "rdm_energy_identity_Ha": e_id - res.energy},
        "clocks": clk}), flush=True)


# ------------------------------------------------------------- time to 1e-6 --

def run_time_to(args):
    """Time-to-1e-6 Ha of the FP64 and mixed Davidson on the same B300 for the
    plain-FP64 (n=8, 3/3, full 56 x 56), precision (n=16, 5/5, 2000 x 2000) and
    differentiation (n=20, 7/7, 5000 x 5000) configurations: E_ref is the FP64 GPU
    solve at a 1e-9 residual; each solver's time is the first FP64-evaluated Ritz
    value within 1e-6 Ha of E_ref (trace clock), after one untimed solve."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2606_26760_b300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    import paper_2606_26760_b300 as hq
    import synth

    dev = torch.device("cuda", local)
    out = {}
    for wl in ("fp64_small", "precision", "differentiation"):
        w = synth.workload(wl)
        n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
        ham = hq.Hamiltonian(torch.tensor(w["h"], device=dev), torch.tensor(w["eri"], device=dev),
                             na, nb, w["e_nuc"])
        sub = hq.build_subspace(torch.from_numpy(w["alpha"].view(np.int64).copy()).to(dev),
                                torch.from_numpy(w["beta"].view(np.int64).copy()).to(dev), n, na, nb)
        la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
        hq.autotune(ham, sub, la, lb, hq.PREC_FP32_BF16C)
        ref = hq.davidson(ham, sub, la, lb, tol_residual=1e-9, tol_energy=1e-12, max_iter=2000)
        e_ref = ref.energy
        row = {"N": sub.N, "E_ref": e_ref, "E_ref_residual": ref.residual}
        for name, kw in (("fp64", dict(precision=hq.DAVIDSON_FP64)),
                         ("mixed_bf16c", dict(precision=hq.DAVIDSON_MIXED,
                                              inner_precision=hq.PREC_FP32_BF16C, inner_tol=3e-2)),
                         ("mixed_bf16ab", dict(precision=hq.DAVIDSON_MIXED,
                                               inner_precision=hq.PREC_FP32_BF16AB, inner_tol=3e-2)),
                         ("mixed_fp32", dict(precision=hq.DAVIDSON_MIXED,
                                             inner_precision=hq.PREC_FP32, inner_tol=3e-2))):
            for rep in range(2):
                r = hq.davidson(ham, sub, la, lb, tol_residual=1e-6, tol_energy=1e-8,
                                max_subspace=16, max_iter=2000, trace_cap=4096, **kw)
            tt = next((t for th, t, k in zip(r.trace["theta"], r.trace["time"], r.trace["kind"])
                       if k == 0 and abs(th - e_ref) <= 1e-6), None)
            row[name] = {"time_to_1e-6_Ha_s": sig3(tt), "solve_s": sig3(r.seconds),
                         "abs_err_Ha": abs(r.energy - e_ref),
                         "sigmas_fp64_fp32": [r.n_sigma_fp64, r.n_sigma_fp32]}
        a, b = row["fp64"]["time_to_1e-6_Ha_s"], row["mixed_bf16c"]["time_to_1e-6_Ha_s"]
        row["speedup_mixed_bf16c_vs_fp64"] = sig3(a / b) if a and b else None
        out[wl] = row
        del ham, sub, la, lb
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "Davidson time-to-1e-6 Ha: mixed vs FP64 on the same B300",
                      "unit": "s", "higher_is_better": False, "data": "synthetic",
                      "configs": out}), flush=True)


# ------------------------------------------------------------------ B300 --

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "bond_scan":
        return run_bond_scan(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "time_to":
        return run_time_to(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2606_26760_b300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    import paper_2606_26760_b300 as hq
    import synth

    w = synth.workload(args.workload)
    n, na, nb = w["n_orb"], w["n_alpha"], w["n_beta"]
    dev = torch.device("cuda", local)
    h_d = torch.tensor(w["h"], device=dev)
    eri_d = torch.tensor(w["eri"], device=dev)
    a_d = torch.from_numpy(w["alpha"].view(np.int64)).to(dev)
    b_d = torch.from_numpy(w["beta"].view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.probe == "pt2":
        # Step 1'/Step 2 on a converged eigenvector: the classical expansion of the
        # 1000 largest amplitudes and one PT2 scoring of every candidate (untimed)
        ham_p = hq.Hamiltonian(h_d, eri_d, na, nb, w["e_nuc"])
        sub_p = hq.build_subspace(a_d, b_d, n, na, nb)
        la_p, lb_p = hq.string_links(ham_p, sub_p, 0), hq.string_links(ham_p, sub_p, 1)
        res = hq.davidson(ham_p, sub_p, la_p, lb_p, precision=hq.DAVIDSON_MIXED,
                          inner_precision=hq.PREC_FP32_BF16AB, inner_tol=3e-2,
                          tol_residual=1e-6, tol_energy=1e-8, max_iter=600)
        xa, xb = hq.classical_expansion(ham_p, sub_p, res.c, 1000)
        hq.pt2_score(ham_p, sub_p, res.c, res.energy, xa, xb)
        torch.cuda.synchronize()
        print(json.dumps({"probe": "pt2", "N": sub_p.N, "candidates": int(xa.numel())}))
        return

    if args.probe:
        part, pname, *rest = args.probe.split(":")
        prec = {"fp64": hq.PREC_FP64, "fp32": hq.PREC_FP32, "bf16ab": hq.PREC_FP32_BF16AB,
                "bf16x3ab": hq.PREC_FP32_BF16X3AB, "bf16c": hq.PREC_FP32_BF16C,
                "fp64dfab": hq.PREC_FP64_DFAB}[pname]
        ham_p = hq.Hamiltonian(h_d, eri_d, na, nb, w["e_nuc"])
        sub_p = hq.build_subspace(a_d, b_d, n, na, nb)
        la_p, lb_p = hq.string_links(ham_p, sub_p, 0), hq.string_links(ham_p, sub_p, 1)
        tuning = None
        if args.tuning:
            hq.set_tuning(la_p, lb_p, *[int(v) for v in args.tuning.split(",")])
            tuning = la_p.tuning()
        elif "tune" in rest:  # the autotuner's tiles (its trial launches come first)
            hq.autotune(ham_p, sub_p, la_p, lb_p, prec)
            tuning = la_p.tuning()
        x = torch.tensor(synth.random_vector(sub_p.N, 3), device=dev)
        x = x if prec in (hq.PREC_FP64, hq.PREC_FP64_DFAB) else x.float()
        y = torch.zeros_like(x)
        if part == "sigma":
            hq.sigma(ham_p, sub_p, la_p, lb_p, x, out=y, precision=prec)
        else:
            hq.sigma_part(ham_p, sub_p, la_p, lb_p, x, y, part, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"probe": args.probe, "N": sub_p.N, "tuning": tuning}))
        return

    # inner_tol 3e-2: the BF16 inner operator is accurate to ~1e-2, so asking the
    # inner solve for more only adds FP32 iterations before the next FP64 refinement
    solve_opts = dict(precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32_BF16C,
                      inner_tol=3e-2,
                      tol_residual=1e-6, tol_energy=1e-8, max_subspace=16, max_iter=600,
                      trace_cap=1024)

    def step(h_in, eri_in, a_in, b_in):
        ham_s = hq.Hamiltonian(h_in, eri_in, na, nb, w["e_nuc"])
        sub_s = hq.build_subspace(a_in, b_in, n, na, nb)
        la_s, lb_s = hq.string_links(ham_s, sub_s, 0), hq.string_links(ham_s, sub_s, 1)
        if args.tuning:
            hq.set_tuning(la_s, lb_s, *[int(v) for v in args.tuning.split(",")])
        else:
            hq.autotune(ham_s, sub_s, la_s, lb_s, hq.PREC_FP32_BF16C)  # cached after the first step
        res = hq.davidson(ham_s, sub_s, la_s, lb_s, **solve_opts)
        g1, g2 = hq.rdm(sub_s, la_s, lb_s, res.c)
        gh, ge = hq.energy_backward(n, 1.0, g1, g2)
        pa, pb, wt = hq.spin_marginals(sub_s, res.c, want_w=True)
        return res, gh, ge, pa, pb

    if args.profile:
        for _ in range(args.warmup + args.steps):
            step(h_d, eri_d, a_d, b_d)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "steps": args.steps, "warmup": args.warmup}))
        return

    # reference energy for time-to-1e-6 Ha: FP64 Davidson to a tight residual
    ham = hq.Hamiltonian(h_d, eri_d, na, nb, w["e_nuc"])
    sub = hq.build_subspace(a_d, b_d, n, na, nb)
    la, lb = hq.string_links(ham, sub, 0), hq.string_links(ham, sub, 1)
    hq.autotune(ham, sub, la, lb, hq.PREC_FP32_BF16C)
    N = sub.N
    ref = hq.davidson(ham, sub, la, lb, precision=hq.DAVIDSON_FP64, tol_residual=1e-9,
                      max_iter=400, max_subspace=24)
    E_ref = ref.energy

    def time_to(trace, tol=1e-6):
        for th, t, k in zip(trace["theta"], trace["time"], trace["kind"]):
            if k == 0 and abs(th - E_ref) <= tol:
                return t
        return None

    for _ in range(args.warmup):
        step(h_d, eri_d, a_d, b_d)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times, results = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        ev0.record(stream)
        out = step(h_d, eri_d, a_d, b_d)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        results.append(out[0])
    barrier()
    launches_per_step = count_launches(lambda: step(h_d, eri_d, a_d, b_d), torch)

    # e2e: host buffers through the public API, copies inside the timed region
    h_h = torch.tensor(w["h"]).pin_memory()
    eri_h = torch.tensor(w["eri"]).pin_memory()
    a_h = torch.from_numpy(w["alpha"].view(np.int64).copy()).pin_memory()
    b_h = torch.from_numpy(w["beta"].view(np.int64).copy()).pin_memory()
    e2e_times = []
    d2h = 0
    for _ in range(max(1, args.steps // 2)):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        res, gh, ge, pa, pb = step(h_h.to(dev, non_blocking=True), eri_h.to(dev, non_blocking=True),
                                   a_h.to(dev, non_blocking=True), b_h.to(dev, non_blocking=True))
        outs = [x.cpu() for x in (gh, ge, pa, pb)]
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        d2h = sum(x.numel() * x.element_size() for x in outs) + 8
    clk = clocks.stop()
    h2d = sum(x.numel() * x.element_size() for x in (h_h, eri_h, a_h, b_h))

    # kernel-level sigma rates in every precision, and each half of the step's product
    c64 = torch.tensor(synth.random_vector(N, 3), device=dev)
    c32 = c64.float()

    def timed(fn, reps=20):  # 5 warm-up calls, then the median of `reps` timed calls
        for _ in range(5):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record(stream)
            fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            ts.append(ev0.elapsed_time(ev1) / 1e3)
        ts.sort()
        return ts[len(ts) // 2]

    precs = {"fp64": (hq.PREC_FP64, c64), "fp32": (hq.PREC_FP32, c32),
             "fp32_bf16ab": (hq.PREC_FP32_BF16AB, c32), "fp32_bf16x3ab": (hq.PREC_FP32_BF16X3AB, c32),
             "fp32_bf16c": (hq.PREC_FP32_BF16C, c32), "fp64_dfab": (hq.PREC_FP64_DFAB, c64)}
    t_sig = {}
    for name, (p, x) in precs.items():
        out = torch.empty_like(x)
        t_sig[name] = timed(lambda: hq.sigma(ham, sub, la, lb, x, out=out, precision=p),
                            reps=20)
    out32 = torch.empty_like(c32)
    t_same = timed(lambda: hq.sigma_part(ham, sub, la, lb, c32, out32, "same",
                                         precision=hq.PREC_FP32_BF16C))
    t_opp = timed(lambda: hq.sigma_part(ham, sub, la, lb, c32, out32, "opposite",
                                        precision=hq.PREC_FP32_BF16C))

    # FP64 and the mixed variants: time-to-1e-6 Ha on the same GPU
    variants = {"fp64": dict(precision=hq.DAVIDSON_FP64),
                "mixed_fp32": dict(precision=hq.DAVIDSON_MIXED, inner_precision=hq.PREC_FP32,
                                   inner_tol=3e-2),
                "mixed_bf16x3": dict(precision=hq.DAVIDSON_MIXED,
                                     inner_precision=hq.PREC_FP32_BF16X3AB, inner_tol=3e-2),
                "mixed_bf16ab": dict(precision=hq.DAVIDSON_MIXED,
                                     inner_precision=hq.PREC_FP32_BF16AB, inner_tol=3e-2)}
    runs = {}
    for name, kw in variants.items():
        runs[name] = hq.davidson(ham, sub, la, lb, tol_residual=1e-6, tol_energy=1e-8,
                                 max_subspace=16, max_iter=600, trace_cap=1024, **kw)
    fp64_runs = [runs["fp64"]]

    def best_time(rs):
        ts = [x for x in (time_to(r.trace) for r in rs) if x is not None]
        return min(ts) if ts else None

    tt_fp64 = best_time(fp64_runs)
    tt_mixed = best_time(results)
    tt_variants = {k: best_time([r]) for k, r in runs.items() if k != "fp64"}

    roof = rooflines(hq, sub, la, lb, n, nb, t_same, t_opp, t_sig, results)

    # Step 1'/Step 2 on the converged eigenvector: the 1000 largest amplitudes, their
    # classical singles/doubles expansion (Eq. classical_expansion) and the PT2 scores
    # of every candidate (Eq. pt2_score); public API calls, timed alone
    c_eig = results[-1].c
    e_eig = results[-1].energy

    def timed_once(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return min(ts), out

    t_top, _ = timed_once(lambda: hq.top_amplitudes(sub, c_eig, 1000))
    t_exp, (cxa, cxb) = timed_once(lambda: hq.classical_expansion(ham, sub, c_eig, 1000))
    t_pt2, _ = timed_once(lambda: hq.pt2_score(ham, sub, c_eig, e_eig, cxa, cxb))
    selection = {"top_1000_ms": 1e3 * t_top, "expansion_1000_ms": 1e3 * t_exp,
                 "n_candidates": int(cxa.numel()), "pt2_ms": 1e3 * t_pt2,
                 "pt2_candidates_per_s": cxa.numel() / t_pt2}

    # the outer iteration around the solve (Steps 1, 1', 2, 3 warm start): four
    # iterations of HiNqsLoop on this Hamiltonian, 200,000 seeded HF-weighted
    # determinant samples per iteration standing in for the Transformer's draws
    # (resident on the device before the clock starts); K_0 = 20,000, K = 10,000,
    # B_max = 40,000, N_e = 1000, mixed Davidson as in the step
    from paper_2606_26760_b300.loop import HiNqsLoop
    loop_opts = {k: v for k, v in solve_opts.items() if k != "trace_cap"}
    samples = [(torch.from_numpy(synth.hf_weighted_samples(n, na, 200_000, 900 + 2 * t).view(np.int64)).to(dev),
                torch.from_numpy(synth.hf_weighted_samples(n, nb, 200_000, 901 + 2 * t).view(np.int64)).to(dev))
               for t in range(4)]
    loop = HiNqsLoop(ham, k0=20_000, k=10_000, b_max=40_000, n_top=1000, davidson_opts=loop_opts)
    loop_iters = []
    for t in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec = loop.step(samples[t])
        torch.cuda.synchronize()
        loop_iters.append({"t": t, "ms": 1e3 * (time.perf_counter() - t0),
                           "candidates": rec.n_candidates, "basis": rec.n_basis,
                           "strings": [rec.n_alpha_strings, rec.n_beta_strings],
                           "energy": rec.energy, "warm_start": rec.warm_start})
    outer_loop = {"iterations": loop_iters,
                  "note": "HiNqsLoop.step: candidate pool, classical expansion (t >= 1), "
                          "H_xx or PT2 scores, basis update, product subspace, links, "
                          "warm-started mixed Davidson"}
    del loop, samples

    # the reference arm's sample on this GPU: the same whole path (subspace, FP64
    # ground state to a 1e-6 residual, RDMs, marginals) on the sub-problem of the
    # first 30 alpha and 30 beta strings, for a like-for-like ratio with that arm
    a30, b30 = a_d[:30].contiguous(), b_d[:30].contiguous()

    def small_step():
        ham_k = hq.Hamiltonian(h_d, eri_d, na, nb, w["e_nuc"])
        sub_k = hq.build_subspace(a30, b30, n, na, nb)
        la_k, lb_k = hq.string_links(ham_k, sub_k, 0), hq.string_links(ham_k, sub_k, 1)
        r_k = hq.davidson(ham_k, sub_k, la_k, lb_k, precision=hq.DAVIDSON_FP64,
                          tol_residual=1e-6, tol_energy=1e-8)
        hq.rdm(sub_k, la_k, lb_k, r_k.c)
        hq.spin_marginals(sub_k, r_k.c)
        return sub_k.N

    for _ in range(3):
        N_k = small_step()
    ts = []
    for _ in range(10):
        torch.cuda.synchronize()
        ev0.record(stream)
        small_step()
        ev1.record(stream)
        torch.cuda.synchronize()
        ts.append(ev0.elapsed_time(ev1) / 1e3)
    t_k = sum(ts) / len(ts)
    same_sample = {"value": sig3(N_k / t_k), "unit": "dets/s", "N": N_k,
                   "ms_per_step": sig3(1e3 * t_k),
                   "sample": "whole path on the first 30 x 30 strings, as the reference arm"}

    cpu, cpu_detail = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        H_o = oracle.Ham(w["h"], w["eri"], w["e_nuc"], na, nb)
        sa_o, sb_o = oracle.build_subspace(w["alpha"], w["beta"], na, nb)
        rows = np.sort(np.random.default_rng(0).choice(N, 4000, replace=False))
        c_h = c64.cpu().numpy()
        t0 = time.perf_counter()
        oracle.sigma(H_o, sa_o, sb_o, c_h, rows=rows)
        tcpu = time.perf_counter() - t0
        cpu = {"value": len(rows) / tcpu, "unit": "sigma dets/s", "cores": oracle.max_threads(),
               "kind": "oracle",
               "sample": f"{len(rows)} random rows of one FP64 sigma product of the {N}-determinant workload"}
        cpu_detail = cpu_baseline_detail(oracle, synth, np, H_o, sa_o, sb_o, c_h)
        cpu["single_core_dets_per_s"] = sig3(cpu_detail["single_core"]["value"])
        cpu["small_lanczos_time_to_1e-6_Ha_s"] = sig3(cpu_detail["small"]["time_to_1e-6_Ha_s"])

    t_mean = sum(times) / len(times)
    if world > 1:
        tt = torch.tensor([t_mean], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_mean = float(tt)
    value = world * N / t_mean
    e2e_mean = sum(e2e_times) / len(e2e_times)
    last = results[-1]
    # headline figures of the metric go last on the line (the part a tail keeps)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "dets/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_mean,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+bf16+f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: n_orb={n} n_alpha={na} n_beta={nb} "
                               f"{sub.Na}x{sub.Nb} strings, N={N} determinants",
                   "step": "ham+subspace+links+mixed Davidson to 1e-6 Ha+RDM backward+marginals",
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": world * N / e2e_mean, "unit": "dets/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": None if launches_per_step is None else launches_per_step * args.steps,
        "gpu_launches_note": "library kernels of one untimed step (profiler count) x steps; "
                             "the mixed solver's iteration count varies slightly between steps",
        "selection": {k: sig3(v) for k, v in selection.items()},
        "outer_loop_ms": [sig3(it["ms"]) for it in outer_loop["iterations"]],
        "same_sample_as_reference": same_sample,
        "cpu_baseline": cpu,
        "roofline": roof,
        "clocks": clk,
        "energy": {"mixed": last.energy, "fp64_ref": E_ref, "abs_err_Ha": sig3(abs(last.energy - E_ref)),
                   "mixed_sigmas_fp64_fp32": [last.n_sigma_fp64, last.n_sigma_fp32],
                   "fp64_sigmas": fp64_runs[-1].n_sigma_fp64, "mixed_status": last.status},
        "sigma_ms": {k: sig3(1e3 * v) for k, v in t_sig.items()},
        "sigma_dets_per_s": {k: sig3(N / v) for k, v in t_sig.items()},
        "time_to_1e-6_Ha_s": {"mixed_bf16c": sig3(tt_mixed), "fp64": sig3(tt_fp64),
                              **{k: sig3(v) for k, v in tt_variants.items()},
                              "speedup_mixed_vs_fp64": sig3(tt_fp64 / tt_mixed)
                              if (tt_fp64 and tt_mixed) else None},
    }
    if args.detail:
        print(json.dumps({"trace_mixed": results[-1].trace, "trace_fp64": fp64_runs[-1].trace,
                          "outer_loop": outer_loop, "cpu_detail": cpu_detail}), file=sys.stderr)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
