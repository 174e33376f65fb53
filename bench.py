#!/usr/bin/env python
"""Benchmark: atoms/s of lMBD energies + forces on one GB300 (replicas on N GPUs).

Workload: periodic random box of 4096 atoms at 0.1 atoms/A^3 (minimum separation
1.1 A, 4 species, synthetic free-atom parameters, Hirshfeld ratios U[0.6, 1]),
r_SCS = 5 A, MBD sphere 7 A (r_MBD,1 = r_MBD,2 = 7 A), 12 Gauss-Legendre
frequencies, series order 6, FP64 energies and forces.  A step is one call of
lmbd_energy_forces on the resident structure (all stages, forces included).

Prints one JSON line on rank 0.  ``--impl reference`` times the CPU oracle (the
project's plain float64 PyTorch implementation) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atoms/s for lMBD energy+forces on 1 GB300 (batched vs per-atom launch); serve p50/p99"
FP64_PEAK_TFLOPS = 1.25          # nominal GB300 FP64 (DFMA and DMMA), profiling recipe table
FP32_PEAK_TFLOPS = 80.5          # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (unit counts and clock)
# DRAM bytes (read + write) of the SCS factor kernel (k_scs_factor alone) per atom: ncu on the
# 512-atom box, profiles/ncu_scs_factor_box512.md; scaled to a launch by atoms / launches
SCS_FACTOR_DRAM_BYTES_PER_ATOM = 1.189e6
PRECISION = ("chain products: 6-digit (energy blocks) / 5-digit (adjoint-only blocks) bf16 Ozaki slices "
             "of the FP64 operands, exact integer recombination, FP64 scaling; adjoint pair product: "
             "5-digit slices; SCS: FP32 Cholesky and solves with FP64 iterative refinement to FP64 "
             "accuracy; everything else FP64")
PRECISION_FP64 = ("chain and adjoint pair products in FP64; SCS: FP32 Cholesky and solves with FP64 "
                  "iterative refinement to FP64 accuracy; everything else FP64")
WORKLOAD = ("periodic random box, 4096 atoms, 0.1 atoms/A^3, 4 species; r_SCS 5 A, MBD sphere 7 A "
            "(r_MBD,1 = r_MBD,2 = 7 A), 12 omega, n_max 6; energies + forces within 1e-10 rel. / "
            "1e-8 eV/A of the FP64 oracle (see precision)")
SAMPLE_ATOMS = 64                # oracle sample: same density and cutoffs, same local problem sizes
# digit-plane products per FP64 product of the sliced tensor-core kernels: S digits keep the
# pairs (k, l) with k + l <= S + 1, S (S + 1) / 2 of them (ozaki.cuh); the chain uses 6 digits for
# the energy blocks and 5 for the adjoint-only blocks, the pair kernel 5
DIG_E, DIG_A, DIG_P = 6, 5, 5


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--atoms", type=int, default=4096)
    ap.add_argument("--per-atom-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sweep", default=None,
                    help="comma-separated atom counts: atoms/s and HBM footprint per size (one JSON line each)")
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="device memory budget of the context for --sweep (0 = free memory less 1 GiB)")
    ap.add_argument("--serve", action="store_true", help="serving run: Poisson arrivals, continuous batching")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--hbm-gb", type=float, default=150.0)
    ap.add_argument("--max-atoms", type=int, default=20000)
    ap.add_argument("--large-slots", type=int, default=1,
                    help="slots of the large-request lane (normal-priority streams); 0 = no lanes")
    ap.add_argument("--large-atoms", type=int, default=2048)
    ap.add_argument("--omega-ref", type=float, default=0.0,
                    help="> 0: the paper's Lorentzian frequency model with this reference frequency (Ha)")
    ap.add_argument("--lanczos", type=int, default=0,
                    help="> 0: the paper's polynomial-fit series coefficients from this many Lanczos steps")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default SCS bucket width")
    ap.add_argument("--paper-forces", action="store_true",
                    help="the paper's approximate forces (Sec. III.D) instead of the exact gradient")
    ap.add_argument("--mma", default="tc05", choices=["warp", "tc05"],
                    help="tensor-core path of the sliced chain product: warp-level mma.sync or tcgen05")
    ap.add_argument("--precision", default="sliced", choices=["sliced", "fp64"],
                    help="arithmetic of the two large products: bf16 digit slices (default) or FP64")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the FP64-products measurement reported beside the default line (0 = skip)")
    ap.add_argument("--sparse-steps", type=int, default=2,
                    help="timed steps of the block-sparse T_LR comparison (0 = skip it)")
    ap.add_argument("--fit-nodes", type=int, default=0,
                    help="> 0: the paper's fitted integrand phi(omega) from omega = 0 and this many fit nodes")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def structure(n_atoms, seed):
    from paper_2407_06409_gb300 import inputs
    return inputs.box(n_atoms, density=0.1, min_sep=1.1, n_species=4, seed=seed)


# ----------------------------------------------------------------------------------------
# CPU oracle timing (baseline leg and the reference arm)
# ----------------------------------------------------------------------------------------
def oracle_step(sample):
    import oracle
    p = oracle.Params(r_scs=5.0, r_mbd1=7.0, r_mbd2=7.0, r_sphere=7.0, n_freq=12, series_order=6)
    so = oracle.System(sample.positions, sample.cell, sample.species, sample.hirshfeld, sample.table, p)
    t0 = time.perf_counter()
    so.energies_forces()
    return time.perf_counter() - t0


def cpu_sample(seed):
    return structure(SAMPLE_ATOMS, seed)


def sample_text():
    return (f"energies + forces of a {SAMPLE_ATOMS}-atom periodic box at the same density and cutoffs "
            "(every atom's K1/K2/sphere site lists, periodic images included, have the sizes of the "
            "4096-atom box); atoms/s = sample atoms / wall time")


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import torch
    cores = torch.get_num_threads()
    sample = cpu_sample(args.seed)
    for _ in range(max(0, args.warmup)):
        oracle_step(sample)
    times = [oracle_step(sample) for _ in range(max(1, args.steps))]
    t = statistics.mean(times)
    value = SAMPLE_ATOMS / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "atoms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "atoms": args.atoms, "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": value, "unit": "atoms/s", "cores": cores, "kind": "oracle",
                             "sample": sample_text()},
            "e2e": {"value": value, "unit": "atoms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.idx = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2407_06409_gb300 import build, lmbd

    if not os.path.exists(lmbd.LIB_PATH):
        build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    s = structure(args.atoms, args.seed + rank)
    model = lmbd.LMBD(s.table, lmbd.default_params(), 12, 6)
    if args.omega_ref > 0:
        model.set_frequency_model(lmbd.FREQ_LORENTZIAN, args.omega_ref)
    if args.fit_nodes > 0:
        model.set_integrand_fit(args.fit_nodes)
    if args.lanczos > 0:
        model.set_series_fit(args.lanczos)
    if args.paper_forces:
        model.set_force_model(lmbd.FORCES_PAPER)
    model.set_mma_path(lmbd.MMA_TC05 if args.mma == "tc05" else lmbd.MMA_WARP)
    if args.precision == "fp64":
        model.set_precision(lmbd.PREC_FP64)
    pos = torch.tensor(s.positions, device=dev)
    cell = torch.tensor(s.cell, device=dev)
    sp = torch.tensor(s.species, dtype=torch.int32, device=dev)
    nu = torch.tensor(s.hirshfeld, device=dev)
    stream = torch.cuda.current_stream(dev)

    # SCS launch shapes picked by the library's autotuner on this structure (untimed)
    bucket_width = None if args.no_autotune else model.autotune(pos, cell, sp, nu)
    for _ in range(max(3, args.warmup)):
        model.energy_forces(pos, cell, sp, nu, forces=True)
    torch.cuda.synchronize(dev)

    # ---- timed region: device-resident inputs --------------------------------------------
    model.set_profiling(True)
    sampler = ClockSampler(local)
    phase_ms, phase_flops, phase_launch = {}, {}, {}
    kernel_ms = {"scs_factor": 0.0, "scs_adjoint": 0.0}
    launches = 0
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        model.energy_forces(pos, cell, sp, nu, forces=True)
        st = model.stats()
        launches += st["kernel_launches"]
        for k in kernel_ms:
            kernel_ms[k] += st["ms_kernel"][k]
        for ph in lmbd.PHASES:
            phase_ms[ph] = phase_ms.get(ph, 0.0) + st["ms"][ph]
            phase_flops[ph] = phase_flops.get(ph, 0.0) + st["flops"][ph]
            phase_launch[ph] = phase_launch.get(ph, 0) + st["launches"][ph]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    model.set_profiling(False)
    from paper_2407_06409_gb300.replicas import job_throughput
    sec, value = job_throughput(ms_total * 1e-3, args.atoms * args.steps, device=dev)
    ms_total = sec * 1e3
    ms_step = ms_total / args.steps

    # ---- end to end: pinned host buffers, copies inside the timed region ------------------
    pos_h = torch.tensor(s.positions).pin_memory()
    cell_h = torch.tensor(s.cell).pin_memory()
    sp_h = torch.tensor(s.species, dtype=torch.int32).pin_memory()
    nu_h = torch.tensor(s.hirshfeld).pin_memory()
    model.energy_forces(pos_h, cell_h, sp_h, nu_h, forces=True)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e_h, f_h = model.energy_forces(pos_h, cell_h, sp_h, nu_h, forces=True)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s, e2e_value = job_throughput(e2e_s, args.atoms * args.steps, device=dev)
    e2e = {"value": e2e_value, "unit": "atoms/s",
           "h2d_bytes_per_step": int(pos_h.numel() * 8 + cell_h.numel() * 8 + sp_h.numel() * 4 + nu_h.numel() * 8),
           "d2h_bytes_per_step": int(e_h.numel() * 8 + f_h.numel() * 8)}

    # ---- plain one-launch-per-atom form, same arithmetic ----------------------------------
    per_atom = None
    if args.per_atom_steps > 0:
        model.set_launch_mode(lmbd.LAUNCH_PER_ATOM)
        torch.cuda.synchronize(dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.per_atom_steps):
            model.energy_forces(pos, cell, sp, nu, forces=True)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        pms = a0.elapsed_time(a1) / args.per_atom_steps
        per_atom = {"value": world * args.atoms / (pms * 1e-3), "ms_per_step": pms,
                    "launches_per_step": model.stats()["kernel_launches"]}
        model.set_launch_mode(lmbd.LAUNCH_BATCHED)

    # ---- the same workload with FP64 products (same run, fewer steps) -----------------------
    fp64_line = None
    if args.precision == "sliced" and args.fp64_steps > 0:
        model.set_precision(lmbd.PREC_FP64)
        model.energy_forces(pos, cell, sp, nu, forces=True)
        torch.cuda.synchronize(dev)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.fp64_steps):
            model.energy_forces(pos, cell, sp, nu, forces=True)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        fms = b0.elapsed_time(b1) / args.fp64_steps
        fp64_line = {"value": world * args.atoms / (fms * 1e-3), "unit": "atoms/s", "ms_per_step": fms,
                     "steps": args.fp64_steps, "warmup": 1, "precision": PRECISION_FP64}
        model.set_precision(lmbd.PREC_SLICED)

    # ---- block-sparse T_LR: the benchmark cutoffs and a split-cutoff sphere -----------------
    sparse_line = None
    if args.sparse_steps > 0 and world == 1:
        sparse_line = sparse_comparison(args, s, (pos, cell, sp, nu), dev, stream)

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel ---------------------------------------------------
    fp64 = ("scs", "chain", "adj_pair", "adj_scs")
    dom = max(fp64, key=lambda ph: phase_ms.get(ph, 0.0))
    avg_ms = phase_ms[dom] / max(1, phase_launch[dom])
    kernel_names = {"scs": "k_scs_factor", "chain": "k_chain_tc" if args.mma == "tc05" else "k_chain_oz2",
                    "adj_pair": "k_pair_tc" if args.mma == "tc05" else "k_mbd_adj_pair_oz2",
                    "adj_scs": "k_scs_adjoint2"}
    st_last = model.stats()
    if dom == "scs":
        # The SCS factor kernel.  Method work (the dense linear algebra of the local screening
        # solves): per centre and SCS frequency a Cholesky factorisation, (3 n1)^3 / 3 flops, and
        # 12 (3 n1)^2 for the triangular solves with 3 right-hand sides (the count of the work
        # estimate of the scope table, independent of how many refinement corrections the
        # kernel makes).  The factor runs on the FP32 SIMT pipe, so the peak is that pipe's
        # nominal rate from unit counts and the maximum clock.  Time: the kernel's own bucket
        # launches, fork to join (CUDA events around them in the library).
        nq = 2 if args.omega_ref > 0 else (args.fit_nodes + 2 if args.fit_nodes > 0 else 13)
        n1 = model.site_counts(args.atoms)[:, 0].astype(float)
        N1 = 3.0 * n1
        w_method = nq * float(np.sum(N1 ** 3 / 3.0 + 12.0 * N1 ** 2))
        n_fac = max(1, phase_launch[dom] // args.steps - 2)   # less k_pair_radial and k_scs_fill
        t_fac = kernel_ms["scs_factor"] / args.steps * 1e-3 if kernel_ms["scs_factor"] > 0 else avg_ms * 1e-3
        work = w_method / n_fac
        achieved = work / (t_fac / n_fac) / 1e12
        # the composite bound of the kernel's full instruction mix, as a second figure: FP32 work
        # (factor, three solves of 3 right-hand sides) plus the float-float right-hand side and
        # residuals (the FP64-equivalent flop count of those sums, each float-float multiply-add
        # about 20 FP32 operations, i.e. 10 per FP64 flop), all on the FP32 pipe
        w32 = nq * float(np.sum(N1 ** 3 / 3.0 + 18.0 * N1 ** 2))
        pairs, adj = float(st_last["scs_pairs"]), float(st_last["scs_adjacency"])
        wff = nq * (60.0 * adj + 36.0 * (pairs - adj / 2.0) + 2.0 * pairs)
        t_star = (w32 + 10.0 * wff) / (FP32_PEAK_TFLOPS * 1e12)
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS,
                    "traffic": SCS_FACTOR_DRAM_BYTES_PER_ATOM * args.atoms / n_fac,
                    "kernel": kernel_names[dom], "launches_per_step": n_fac, "ms_per_step": t_fac * 1e3,
                    "work_per_step": w_method,
                    "peak_note": "method flops sum_k nq [(3 n1)^3/3 + 12 (3 n1)^2] over the kernel's own time, "
                                 "against the FP32 SIMT pipe it runs on: 152 SMs x 128 lanes x 2 flops x "
                                 "2.07 GHz = 80.5 TFLOP/s nominal (unit counts and maximum clock)",
                    "composite": {"peak_note": "the kernel's whole instruction mix on the FP32 pipe (80.5 "
                                               "TFLOP/s): factor, solves and refinement corrections, plus the "
                                               "float-float right-hand side and residuals at 10 FP32 operations "
                                               "per FP64-equivalent flop",
                                  "work_fp32": w32, "work_float_float_fp64_equiv": wff, "t_star_ms": t_star * 1e3,
                                  "frac": t_star / t_fac}}
    elif dom in ("chain", "adj_pair"):
        # sliced products on the bf16 tensor cores: the bf16 work is the FP64 product's flops times
        # the digit pairs per product; peak = the measured sustained bf16 rate (timed inside a step)
        order, forces_on = 6, True
        nvec = order - 1 if forces_on else (order + 1) // 2
        pairs = lambda d: d * (d + 1) // 2
        if dom == "chain":
            per = [pairs(DIG_E if m + 1 <= (order + 1) // 2 else DIG_A) for m in range(1, nvec)]
            pair_mult = sum(per) / len(per)
        else:
            pair_mult = pairs(DIG_P)
        pk = measured_peaks()
        peak = pk.get("bf16_tflops_sustained") or 1700.0
        work = phase_flops[dom] / max(1, phase_launch[dom]) * pair_mult
        achieved = work / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else 0.0
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "kernel": kernel_names[dom],
                    "peak_note": ("bf16 digit-plane products (%.1f per FP64 product) against the measured "
                                  "sustained cuBLAS bf16 rate (MEASURED_PEAKS.json)" % pair_mult)
                    if pk.get("bf16_tflops_sustained") else "of fallback: 1.7 PFLOP/s sustained bf16"}
    else:
        flops_launch = phase_flops[dom] / max(1, phase_launch[dom])
        achieved = flops_launch / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else 0.0
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": kernel_names[dom],
                    "peak_note": "FP64 rate against the nominal FP64 peak"}
    phases = {ph: {"ms_per_step": phase_ms[ph] / args.steps, "launches_per_step": phase_launch[ph] // args.steps,
                   "tflops": (phase_flops[ph] / (phase_ms[ph] * 1e-3) / 1e12) if phase_ms[ph] > 0 and phase_flops[ph] > 0 else None}
              for ph in lmbd.PHASES}

    # ---- CPU baseline: the oracle on a bounded sample ---------------------------------------
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = torch.get_num_threads()
        sample = cpu_sample(args.seed)
        t = oracle_step(sample)
        cpu = {"value": SAMPLE_ATOMS / t, "unit": "atoms/s", "cores": cores, "kind": "oracle",
               "sample": sample_text()}

    st = model.stats()
    line = {"metric": METRIC, "value": value, "unit": "atoms/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + (f"; Lorentzian frequency model, omega_ref {args.omega_ref} Ha"
                                               if args.omega_ref > 0 else "")
                       + (f"; fitted integrand, {args.fit_nodes} fit nodes" if args.fit_nodes > 0 else "")
                       + (f"; polynomial-fit c_n, {args.lanczos} Lanczos steps" if args.lanczos > 0 else "")
                       + ("; the paper's approximate forces" if args.paper_forces else ""),
                       "atoms": args.atoms, "parallelism": f"replicas x{world}",
                       "l2": f"inputs resident; per-step working set {st['bytes_workspace'] / 1e9:.1f} GB > 129 MB L2",
                       "sites_per_atom": st["n_sites"] / args.atoms, "max_k1": st["max_k1"],
                       "scs_bucket_width": bucket_width, "chain_mma": args.mma,
                       "max_sphere": st["max_sphere"],
                       "precision": PRECISION if args.precision == "sliced" else PRECISION_FP64},
            "roofline": roofline, "phases": phases, "cpu_baseline": cpu, "e2e": e2e,
            "fp64_products": fp64_line, "sparse_tlr": sparse_line,
            "gpu_launches": launches, "per_atom_launch": per_atom, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# block-sparse T_LR (Sec. III.A: the secondary cutoff r_MBD,2) against the dense path
# ----------------------------------------------------------------------------------------
SPLIT_CUTOFFS = (6.0, 3.0)       # r_MBD,1, r_MBD,2 (A); sphere r_MBD,1 + r_MBD,2 = 9 A


def sparse_comparison(args, s, dev_args, dev, stream):
    """Energy+forces atoms/s of the dense and the block-sparse T_LR paths on the benchmark
    structure, at the benchmark cutoffs and with split MBD cutoffs (the paper's sphere
    r_MBD,1 + r_MBD,2), plus the rate of the sparse chain kernel on the FP32 pipe."""
    import torch
    from paper_2407_06409_gb300 import lmbd

    def timed(params, sparse):
        m = lmbd.LMBD(s.table, params, 12, 6)
        m.set_sparse_tlr(sparse)
        m.energy_forces(*dev_args, forces=True)
        torch.cuda.synchronize(dev)
        m.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        chain_ms = chain_flops = pair_ms = pair_flops = 0.0
        e0.record(stream)
        for _ in range(args.sparse_steps):
            m.energy_forces(*dev_args, forces=True)
            st = m.stats()
            chain_ms += st["ms"]["chain"]
            chain_flops += st["flops"]["chain"]
            pair_ms += st["ms"]["adj_pair"]
            pair_flops += st["flops"]["adj_pair"]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.sparse_steps
        out = {"value": args.atoms / (ms * 1e-3), "unit": "atoms/s", "ms_per_step": ms,
               "tlr_pairs": st["tlr_pairs"], "max_sphere": st["max_sphere"],
               "workspace_gb": st["bytes_workspace"] / 1e9}
        if sparse and chain_ms > 0:
            # 2 flops per FP64-equivalent multiply-add; a float-float multiply-add is 12 FP32
            # instructions (1 multiply, 3 FMAs for the exact product and cross terms, 6 for the
            # two-sum, 2 for the low part) on the 40.3 T instructions/s FP32 pipe
            for key, ms_k, fl in (("chain", chain_ms, chain_flops), ("adj_pair", pair_ms, pair_flops)):
                instr = fl / 2.0 * 12.0 / (ms_k * 1e-3)
                out[key] = {"ms_per_step": ms_k / args.sparse_steps,
                            "fp64_equiv_tflops": fl / (ms_k * 1e-3) / 1e12,
                            "fp32_issue_frac": instr / (FP32_PEAK_TFLOPS / 2.0 * 1e12)}
        del m
        torch.cuda.empty_cache()
        return out

    r1, r2 = SPLIT_CUTOFFS
    res = {"workload_bench": "the benchmark cutoffs (r_MBD,1 = r_MBD,2 = sphere 7 A)",
           "workload_split": f"the benchmark structure with r_MBD,1 {r1} A, r_MBD,2 {r2} A, sphere "
                             f"r_MBD,1 + r_MBD,2 = {r1 + r2} A",
           "steps": args.sparse_steps, "warmup": 1}
    res["bench_dense"] = timed(lmbd.default_params(), False)
    res["bench_sparse"] = timed(lmbd.default_params(), True)
    split = lmbd.default_params(r_mbd1=r1, r_mbd2=r2, r_sphere=0.0)
    res["split_dense"] = timed(split, False)
    res["split_sparse"] = timed(split, True)
    return res


# ----------------------------------------------------------------------------------------
# linear-scaling sweep: atoms/s and device footprint against N
# ----------------------------------------------------------------------------------------
def run_sweep(args):
    import torch
    from paper_2407_06409_gb300 import build, lmbd

    if not os.path.exists(lmbd.LIB_PATH):
        build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    for n in [int(x) for x in args.sweep.split(",") if x]:
        s = structure(n, args.seed)
        model = lmbd.LMBD(s.table, lmbd.default_params(), 12, 6)
        if args.budget_gb > 0:
            model.set_memory_budget(int(args.budget_gb * 1e9))
        pos = torch.tensor(s.positions, device=dev)
        cell = torch.tensor(s.cell, device=dev)
        sp = torch.tensor(s.species, dtype=torch.int32, device=dev)
        nu = torch.tensor(s.hirshfeld, device=dev)
        torch.cuda.synchronize(dev)
        free0, total = torch.cuda.mem_get_info(dev)
        model.energy_forces(pos, cell, sp, nu, forces=True)
        torch.cuda.synchronize(dev)
        free1, _ = torch.cuda.mem_get_info(dev)
        steps = max(1, args.steps)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            model.energy_forces(pos, cell, sp, nu, forces=True)
        ev1.record()
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1) / steps
        st = model.stats()
        line = {"mode": "sweep", "atoms": n, "atoms_per_s": n / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
                "warmup": 1, "device_bytes": st["bytes_workspace"], "arena_bytes": st["bytes_arena"],
                "device_used_delta": int(free0 - free1), "bytes_per_atom": st["bytes_workspace"] / n,
                "waves_scs": st["waves_scs"], "waves_mbd": st["waves_mbd"],
                "scs_recomputed": st["scs_recomputed"], "budget_gb": args.budget_gb or None,
                "device_total": int(total), "sites_per_atom": st["n_sites"] / n}
        print(json.dumps(line), flush=True)
        model.close()
        del pos, cell, sp, nu
    return 0


# ----------------------------------------------------------------------------------------
# serving: Poisson arrivals, continuous batching over several contexts
# ----------------------------------------------------------------------------------------
class MemSampler:
    """Device memory in use (cudaMemGetInfo) sampled from a host thread."""

    def __init__(self, dev, period=0.1):
        import threading
        self.dev, self.period = dev, period
        self.peak = 0
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        import torch
        while not self._stop.is_set():
            free, total = torch.cuda.mem_get_info(self.dev)
            self.peak = max(self.peak, total - free)
            self._stop.wait(self.period)

    def start(self):
        self._t.start()

    def stop(self):
        self._stop.set()
        self._t.join()
        return self.peak


def run_serve(args):
    import torch
    from paper_2407_06409_gb300 import build, inputs, lmbd, serve

    if not os.path.exists(lmbd.LIB_PATH):
        build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    table, items = inputs.serving_workload(args.requests, rate=args.rate, lo=50, hi=args.max_atoms,
                                           seed=args.seed)
    t_gen = time.perf_counter() - t_gen
    engines = serve.make_engines(table, args.slots, args.large_slots)
    warm = inputs.box(200, seed=12345, table=table)
    for e in engines:
        e.run(warm, 50e9)
        e.release()
    torch.cuda.synchronize(dev)
    free0, total = torch.cuda.mem_get_info(dev)
    srv = serve.Server(engines, hbm_bytes=args.hbm_gb * 1e9, large_atoms=args.large_atoms,
                       large_slots=args.large_slots)
    mem = MemSampler(dev)
    clocks = ClockSampler(0)
    mem.start()
    clocks.start()
    res = srv.serve(items, realtime=True)
    clk = clocks.stop()
    peak_used = mem.stop()
    summ = serve.summarize(res, large_atoms=args.large_atoms)
    sizes = [r.n_atoms for r in res]
    line = {"mode": "serve", "metric": "lMBD serving (energies + forces): p50/p99 latency and atoms/s",
            **summ, "rate_req_per_s": args.rate, "slots": args.slots, "hbm_cap_gb": args.hbm_gb,
            "lanes": {"large_slots": srv.large_slots, "large_atoms": args.large_atoms},
            "peak_reserved_gb": srv.peak_accounted / 1e9,
            "peak_device_used_gb_above_idle": (peak_used - (total - free0)) / 1e9,
            "idle_slot_releases": srv.releases, "md_frames": sum(1 for it in items if it.frame > 0),
            "size_range": [int(min(sizes)), int(max(sizes))], "mean_atoms": float(sum(sizes) / len(sizes)),
            "workload_gen_s": t_gen, "dtype": "f64", "data": "synthetic", "clocks": clk}
    if summ["errors"]:
        line["first_error"] = next(r.error for r in res if r.error)
    print(json.dumps(line), flush=True)
    for e in engines:
        e.close()
    return 0 if summ["errors"] == 0 else 1


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.sweep:
        return run_sweep(args)
    if args.serve:
        return run_serve(args)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
