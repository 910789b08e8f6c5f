#!/usr/bin/env python3
"""Benchmark of the exact-diagonalization solver: solves/s on one synthetic cluster workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 4x4|cdmft|2x4] [--precision fp32|fp64] [--gf band|cf|none]

A step is one whole solve through the C ABI: ed_cluster_create (basis and hopping tables),
ed_ground_state (Lanczos, retrace, FP64 polish) and ed_green (starting vectors, Lanczos /
band Lanczos, G on the frequency grid), then ed_cluster_destroy.  Under torchrun every rank
solves its own seeded instance of the workload (independent problems, no data exchange):
weak scaling, value = solves of all ranks / max-over-ranks time.

The JSON line carries the kernel roofline of the fused Lanczos step (the dominant kernel),
measured with CUDA events on the library's stream over the timed region, and a CPU baseline:
the oracle timed on a bounded sample of the same workload.  ``--impl reference`` times that
oracle instead of the GPU path.
"""

from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_18643_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    # name: (generator(instance), label, default precision, default gf, frequencies)
    "4x4": (W.periodic_4x4, "4x4 periodic Hubbard, t=-1, t'=0.3 seeded sign, U=8, mu=4, N_up=N_dn=8 (d=12870^2); "
            "ground state + band-Lanczos G from the 16 c+/c starting vectors on 1000 Matsubara frequencies "
            "(beta=50)", "fp32", "band", 1000),
    "cdmft": (W.cdmft_2x2_bath, "2x2 plaquette + 8 bath, U=8, mu=4, N_up=N_dn=6 (d=924^2)", "fp32", "cf", 1000),
    "2x4": (lambda instance=0: W.plain_2x4(), "2x4 open Hubbard, U=4, mu=2, N_up=N_dn=4 (d=70^2)", "fp64", "cf", 1000),
    "2x7": (lambda instance=0: W.served_request(np.random.default_rng(20230529 + 7000 + instance), sizes=(14,)),
            "2x7 open Hubbard, t=-1, t'=+-0.3 seeded, U=8, mu=4, N_up=N_dn=7 (d=3432^2); band-Lanczos G on 1000 "
            "Matsubara frequencies (beta=50)", "fp32", "band", 1000),
    "hpsi": (W.periodic_4x4, "standalone H.psi of the band Lanczos: 4x4 periodic cluster, sector N_up=9, N_dn=8 "
             "(11440 x 12870 = 147,232,800 states, rows padded to 12928), FP32 vectors (two-pass kernels)",
             "fp32", "none", 0),
    "batch": (lambda instance=0: W.batched_family(512, instance=instance),
              "512 seeded clusters of 4-12 orbitals (chains, 2-leg ladders, 2x2 plaquettes + 0-8 bath), "
              "|t| ~ U[0.5,1.5], U ~ U[2,10], mu = U/2, random fillings; both spins", "fp32", "cf", 512),
    "sym": (lambda instance=0: W.open_3x4_c2v()[0],
            "3x4 open Hubbard, t=-1, U=4, mu=2, N_up=N_dn=6 (d=853,776) in its C2v irrep sectors (213,248-213,840 "
            "states); ground state + G of the 12 sites on 64 Matsubara frequencies (beta=50)", "fp64", "cf", 64),
    "lattice": (W.cdmft_2x2_bath,
                "lattice steps fed by the 2x2 plaquette + 8 bath impurity (U=8, mu=4, N_up=N_dn=6): CPT of the "
                "square lattice (t=-1, t'=0.3) periodized on a 64x64 k grid x 256 Matsubara frequencies, CDMFT "
                "target on a 16x16 reduced zone, distance + gradient for 64 trial baths", "fp64", "cf", 256),
    "davidson": (W.cdmft_2x2_bath,
                 "2x2 plaquette + 8 bath, U=8, mu=4, N_up=N_dn=6 (d=924^2): the 4 lowest states (block Davidson) "
                 "and the mixed-state G at T=0.05 on 256 Matsubara frequencies (beta=50), FP64", "fp64", "cf", 256),
    "served": (None, "stream of solve requests: open 2xW clusters of 8/10/12/14 orbitals (uniform), t=-1, "
               "t'=+-0.3 seeded per bond, U=8, mu=4, half filling; ground state + G on 2048 Matsubara "
               "frequencies (beta=50); continued fractions up to 10 orbitals, band Lanczos from 12",
               "fp32", "mixed", 2048),
}
ETA = 0.05
BETA = 50.0
# Krylov vectors per part of the band Green function: the paper's runs stop at R = 100-500 (Sec. 4.4)
BAND_MAX_DIM = {"4x4": 512, "2x7": 512}
# Frequency axis of the single-cluster workloads' G.  The band workloads (4x4, 2x7) evaluate G on
# the Matsubara axis, where the CDMFT loop and the VCA integrals of the paper consume it (Secs. 5-6)
# and where a band run converges on the grid within its preset maximum; on the real axis at
# eta = 0.05 the 4x4 band space of 512 vectors per part is far from resolving the spectrum (its
# FP32 and FP64 G then differ by O(1) there, both unconverged).
AXIS = {"4x4": "matsubara", "2x7": "matsubara", "cdmft": "real", "2x4": "real"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="4x4")
    ap.add_argument("--requests", type=int, default=32, help="served workload: requests per stream")
    ap.add_argument("--clusters", type=int, default=512, help="batch workload: clusters (512 is the named workload)")
    ap.add_argument("--max-orb", type=int, default=12, help="batch workload: largest cluster (orbitals)")
    ap.add_argument("--rates", type=str, default="1,4,16",
                    help="served workload: Poisson arrival rates as multiples of 1 / (mean sequential FP64 solve time)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default=None)
    ap.add_argument("--gf", choices=["band", "cf", "none"], default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="single-cluster workloads: timed solves of the plain FP64 GPU path on the same config "
                         "(fp64_value beside the FP32-storage value; 0 skips it)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sequential", type=int, default=0,
                    help="batch workload: also time this many clusters one by one through the single-cluster "
                         "FP64 path (the plain FP64 GPU path, continued fractions run to convergence as in the "
                         "batch) and report its solves/s")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world, device):
    """The largest x over all ranks (the timed region of the slowest rank); x itself at N = 1."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second of the slowest rank's timed region (weak scaling:
    every rank solves its own seeded instances, no data exchange)."""
    return world * units_per_rank / (ms / 1e3)


# ----------------------------------------------------------------------------- measurement helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for r in csv.reader(io.StringIO(out)):
            if len(r) >= 9:
                self.rows.append([x.strip() for x in r])

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": float(np.median(load)) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# The source of the two-pass H.psi kernels (everything between these markers of hpsi.cu): a
# committed ncu summary's traffic is used only while this text is the one it was taken on.
TWO_PASS_SLICE = ("// ---- two-pass form for vectors larger than L2", "constexpr int kRowsPerCta")


def kernel_source_hash(kernel_file):
    """sha256 (16 hex digits) of the two-pass kernels' source text in kernel_file."""
    txt = open(os.path.join(ROOT, "paper_2305_18643_gb300", "csrc", kernel_file)).read()
    a, b = txt.index(TWO_PASS_SLICE[0]), txt.index(TWO_PASS_SLICE[1])
    return hashlib.sha256(txt[a:b].encode()).hexdigest()[:16]


def ncu_traffic(kernel_file, summary_file):
    """(DRAM bytes, algorithmic bytes) of one captured launch from a committed ncu summary, if it
    was taken on this kernel source, else None."""
    p = os.path.join(ROOT, "profiles", summary_file)
    try:
        txt = open(p).read()
        sha = kernel_source_hash(kernel_file)
        m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
        t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
        a = re.search(r"alg_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
        if m and t and a and m.group(1) == sha:
            return float(t.group(1)), float(a.group(1))
    except OSError:
        pass
    return None


def scaled_traffic(captured, alg_bytes_per_launch):
    """DRAM bytes per launch of the timed kernel from a captured launch of the same kernels:
    traffic grows in proportion to the elements processed, so it is scaled by the algorithmic
    bytes (a timed launch may carry 16 products, or another sector, than the captured one)."""
    if not captured or not alg_bytes_per_launch:
        return None
    return captured[0] * alg_bytes_per_launch / captured[1]


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2305_18643_gb300 import build, ed

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build.build()
    ed.lib()
    gen, label, prec_d, gf_d, nfreq = WORKLOADS[args.workload]
    prec = args.precision or prec_d
    gf = args.gf or gf_d
    if args.workload == "batch":
        return run_batch(args, rank, world, local_rank, torch, ed)
    if args.workload == "served":
        return run_served(args, rank, world, local_rank, torch, ed)
    if args.workload == "hpsi":
        return run_hpsi(args, rank, world, local_rank, torch, ed)
    if args.workload == "sym":
        return run_sym(args, rank, world, local_rank, torch, ed)
    if args.workload == "lattice":
        return run_lattice(args, rank, world, local_rank, torch, ed)
    if args.workload == "davidson":
        return run_davidson(args, rank, world, local_rank, torch, ed)
    c = gen(instance=rank)
    ns = c["t"].shape[0]
    axis_name = AXIS.get(args.workload, "real")
    omega = W.matsubara_grid(nfreq, BETA) if axis_name == "matsubara" else W.real_grid(nfreq)
    axis = ed.ED_AXIS_MATSUBARA if axis_name == "matsubara" else ed.ED_AXIS_REAL
    precision = ed.ED_FP32 if prec == "fp32" else ed.ED_FP64
    gf_method = ed.ED_GF_BAND if gf == "band" else ed.ED_GF_CF
    G_dev = torch.empty((nfreq, ns, ns, 2), dtype=torch.float64, device="cuda")
    info = {}
    band_dim = BAND_MAX_DIM.get(args.workload)

    def solve(to_host):
        h = ed.ed_cluster_create(c, precision=precision, gf_method=gf_method, seed=1234 + rank)
        try:
            if band_dim:
                ed.ed_set_option(h, ed.ED_OPT_BAND_MAX_DIM, band_dim)
            st, E0, res, it = ed.ed_ground_state(h)
            info.update(E0=E0, residual=res, gs_iters=it, gs_status=st)
            if gf != "none":
                if to_host:
                    st, G = ed.ed_green(h, omega, ETA, ns, axis=axis)  # host buffer: the library copies G out
                else:
                    st, _ = ed.ed_green(h, omega, ETA, ns, axis=axis, out_ptr=G_dev.data_ptr())
                info["green_status"] = st
                info["gf_steps"], info["gf_max_steps"] = ed.ed_green_stats(h)
        finally:
            ed.ed_cluster_destroy(h)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def timed(to_host, steps, profile):
        barrier()
        if profile:
            ed.ed_profile_enable(1)
        launches0 = ed.ed_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            solve(to_host)
        e1.record()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        launches = ed.ed_launch_count() - launches0
        return ms, launches

    for _ in range(args.warmup):
        solve(False)
    with ClockSampler(local_rank) as clk:
        ms, launches = timed(False, args.steps, True)
    prof = {k: ed.ed_profile_read(k) for k in range(ed.ED_K_COUNT)}
    ed.ed_profile_enable(0)
    e2e = None
    if not args.no_e2e:
        ms_e2e, _ = timed(True, args.steps, False)
        e2e = {"value": whole_job_rate(args.steps, world, ms_e2e), "unit": "solves/s",
               "h2d_bytes_per_step": int(8 * (ns * ns + ns + len(c["eps"]) + c["theta"].size + 1)),
               "d2h_bytes_per_step": int(nfreq * ns * ns * 16 if gf != "none" else 0) + 8}
    value = whole_job_rate(args.steps, world, ms)
    peak, peak_kind = measured_peak_hbm()
    peak_src = peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind

    def roofline_of(kid, name, captured):
        n_l, ms_l, by_l = prof[kid]
        ach = (by_l / 1e9) / (ms_l / 1e3) if ms_l > 0 else None
        traffic = scaled_traffic(captured, by_l / max(n_l, 1))
        return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": (ach / peak) if ach else None, "traffic": traffic, "peak_source": peak_src,
                "launches": n_l, "total_ms": ms_l, "avg_launch_ms": ms_l / max(n_l, 1),
                "alg_bytes_per_launch": by_l / max(n_l, 1)}

    big = args.workload == "4x4"
    rl_step = roofline_of(ed.ED_K_LANCZOS_STEP, "lanczos_step (fused H.psi + Lanczos epilogue: read v_n, v_{n-1}, "
                          "write w; 3 d s bytes)", ncu_traffic("hpsi.cu", "lanczos_step_4x4.md") if big else None)
    rl_hpsi = roofline_of(ed.ED_K_HPSI, "hpsi (standalone H.psi of the band Lanczos blocks and the FP64 residuals: "
                          "read x, write y; 2 d s bytes)", ncu_traffic("hpsi.cu", "band_hpsi_4x4.md") if big else None)
    # the roofline reported is that of the kernel family with the larger share of the timed region
    dominant, other = (rl_hpsi, rl_step) if rl_hpsi["total_ms"] > rl_step["total_ms"] else (rl_step, rl_hpsi)
    # H.psi per solve, counted in products of the ground-state sector's size: element-products from
    # the algorithmic bytes the library records (3 s per element for a fused step, 2 s for a
    # standalone product; band blocks launch 16 products at once), over d of the sector
    es_ = 4.0 if prec == "fp32" else 8.0
    d0 = math.comb(c["t"].shape[0] + len(c["eps"]), c["n_up"]) * math.comb(c["t"].shape[0] + len(c["eps"]), c["n_dn"])
    elem = prof[ed.ED_K_LANCZOS_STEP][2] / (3 * es_) + prof[ed.ED_K_HPSI][2] / (2 * es_)
    hpsi_per_solve = elem / d0 / max(args.steps, 1)
    green_st = info.get("green_status")
    result = {
        "metric": "ED solves/s (H.psi HBM GB/s and % roofline in `roofline`)",
        "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors, f64 reductions and recurrence, f64-refined ground state" if prec == "fp32" else "f64",
        "data": "synthetic (seeded cluster parameters)",
        "config": {"workload": args.workload + ": " + label, "precision": prec, "green_function": gf,
                   "n_freq": nfreq if gf != "none" else 0, "axis": axis_name,
                   "eta": ETA if axis_name == "real" else None, "beta": BETA if axis_name == "matsubara" else None,
                   "band_krylov_per_part": BAND_MAX_DIM.get(args.workload) if gf == "band" else None,
                   "l2": "inputs larger than L2 (state vectors 0.66-1.33 GB)" if big
                   else "L2 flushed by the step's own traffic",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": dominant,
        "roofline_other": other,
        "solve": {k: info.get(k) for k in ("E0", "residual", "gs_iters", "gs_status", "green_status", "gf_steps",
                                           "gf_max_steps")},
        "kernels_ms": {ed.ed_profile_kernel_name(k): round(v[1], 3) for k, v in prof.items() if v[0]},
        "hpsi_per_solve": hpsi_per_solve,
    }
    if gf == "band":
        result["solve"]["green_stop"] = (
            "converged on the grid" if green_st == ed.ED_OK else
            "preset maximum of %s Krylov vectors per part reached (ED_WARN_NOT_CONVERGED)" % band_dim
            if green_st == ed.ED_WARN_NOT_CONVERGED else "status %s" % green_st)
    if args.fp64_steps > 0 and prec == "fp32":
        result["fp64_arm"] = fp64_arm(args, c, gf_method, band_dim, omega, axis, ns, G_dev, info, world, torch, ed)
        result["fp32_value"] = value
        result["fp64_value"] = result["fp64_arm"]["value"]
        result["fp32_vs_fp64_speedup"] = value / result["fp64_value"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.workload, c, hpsi_per_solve)
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


def run_hpsi(args, rank, world, local_rank, torch, ed):
    """Kernel-level workload: y = H x on the electron sector (N_up + 1, N_dn) of the 4x4 cluster,
    the product the band Lanczos applies to each vector of a block, FP32 (or --precision fp64)
    vectors with rows padded to 128 elements (the two-pass kernels).  A step is 16 products (one
    block); value = products/s, roofline = 2 d s bytes per product over its CUDA-event time."""
    gen, label, prec_d, gf_d, nfreq = WORKLOADS["hpsi"]
    prec = args.precision or prec_d
    c = gen(instance=rank)
    precision = ed.ED_FP32 if prec == "fp32" else ed.ED_FP64
    tdt = torch.float32 if prec == "fp32" else torch.float64
    nu, nd = c["n_up"] + 1, c["n_dn"]
    cl = ed.Cluster(c, precision=precision)
    du, dd = ed.ed_sector_dims(cl.h, nu, nd)
    ld = (dd + 127) // 128 * 128
    g = torch.Generator(device="cuda")
    g.manual_seed(5 + rank)
    x = torch.zeros((du, ld), dtype=tdt, device="cuda")
    x[:, :dd] = torch.rand((du, dd), generator=g, device="cuda", dtype=tdt) * 2 - 1
    y = torch.zeros_like(x)
    stream = torch.cuda.current_stream().cuda_stream
    per_step = 16

    def step():
        for _ in range(per_step):
            ed.ed_hpsi(cl.h, nu, nd, precision, x.data_ptr(), y.data_ptr(), ld, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ed.ed_profile_enable(1)
    l0 = ed.ed_launch_count()
    with ClockSampler(local_rank) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    launches = ed.ed_launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    n_l, ms_l, by_l = ed.ed_profile_read(ed.ED_K_HPSI)
    ed.ed_profile_enable(0)
    peak, peak_kind = measured_peak_hbm()
    ach = (by_l / 1e9) / (ms_l / 1e3) if ms_l > 0 else None
    cl.close()
    es = 4 if prec == "fp32" else 8
    return {
        "metric": "H.psi HBM GB/s (% roofline), band-Lanczos sector of the 4x4 cluster",
        "value": whole_job_rate(args.steps * per_step, world, ms), "unit": "H.psi/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
        "data": "synthetic (uniform random vector, seeded)",
        "config": {"workload": "hpsi: " + label, "products_per_step": per_step,
                   "l2": "inputs larger than L2 (%.2f GB per vector)" % (du * ld * es / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(), "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "hpsi (two-pass: k_down_rows + k_up_cols)", "achieved": ach,
                     "peak": peak, "unit": "GB/s", "frac": (ach / peak) if ach else None,
                     "traffic": scaled_traffic(ncu_traffic("hpsi.cu", "band_hpsi_4x4.md"), by_l / max(n_l, 1)),
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                     "launches": n_l, "avg_launch_ms": ms_l / max(n_l, 1), "alg_bytes_per_launch": by_l / max(n_l, 1)},
        "e2e": None,
    }


def run_sym(args, rank, world, local_rank, torch, ed):
    """Symmetrized sectors (Sec. 4.5-4.6): a step is one solve of the 3x4 cluster in the C2v irrep
    that holds its ground state (basis, stored matrix, FP64 Lanczos ground state, G of the 12
    sites by continued fractions in the N +- 1 product irreps); value = solves/s.  Beside it, the
    same solve on the unsymmetrized sectors (ed_ground_state + ed_green, FP64 continued fractions)
    and the largest difference of the two G.  Roofline: the stored-matrix product (12 bytes per
    entry + 16 per row) over its profiled time; the irrep matrices (~46 MB) sit in L2, so the rate
    is an effective one."""
    gen, label, prec_d, gf_d, nfreq = WORKLOADS["sym"]
    c, gens = W.open_3x4_c2v()
    ns = c["t"].shape[0]
    omega = W.matsubara_grid(nfreq, BETA)
    h = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=ed.ED_GF_CF, seed=1234, tol=1e-12)
    # the irrep of the ground state (lowest irrep energy), found once before timing
    best = None
    for ir in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
        s = ed.ed_sym_create(h, np.array(gens), ir)
        try:
            E = ed.ed_sym_ground_state(s)[0]
        finally:
            ed.ed_sym_destroy(s)
        if best is None or E < best[1]:
            best = (ir, E)
    info = {}

    def solve():
        s = ed.ed_sym_create(h, np.array(gens), best[0])
        try:
            E, r, it, st = ed.ed_sym_ground_state(s)
            info.update(E0=E, residual=r, iters=it, dim=ed.ed_sym_info(s)[0], nnz=ed.ed_sym_info(s)[1])
            info["G"] = ed.ed_sym_green(s, omega, ns, axis=ed.ED_AXIS_MATSUBARA)
        finally:
            ed.ed_sym_destroy(s)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    ed.ed_profile_enable(1)
    l0 = ed.ed_launch_count()
    with ClockSampler(local_rank) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            solve()
        e1.record()
        torch.cuda.synchronize()
    launches = ed.ed_launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    n_l, ms_l, by_l = ed.ed_profile_read(ed.ED_K_HPSI)
    ed.ed_profile_enable(0)
    # the same solve on the unsymmetrized sectors
    e0.record()
    h2 = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=ed.ED_GF_CF, seed=1234, tol=1e-12)
    try:
        st, E_full, r_full, _ = ed.ed_ground_state(h2)
        G_full = ed.ed_green(h2, omega, 0.0, ns, axis=ed.ED_AXIS_MATSUBARA)[1]
    finally:
        ed.ed_cluster_destroy(h2)
    e1.record()
    torch.cuda.synchronize()
    ms_full = e0.elapsed_time(e1)
    ed.ed_cluster_destroy(h)
    peak, peak_kind = measured_peak_hbm()
    ach = (by_l / 1e9) / (ms_l / 1e3) if ms_l > 0 else None
    return {
        "metric": "ED solves/s in the ground state's irrep sectors (Sec. 4.5-4.6)",
        "value": whole_job_rate(args.steps, world, ms), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (fixed cluster parameters)",
        "config": {"workload": "sym: " + label, "irrep_generator_signs": list(best[0]), "irrep_dim": info["dim"],
                   "stored_entries": info["nnz"], "n_freq": nfreq, "axis": "matsubara", "beta": BETA,
                   "l2": "irrep matrices L2-resident (%.0f MB)" % (info["nnz"] * 12 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(), "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "k_sym_spmv (stored irrep matrix times a vector)", "achieved": ach,
                     "peak": peak, "unit": "GB/s", "frac": (ach / peak) if ach else None, "traffic": None,
                     "peak_source": peak_kind, "launches": n_l, "avg_launch_ms": ms_l / max(n_l, 1),
                     "alg_bytes_per_launch": by_l / max(n_l, 1),
                     "note": "effective rate: the matrix and vectors of an irrep fit in L2"},
        "solve": {"E0": info["E0"], "residual": info["residual"], "gs_iters": info["iters"]},
        "unsymmetrized_fp64": {"value": 1e3 / ms_full, "unit": "solves/s", "ms": ms_full, "E0": E_full,
                               "E0_minus_irrep": E_full - info["E0"],
                               "G_max_abs_diff": float(np.max(np.abs(G_full - info["G"]))),
                               "how": "ed_cluster_create, ed_ground_state, ed_green (continued fractions) on the "
                                      "853,776-state sector and its N +- 1 sectors, FP64"},
        "speedup_vs_unsymmetrized": (1e3 / (ms / args.steps)) / (1e3 / ms_full),
        "e2e": None,
    }


def run_lattice(args, rank, world, local_rank, torch, ed):
    """The lattice steps that consume the solver's G (Secs. 3 and 6): the impurity's G_c on the
    Matsubara grid is computed once (untimed); a step is CPT periodized on a 64 x 64 grid of wave
    vectors (Eqs. CPT1, CPT3, with the bath's Gamma), the CDMFT target on a 16 x 16 reduced zone
    and the distance with its gradient for 64 trial baths.  value = CPT (k, omega) points per
    second of the whole step; the kernels are FP64 complex arithmetic on small matrices."""
    gen, label, prec_d, gf_d, nfreq = WORKLOADS["lattice"]
    c = gen(instance=rank)
    ns = c["t"].shape[0]
    om = W.matsubara_grid(nfreq, BETA)
    z = 1j * om
    h = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=ed.ED_GF_CF, seed=1234)
    try:
        Gc = ed.ed_green(h, om, 0.0, ns, axis=ed.ED_AXIS_MATSUBARA)[1]
    finally:
        ed.ed_cluster_destroy(h)
    lat = W.square_superlattice(2, 2, t=-1.0, tp=0.3)
    Gam = ed.ed_hybridization(c["theta"], c["eps"], z)
    k_cpt = W.reduced_zone(lat["E"], (64, 64))
    k_cdmft = W.reduced_zone(lat["E"], (16, 16))
    rng = np.random.default_rng(7 + rank)
    nb = c["eps"].size
    th = np.asarray(c["theta"])[None] * (1.0 + 0.05 * rng.standard_normal((64, ns, nb)))
    ep = np.asarray(c["eps"])[None] + 0.05 * rng.standard_normal((64, nb))
    wts = np.ones(nfreq) / nfreq

    def step():
        ed.ed_cpt_green(lat, Gc, k_cpt, mode=ed.ED_CPT_PERIODIZED, Gamma=Gam)
        A = ed.ed_cdmft_target(lat, Gc, k_cdmft, Gamma=Gam)
        ed.ed_cdmft_distance(th, ep, z, wts, A, grad=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ed.ed_profile_enable(1)
    l0 = ed.ed_launch_count()
    with ClockSampler(local_rank) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    launches = ed.ed_launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    n_l, ms_l, by_l = ed.ed_profile_read(ed.ED_K_LATTICE)
    ed.ed_profile_enable(0)
    npts = len(k_cpt) * nfreq
    return {
        "metric": "CPT (k, omega) points/s of the lattice step (CPT + CDMFT target + distance)",
        "value": whole_job_rate(args.steps * npts, world, ms), "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 complex", "data": "synthetic (seeded bath)",
        "config": {"workload": "lattice: " + label, "cpt_points": npts, "cdmft_k": len(k_cdmft),
                   "trial_baths": 64, "n_freq": nfreq, "beta": BETA,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(), "gpu_launches": int(launches),
        "roofline": None,
        "roofline_note": "FP64 complex Gauss-Jordan on 4x4 matrices (warp per matrix): bound by FP64 "
                         "arithmetic and latency, not HBM; no measured FP64 peak is committed, so no fraction "
                         "is quoted",
        "kernels_ms": {"lattice": round(ms_l, 3), "launches": n_l},
        "e2e": None,
    }


def run_davidson(args, rank, world, local_rank, torch, ed):
    """Several low states (Sec. 4.2; the Davidson_states and temperature options of Sec. 9): a step
    is one solve of the impurity cluster for its 4 lowest states by block Davidson plus the
    mixed-state G at T = 0.05 (continued fractions from each state); value = solves/s.  Beside it,
    the single-state solve (Lanczos ground state + G) of the same cluster."""
    gen, label, prec_d, gf_d, nfreq = WORKLOADS["davidson"]
    c = gen(instance=rank)
    ns = c["t"].shape[0]
    om = W.matsubara_grid(nfreq, BETA)
    info = {}

    def solve(states):
        h = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=ed.ED_GF_CF, seed=1234)
        try:
            if states > 1:
                ed.ed_set_option(h, ed.ED_OPT_DAVIDSON_STATES, states)
                ed.ed_set_option(h, ed.ED_OPT_TEMPERATURE, 0.05)
            st, E0, r, it = ed.ed_ground_state(h)
            info.update(E0=E0, residual=r, iters=it, status=st)
            info["G"] = ed.ed_green(h, om, 0.0, ns, axis=ed.ED_AXIS_MATSUBARA)[1]
            if states > 1:
                E, wts = ed.ed_low_states(h)
                info.update(E=E.tolist(), weights=wts.tolist())
        finally:
            ed.ed_cluster_destroy(h)

    for _ in range(args.warmup):
        solve(4)
    torch.cuda.synchronize()
    l0 = ed.ed_launch_count()
    with ClockSampler(local_rank) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            solve(4)
        e1.record()
        torch.cuda.synchronize()
    launches = ed.ed_launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    mixed = dict(info)
    e0.record()
    solve(1)
    e1.record()
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    return {
        "metric": "ED solves/s with 4 low states and the mixed-state G (block Davidson)",
        "value": whole_job_rate(args.steps, world, ms), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded bath)",
        "config": {"workload": "davidson: " + label, "states": 4, "temperature": 0.05, "n_freq": nfreq,
                   "beta": BETA, "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(), "gpu_launches": int(launches),
        "roofline": None,
        "roofline_note": "the FP64 H.psi of the Davidson basis is the FP64 path's kernel (FP64-ALU-bound); the "
                         "sector (6.8 MB per vector) is L2-resident",
        "solve": {"E": mixed.get("E"), "weights": mixed.get("weights"), "max_residual": mixed["residual"],
                  "iters": mixed["iters"], "status": mixed["status"]},
        "single_state": {"value": 1e3 / ms1, "unit": "solves/s", "ms": ms1, "E0": info["E0"],
                         "how": "ed_ground_state (Lanczos) + ed_green on the same cluster, FP64"},
        "e2e": None,
    }


def fp64_arm(args, c, gf_method, band_dim, omega, axis, ns, G32_dev, info32, world, torch, ed):
    """The plain FP64 GPU path on the same cluster, frequencies and Krylov size: --fp64-steps
    solves timed with CUDA events, and the difference of its E0 and G from the FP32-storage arm's
    last solve (whose G is still in G32_dev)."""
    G64 = torch.empty_like(G32_dev)
    res = {}

    def solve():
        h = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=gf_method, seed=1234)
        try:
            if band_dim:
                ed.ed_set_option(h, ed.ED_OPT_BAND_MAX_DIM, band_dim)
            st, E0, r, it = ed.ed_ground_state(h)
            res.update(E0=E0, residual=r, gs_iters=it)
            st, _ = ed.ed_green(h, omega, ETA, ns, axis=axis, out_ptr=G64.data_ptr())
            res["green_status"] = st
            res["gf_steps"] = ed.ed_green_stats(h)
        finally:
            ed.ed_cluster_destroy(h)

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.fp64_steps):
        solve()
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    dG = float((G32_dev - G64).abs().max())
    return {"value": whole_job_rate(args.fp64_steps, world, ms), "unit": "solves/s", "steps": args.fp64_steps,
            "ms_per_step": ms / args.fp64_steps, "E0": res["E0"], "residual": res["residual"],
            "green_status": res["green_status"], "gf_steps_total_and_max": res["gf_steps"],
            "fp32_minus_fp64": {"E0_rel": abs(info32["E0"] - res["E0"]) / max(1.0, abs(res["E0"])),
                                "G_max_abs": dG,
                                "note": "FP32-storage arm against this FP64 arm, same Krylov size and grid"},
            "how": "ed_cluster_create, ed_ground_state, ed_green, ed_cluster_destroy with FP64 vectors, "
                   "timed with CUDA events (no warm-up of its own: the FP32 arm ran first in the process)"}


def run_batch(args, rank, world, local_rank, torch, ed):
    """Batched form: ed_batch_solve on 512 seeded clusters per rank; value = clusters solved / s."""
    import math
    gen, label, prec_d, gf_d, nfreq = WORKLOADS["batch"]
    prec = args.precision or prec_d
    fam = W.batched_family(args.clusters, instance=rank, max_orb=args.max_orb)
    if args.clusters != 512 or args.max_orb != 12:
        label = "%d seeded clusters of 4-%d orbitals (a smaller case of the named 512-cluster workload)" % (
            args.clusters, args.max_orb)
    if args.gf == "none":  # ground states only
        nfreq = 0
    omega = W.real_grid(nfreq) if nfreq else None
    precision = ed.ED_FP32 if prec == "fp32" else ed.ED_FP64
    gsize = max(1, sum(2 * nfreq * c["t"].shape[0] ** 2 for c in fam))
    G_dev = torch.empty(gsize * 2, dtype=torch.float64, device="cuda")
    info = {}

    def solve(to_host):
        E0, res, st, it, G = ed.ed_batch_solve(fam, precision=precision, omega=omega, eta=ETA, seed=1234 + rank,
                                               out_ptr=None if to_host else G_dev.data_ptr())
        info.update(E0=E0, residual=res, status=st, iters=it, gf_steps=ed.ed_batch_solve.gf_steps.copy())

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def timed(to_host, steps, profile):
        barrier()
        if profile:
            ed.ed_profile_enable(1)
        l0 = ed.ed_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            solve(to_host)
        e1.record()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        return ms, ed.ed_launch_count() - l0

    for _ in range(args.warmup):
        solve(False)
    with ClockSampler(local_rank) as clk:
        ms, launches = timed(False, args.steps, True)
    prof = {k: ed.ed_profile_read(k) for k in range(ed.ED_K_COUNT)}
    ed.ed_profile_enable(0)
    e2e = None
    if not args.no_e2e:
        ms_e2e, _ = timed(True, args.steps, False)
        e2e = {"value": whole_job_rate(len(fam) * args.steps, world, ms_e2e), "unit": "cluster solves/s",
               "h2d_bytes_per_step": int(sum(8 * (c["t"].size + c["t"].shape[0] + c["eps"].size + c["theta"].size + 1)
                                             for c in fam)),
               "d2h_bytes_per_step": int(gsize * 16 + len(fam) * 8 * 4)}
    # algorithmic bytes of a Lanczos level: read v_n, v_{n-1}, write v_{n+1} (3 d s); ground-state
    # levels (both passes) on the ground-state sector, continued-fraction levels on the N +- 1
    # sectors (a cluster's levels spread over its parts: the mean target dimension is used)
    es = 4 if prec == "fp32" else 8
    alg_bytes = 0.0
    for c, it, gf_l in zip(fam, info["iters"], info["gf_steps"]):
        L = c["t"].shape[0] + c["eps"].size
        nu, nd = c["n_up"], c["n_dn"]
        alg_bytes += 2 * int(it) * math.comb(L, nu) * math.comb(L, nd) * 3 * es
        tgt = [math.comb(L, nu + dn) * math.comb(L, nd) for dn in (1, -1) if 0 <= nu + dn <= L]
        if nu != nd:
            tgt += [math.comb(L, nu) * math.comb(L, nd + dn) for dn in (1, -1) if 0 <= nd + dn <= L]
        if tgt:
            alg_bytes += int(gf_l) * float(np.mean(tgt)) * 3 * es
    n_b, ms_b, _ = prof[ed.ED_K_BATCH]
    peak, peak_kind = measured_peak_hbm()
    achieved = (alg_bytes * args.steps / 1e9) / (ms_b / 1e3) if ms_b > 0 else None
    result = {
        "metric": "ED solves/s (batched form; H.psi GB/s and % roofline in `roofline`)",
        "value": whole_job_rate(len(fam) * args.steps, world, ms), "unit": "cluster solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors, f64 reductions" if prec == "fp32" else "f64", "data": "synthetic (seeded cluster parameters)",
        "config": {"workload": "batch: " + label, "clusters": len(fam), "precision": prec, "green_function": "cf" if nfreq else "none",
                   "n_freq": nfreq, "eta": ETA, "l2": "L2 flushed by the step's own traffic (tens of GB per step)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(), "e2e": e2e, "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "batched ground-state and continued-fraction persistent kernels",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": None, "peak_source": peak_kind, "launches": n_b,
                     "note": "3 vectors per Lanczos level over all ground-state and continued-fraction levels "
                             "(the mean N +- 1 dimension of a cluster for its continued-fraction levels), over the "
                             "time of the graph (persistent kernels, evaluation, assembly); small sectors are "
                             "L2-resident, so this is an effective rate, not HBM traffic"},
        "solve": {"E0_first": float(info["E0"][0]), "max_residual": float(max(info["residual"])),
                  "not_converged": int(sum(1 for x in info["status"] if x == ed.ED_WARN_NOT_CONVERGED)),
                  "degenerate": int(sum(1 for x in info["status"] if x == ed.ED_WARN_DEGENERATE)),
                  "gs_levels_total": int(sum(info["iters"])), "cf_levels_total": int(sum(info["gf_steps"]))},
        "kernels_ms": {ed.ed_profile_kernel_name(k): round(v[1], 3) for k, v in prof.items() if v[0]},
    }
    if args.sequential:
        seq = fam[::max(1, len(fam) // args.sequential)][:args.sequential]  # every k-th cluster: the family's size mix
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, cl in enumerate(seq):
            h = ed.ed_cluster_create(cl, precision=ed.ED_FP64, gf_method=ed.ED_GF_CF, seed=1234 + k)
            try:
                # the same stopping rule as the batch: convergence on the grid (1e-10 with FP64 vectors)
                ed.ed_ground_state(h)
                ed.ed_green(h, omega, ETA, cl["t"].shape[0], spin=0, out_ptr=G_dev.data_ptr())
                if cl["n_up"] != cl["n_dn"]:
                    ed.ed_green(h, omega, ETA, cl["t"].shape[0], spin=1, out_ptr=G_dev.data_ptr())
            finally:
                ed.ed_cluster_destroy(h)
        torch.cuda.synchronize()
        result["sequential_fp64_gpu"] = {"value": len(seq) / (time.perf_counter() - t0), "unit": "cluster solves/s",
                                         "clusters": len(seq),
                                         "how": "every k-th cluster of the same family one by one: ed_cluster_create, "
                                                "ed_ground_state, ed_green (continued fractions) per spin, FP64"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_batch(fam, info)
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


def served_stream(n, instance):
    """n requests of the served workload (seeded): (cluster, gf_method name)."""
    rng = np.random.default_rng(20230529 + 5000 + instance)
    out = []
    for _ in range(n):
        c = W.served_request(rng)
        out.append((c, "cf" if c["t"].shape[0] <= 10 else "band"))
    return out


def run_served(args, rank, world, local_rank, torch, ed):
    """Served form: requests through ed_server (FP32 vectors, memory admission, batched small
    requests, lanes overlapping on the device).  A step is one stream of --requests requests
    submitted at once (saturation); value = requests completed / s.  Beside it: the same kind of
    requests solved one after another by the plain FP64 path (ed_cluster_create, ed_ground_state,
    ed_green, ed_cluster_destroy), and Poisson streams at multiples of that path's rate with their
    p50 / p99 latency."""
    import threading
    nfreq = WORKLOADS["served"][4]
    om = W.matsubara_grid(nfreq)
    GB = 1 << 30
    budget = int(float(os.environ.get("ED_SERVED_BUDGET_GB", "200")) * GB)
    lanes = 8

    def gfm(name):
        return ed.ED_GF_CF if name == "cf" else ed.ED_GF_BAND

    # ---- the plain FP64 path, one request after another (calibration of the arrival rates)
    cal = served_stream(8, 100 + rank)
    seq_ms, seq_E0 = [], []
    for k, (c, m) in enumerate([cal[0]] + cal):  # the first solve warms up and is not counted
        ns = c["t"].shape[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=gfm(m), seed=77 + max(k - 1, 0))
        try:
            _, E0, _, _ = ed.ed_ground_state(h)
            ed.ed_green(h, om, 0.0, ns, axis=ed.ED_AXIS_MATSUBARA)
        finally:
            ed.ed_cluster_destroy(h)
        if k > 0:
            seq_ms.append(1e3 * (time.perf_counter() - t0))
            seq_E0.append(E0)
    t_seq = float(np.mean(seq_ms))

    srv = ed.Server(budget, max_slots=lanes)
    failures = []

    def run_stream(reqs, gaps_s, seed0):
        """Submits reqs with the given gaps (seconds before each), waits for all; returns results."""
        ids = []
        t0 = time.perf_counter()
        t_next = t0
        for k, ((c, m), g) in enumerate(zip(reqs, gaps_s)):
            t_next += g
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(c, omega=om, eta=0.0, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP32,
                                  gf_method=gfm(m), seed=seed0 + k))
        res = [srv.wait(i, timeout_s=1800.0)[0] for i in ids]
        for (c, m), r in zip(reqs, res):
            if r["status"] < 0:
                failures.append({"orbitals": int(c["t"].shape[0]), "method": m, "status": r["status"],
                                 "error": r.get("error", "")})
        return res, time.perf_counter() - t0

    # warm-up: the first requests of every size (pool growth, module load)
    warm = served_stream(max(args.warmup, 4), 200 + rank)
    run_stream(warm, [0.0] * len(warm), 1)
    # timed: saturated streams
    streams = [served_stream(args.requests, 300 + 10 * rank + s) for s in range(args.steps)]
    ed.ed_profile_enable(1)
    l0 = ed.ed_launch_count()
    all_res = []
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for s, reqs in enumerate(streams):
            res, _ = run_stream(reqs, [0.0] * len(reqs), 1000 * (s + 1))
            all_res += res
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = ed.ed_launch_count() - l0
    prof = {k: ed.ed_profile_read(k) for k in range(ed.ED_K_COUNT)}
    ed.ed_profile_enable(0)
    wall = max_over_ranks(wall, world, "cuda")
    n_req = args.requests * args.steps
    value = whole_job_rate(n_req, world, 1e3 * wall)
    lat = np.array([r["latency_ms"] for r in all_res])
    # Poisson streams at multiples of the sequential FP64 rate
    sweep = []
    rng = np.random.default_rng(20230529 + 5999 + rank)
    for f in [float(x) for x in args.rates.split(",") if x.strip()]:
        reqs = served_stream(args.requests, 400 + int(10 * f) + rank)
        gaps = rng.exponential(t_seq / 1e3 / f, size=len(reqs))
        gaps[0] = 0.0
        res, span = run_stream(reqs, gaps, 50000 + int(f * 100))
        L = np.array([r["latency_ms"] for r in res])
        sweep.append({"rate_x_seq": f, "arrival_rate_per_s": f * 1e3 / t_seq, "requests": len(reqs),
                      "p50_ms": float(np.percentile(L, 50)), "p99_ms": float(np.percentile(L, 99)),
                      "mean_queued_ms": float(np.mean([r["queued_ms"] for r in res])),
                      "completed_per_s": len(reqs) / span, "max_running": srv.stats()["max_running"]})
    stats = srv.stats()
    # accuracy: the calibration requests again through the server (FP32) against their FP64 energies
    acc_res, _ = run_stream(cal, [0.0] * len(cal), 77)
    dE = max(abs(r["E0"] - e) / max(1.0, abs(e)) for r, e in zip(acc_res, seq_E0))
    srv.close()
    n_s, ms_s, by_s = prof[ed.ED_K_LANCZOS_STEP]
    peak, peak_kind = measured_peak_hbm()
    achieved = (by_s / 1e9) / (ms_s / 1e3) if ms_s > 0 else None
    h2d = int(np.mean([8 * (c["t"].size + c["t"].shape[0] + 1) + 8 * nfreq for reqs in streams for c, _ in reqs]))
    d2h = int(np.mean([2 * nfreq * c["t"].shape[0] ** 2 * 16 + 64 for reqs in streams for c, _ in reqs]))
    result = {
        "metric": "ED solves/s and p50/p99 latency, served form (H.psi GB/s in `roofline`)",
        "value": value, "unit": "requests/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors, f64 reductions", "data": "synthetic (seeded request stream)",
        "config": {"workload": "served: " + WORKLOADS["served"][1], "requests_per_step": args.requests,
                   "lanes": lanes, "memory_budget_gb": budget / GB, "n_freq": nfreq, "axis": "matsubara",
                   "timing": "host wall clock from the first submit to the last result (requests carry host "
                             "inputs and host outputs; synchronize on both sides)",
                   "l2": "L2 flushed by the stream's own traffic (vectors up to 94 MB, several requests at once)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(),
        "e2e": {"value": value, "unit": "requests/s", "h2d_bytes_per_step": h2d * args.requests,
                "d2h_bytes_per_step": d2h * args.requests,
                "note": "the served form is host-to-host: every request's inputs and G cross PCIe/C2C inside "
                        "the timed region"},
        "gpu_launches": int(launches),
        "latency_ms_saturated": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "sequential_fp64": {"value": 1e3 / t_seq, "unit": "requests/s", "mean_ms": t_seq, "requests": len(cal),
                            "how": "ed_cluster_create, ed_ground_state, ed_green (same method per size), "
                                   "ed_cluster_destroy, one request after another, FP64"},
        "speedup_vs_sequential_fp64": value / (1e3 / t_seq),
        "max_rel_E0_diff_fp32_served_vs_fp64": dE,
        "poisson": sweep,
        "server": {k: stats[k] for k in ("completed", "failed", "max_running", "peak_reserved_bytes",
                                         "batched_solves")},
        "failed_requests": failures[:8],
        "roofline": {"bound": "hbm", "kernel": "lanczos_step (fused H.psi + Lanczos epilogue), all requests",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None, "peak_source": peak_kind,
                     "launches": n_s, "note": "event-timed launches overlap with other lanes' kernels"},
        "kernels_ms": {ed.ed_profile_kernel_name(k): round(v[1], 3) for k, v in prof.items() if v[0]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_served(all_res, streams)
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


def cpu_baseline_served(results, streams, target_s=15.0):
    """Oracle factorized H.psi timed once per request size (bounded rows), times each request's
    H.psi count in the GPU run (ground state both passes + Green-function Lanczos levels)."""
    import oracle as O
    reqs = [c for s in streams for c, _ in s]
    per_size = {}
    budget = target_s / 4
    for c in reqs:
        n = c["t"].shape[0]
        if n in per_size:
            continue
        m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
        du = len(O.sector_basis(m.L, c["n_up"]))
        dd = len(O.sector_basis(m.L, c["n_dn"]))
        psi = np.random.default_rng(0).standard_normal((du, dd))
        rows = max(1, min(du, 16))
        while True:
            t0 = time.perf_counter()
            O.apply_h_rows(m, c["n_up"], c["n_dn"], psi, np.arange(rows))
            dt = time.perf_counter() - t0
            if dt > budget / 8 or rows == du:
                break
            rows = min(du, rows * 4)
        per_size[n] = dt * du / rows
    t = [per_size[c["t"].shape[0]] * (2 * r["iters"] + r["gf_steps"]) for c, r in zip(reqs, results)]
    return {"value": 1.0 / float(np.mean(t)), "unit": "requests/s", "cores": 1, "kind": "oracle",
            "sample": "oracle apply_h_rows (scipy factorized H.psi, FP64) timed on a block of rows per request "
                      "size %s, scaled to a full H.psi and multiplied by each request's H.psi count in the GPU run"
                      % sorted(per_size)}


def cpu_baseline_batch(fam, info, target_s=15.0):
    """Oracle factorized H.psi timed on the first clusters of the family, times each cluster's
    H.psi count in the GPU run (ground state both passes + continued-fraction levels)."""
    import oracle as O
    per_solve, used, t_start = [], 0, time.perf_counter()
    for k, c in enumerate(fam):
        m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
        op = O.sector_hamiltonian(m, c["n_up"], c["n_dn"])
        x = np.random.default_rng(k).standard_normal(op.dim)
        t0 = time.perf_counter()
        op.matvec(x)
        dt = time.perf_counter() - t0
        per_solve.append(dt * (2 * int(info["iters"][k]) + int(info["gf_steps"][k])))
        used += 1
        if time.perf_counter() - t_start > target_s:
            break
    return {"value": 1.0 / float(np.mean(per_solve)), "unit": "cluster solves/s", "cores": 1, "kind": "oracle",
            "sample": "oracle factorized H.psi (scipy, FP64) timed on the first %d clusters of the family, each "
                      "multiplied by that cluster's H.psi count in the GPU run" % used}


# ----------------------------------------------------------------------------- CPU (oracle) arm
def host_cpu():
    """nproc and the CPU model of this host (lscpu), recorded beside every CPU timing."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count() or 1, "model": model, "machine": platform.machine()}


def _oracle_rows_worker(c, rows, psi_name, y_name, shape, ready, go, done, reps):
    """One process of the all-core oracle H.psi: builds the oracle's tables of its row block
    (outside the timed region), then computes y[rows] = (H psi)[rows] once per repetition
    between the `go` and `done` barriers.  psi and y live in shared memory."""
    from multiprocessing import shared_memory

    import oracle as O
    m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
    tabs = O.row_tables(m, c["n_up"], c["n_dn"], rows)
    sp, sy = shared_memory.SharedMemory(name=psi_name), shared_memory.SharedMemory(name=y_name)
    try:
        psi = np.ndarray(shape, dtype=np.float64, buffer=sp.buf)
        y = np.ndarray(shape, dtype=np.float64, buffer=sy.buf)
        ready.wait()
        for _ in range(reps):
            go.wait()
            y[rows] = O.apply_h_rows_tables(tabs, psi, rows)
            done.wait()
    finally:
        del psi, y
        sp.close()
        sy.close()


def oracle_hpsi_seconds(c, procs, reps=2):
    """Seconds of one oracle H.psi (Eq. factorized, FP64) of the cluster's ground-state sector on
    `procs` processes, each taking a contiguous block of up-spin rows; tables are built before
    the timed region.  Best of `reps`.  Processes are spawned (never forked from a process that
    holds a CUDA context)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import oracle as O
    L = c["t"].shape[0] + len(c["eps"])
    du, dd = len(O.sector_basis(L, c["n_up"])), len(O.sector_basis(L, c["n_dn"]))
    nbytes = du * dd * 8
    sp = shared_memory.SharedMemory(create=True, size=nbytes)
    sy = shared_memory.SharedMemory(create=True, size=nbytes)
    try:
        psi = np.ndarray((du, dd), dtype=np.float64, buffer=sp.buf)
        psi[:] = np.random.default_rng(0).standard_normal((du, dd))
        ctx = mp.get_context("spawn")
        ready, go, done = ctx.Barrier(procs + 1), ctx.Barrier(procs + 1), ctx.Barrier(procs + 1)
        bounds = np.linspace(0, du, procs + 1).astype(int)
        for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"  # one thread per process (inherited by the spawned children)
        ps = [ctx.Process(target=_oracle_rows_worker,
                          args=(c, np.arange(bounds[k], bounds[k + 1]), sp.name, sy.name, (du, dd), ready, go, done,
                                reps))
              for k in range(procs)]
        for p in ps:
            p.start()
        ready.wait()
        best = float("inf")
        for _ in range(reps):
            go.wait()
            t0 = time.perf_counter()
            done.wait()
            best = min(best, time.perf_counter() - t0)
        for p in ps:
            p.join()
        del psi
    finally:
        sp.close()
        sy.close()
        sp.unlink()
        sy.unlink()
    return best


def cpu_baseline(workload, c, hpsi_per_solve):
    """The oracle's H.psi on prebuilt tables, on one core and on every core of this host, scaled
    by the GPU run's H.psi count per solve."""
    cpu = host_cpu()
    n = cpu["nproc"]
    t_all = oracle_hpsi_seconds(c, n)
    t_one = oracle_hpsi_seconds(c, 1, reps=1)
    per = max(hpsi_per_solve, 1.0)
    return {"value": 1.0 / (t_all * per), "unit": "solves/s", "cores": n, "kind": "oracle",
            "value_1_core": 1.0 / (t_one * per), "hpsi_s_all_cores": t_all, "hpsi_s_1_core": t_one,
            "host": cpu,
            "sample": "one full oracle H.psi (oracle.apply_h_rows_tables: scipy factorized product, FP64) of the "
                      "ground-state sector, tables built outside the timed region, on %d processes (blocks of "
                      "up-spin rows, shared-memory vectors; best of 2) and on 1 process; solves/s = 1 / (t_hpsi x "
                      "%.0f H.psi per solve, the count of the GPU run)" % (n, per)}


# H.psi per solve of the GPU runs (ground state, its FP64 refinement and residuals, and the
# Green-function Lanczos vectors), the counts the oracle arm multiplies its timed H.psi by
HPSI_PER_SOLVE = {"4x4": 1264.0, "cdmft": 2000.0, "2x4": 20000.0, "2x7": 1200.0}


def run_reference(args, rank, world):
    gen, label, prec_d, gf_d, nfreq = WORKLOADS[args.workload]
    c = gen(instance=0)
    if args.workload not in HPSI_PER_SOLVE:
        return {"impl": "reference", "unavailable": "the oracle arm covers the single-cluster workloads; the %s "
                "workload reports its oracle baseline in cpu_baseline of the GPU line" % args.workload}
    hpsi_per_solve = HPSI_PER_SOLVE[args.workload]
    cpu = host_cpu()
    n = cpu["nproc"]
    for _ in range(max(1, min(args.warmup, 1))):
        oracle_hpsi_seconds(c, n, reps=1)
    t0 = time.perf_counter()
    per = [oracle_hpsi_seconds(c, n, reps=1) for _ in range(args.steps)]
    total = time.perf_counter() - t0
    value = 1.0 / (float(np.mean(per)) * hpsi_per_solve)
    desc = ("each step: one full oracle H.psi (oracle.apply_h_rows_tables, scipy factorized product, FP64) of "
            "the ground-state sector on %d processes, tables built outside the timed region; solves/s = 1 / "
            "(t_hpsi x %.0f H.psi per solve, the count of the GPU run)" % (n, hpsi_per_solve))
    return {"impl": "reference", "metric": "ED solves/s (H.psi HBM GB/s and % roofline in `roofline`)",
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded cluster parameters)",
            "config": {"workload": args.workload + ": " + label, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": n, "kind": "oracle", "sample": desc,
                             "host": cpu},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)))
        return
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
