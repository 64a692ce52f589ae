#!/usr/bin/env python
"""Benchmark: molecular-dynamics force evaluations per second on a 32^3 x 64
lattice (two-flavour Wilson fermions, even-odd pseudofermion action, beta 5.8,
kappa 0.156, seeded links exp(i 0.5 H)), mixed-precision path vs FP64 path,
Wilson-hop HBM bandwidth, end-to-end rate with host buffers, and the FP64 CPU
oracle as the baseline.

One step = one MD update: a force evaluation from scratch (CG on Dhat^+ Dhat from a
zero guess to tol 1e-10, X/Y vectors, fermion and gauge force fused into the
momentum kick) followed by the link update U <- exp(i eps P) U.  The mixed path
runs the CG in FP32 with FP64 reliable updates and the forces in double-float
(FP32-pair) arithmetic accumulated in FP64; the FP64 path is FP64 throughout.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --kernel hop32|hop64|force_df|clover_md [--reps R]   # a few launches, for ncu

Prints one JSON line (rank 0).  With torchrun each rank runs an independent
replica (no collective in the data path; weak scaling).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "force evals/s + Dslash HBM GB/s at 32^3×64, mixed vs FP64; p99 solve latency"
UNIT = "force evals/s"
DIMS = (32, 32, 32, 64)
# DELTA: reliable-update threshold of the mixed CG (|r| < DELTA max|r| triggers an FP64
# residual replacement).  Measured on this workload (force from a zero guess at the
# seeded start): 146 inner iterations for every DELTA from 1e-3 to 3e-5 with 4 -> 3 FP64
# updates; 3e-6 needs 147 iterations and 2 updates (the fastest); 1e-6 needs 158
BETA, KAPPA, ALPHA, TOL, DELTA = 5.8, 0.156, 0.5, 1e-10, 3e-6
# force arithmetic of the mixed path: double-float (FP32 pairs, ~48 bits) accumulated
# in FP64; FP64 and FP32 force arithmetic are timed beside it
FORCE_ARITH = "df64"
EPS = 1.0 / 20
SEED = 4
# FP64 CG iterations of this workload (Dhat^+Dhat, tol 1e-10, zero guess): used only to
# scale the oracle's capped-CG sample in the reference arm (the default arm uses the
# count it measures in the same run)
CG_ITERS_FP64 = 146
# algorithmic (compulsory) bytes per output site of one even-odd hop:
# 8 links + 1 input spinor + 1 output spinor (each array touched once)
HOP_BYTES = {"fp32": 8 * 48 + 96 + 96, "fp64": 8 * 144 + 192 + 192}
# per epilogue: + y read (xpay); the fused CG residual update reads y and r and writes
# r instead of writing the output (x += alpha p is left to the p update)
HOP_BYTES_EPI = {prec: {"hop": b, "xpay": b + s, "xpay_norm": b + s, "cg_update": b - s + s + 2 * s,
                        "residual": b + 2 * s}
                 for prec, b, s in (("fp32", HOP_BYTES["fp32"], 96), ("fp64", HOP_BYTES["fp64"], 192))}
HOP_FLOPS = 1320
# launches shorter than this did no work (a full hop at 32^3 x 64 takes >= 70 us)
HOP_MIN_MS = 0.010
# ncu DRAM traffic (read + write) of one FP32 hop launch at 32^3 x 64, and the hash of
# the kernel sources it was taken from (traffic is reported as null once they change)
NCU_TRAFFIC = {"bytes": 593337600,
               "sources_sha256": "538073696f8c5ae43bd6ab2f31e5d6a4b04b56151b93b477a7430ed15ff8e2de"}
HOP_SOURCES = ["paper_2602_20516_b300/csrc/lgt_dirac.cu", "paper_2602_20516_b300/csrc/lgt_spin.cuh",
               "paper_2602_20516_b300/csrc/lgt_common.cuh"]


def hop_sources_hash():
    h = hashlib.sha256()
    for f in HOP_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "of measured"
    return 6400.0, "of fallback"


def config_block(args):
    return {"workload": "32^3x64 Nf=2 Wilson even-odd MD step: mixed CG (FP32 inner, FP64 reliable "
                        "updates) tol 1e-10 from zero guess + fermion/gauge force (double-float arithmetic, "
                        "FP64 accumulation) into the momentum kick + FP64 link update",
            "lattice": list(DIMS), "beta": BETA, "kappa": KAPPA, "alpha": ALPHA, "tol": TOL,
            "delta": DELTA, "seed": SEED, "eps": EPS,
            "l2": "inputs larger than L2 (FP64 links 1.21 GB + FP32 links 0.40 GB per replica)",
            "parallelism": f"replicas x{args.gpus}"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample(cg_iters, reps=1):
    """Time the FP64 oracle on a bounded sample of one MD step at 32^3 x 64 and
    scale it to one force evaluation: CG capped at 2 iterations (3 operator
    applications with its residual check; per-iteration cost = t/3), the X/Y hops,
    gauge force, fermion force and link update."""
    import numpy as np
    import oracle as O
    d = DIMS
    U = O.random_links(d, SEED, ALPHA)
    phi = O.gaussian_spinor(d, SEED, 0, O.FIELD_SOURCE, 1)
    mom = O.gaussian_momenta(d, SEED, 0)
    est = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.cg(d, U, KAPPA, phi, eo=True, tol=TOL, max_iter=2)
        t_cg = time.perf_counter() - t0
        t1 = time.perf_counter()
        X = O.hop(d, U, phi, out_mask=2)
        Y = O.hop(d, U, X, out_mask=1)
        O.hop(d, U, Y, out_mask=2, dagger=True)
        O.gauge_force(d, U, BETA)
        O.fermion_force_xy(d, U, KAPPA, X, Y)
        O.update_links(d, U, mom, EPS)
        t_rest = time.perf_counter() - t1
        est.append(t_cg / 3.0 * (cg_iters + 1) + t_rest)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle (C, OpenMP) on 32^3x64: CG capped at 2 iterations scaled to {cg_iters} "
              f"iterations (+1 residual apply), plus X/Y hops, gauge force, fermion force, link update")
    return est, cores, sample


# ---------------------------------------------------------------- ranks
# One process per GPU (replicas: every rank runs the whole step on its own lattice,
# with no collective on the data path).  The timing is the slowest rank's, and the
# whole-job throughput counts the units of all ranks.
def max_over_ranks(v, world, device="cuda"):
    """The maximum of v over the ranks (v itself for one rank)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(world, units_per_rank, seconds_max):
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2602_20516_b300 import lgt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_ranks(v):
        return max_over_ranks(v, world)

    lat = lgt.Lattice(DIMS)
    lat.random_links(SEED + rank, ALPHA)
    phi = lat.gaussian_spinor(SEED + rank, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    mom = lat.gaussian_momenta(SEED + rank, 0)
    # every phase (mixed, FP64, FP32 forces, e2e) starts from this same state, so
    # they run the same MD steps on the same fields
    U_start = lat.get_links()
    mom_start = mom.clone()

    def restore():
        lat.set_links(U_start)
        mom.copy_(mom_start)
    # headline mixed path: FP32 CG with FP64 reliable updates, forces in double-float
    # (FP32-pair) arithmetic accumulated in FP64; the FP64 path ignores force_arith
    ap = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=FORCE_ARITH)
    stream = torch.cuda.current_stream()

    def step(sp, stats, a=ap):
        s = lat.md_update(mom, EPS, lgt.UPDATE_P, a, phi, sp)
        lat.md_update(mom, EPS, lgt.UPDATE_U)
        stats.append(s)

    def timed(sp, K, W, kernel_timing=False, clocks=None, a=ap):
        st = []
        restore()
        for _ in range(W):
            step(sp, st, a)
        st.clear()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        lgt.launch_count(reset=True)
        if kernel_timing:
            lgt.kernel_timing_start(65536)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step(sp, st, a)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches = lgt.launch_count()
        # hops enqueued after a solve stopped return at entry (a few us): excluded
        kt = lgt.kernel_timing_stop(HOP_MIN_MS) if kernel_timing else None
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        return ms, st, launches, kt, clk

    K, W = args.steps, args.warmup
    sp_mixed = lgt.solver("mixed", tol=TOL, delta=DELTA)
    sampler = ClockSampler(local)
    ms, st, launches, kt, clk = timed(sp_mixed, K, W, kernel_timing=True, clocks=sampler)
    ms_max = max_ranks(ms)
    value = whole_job_rate(world, K, ms_max / 1e3)
    iters = statistics.mean(s["iters"] for s in st)
    rel = statistics.mean(s["reliable_updates"] for s in st)

    # FP64 path, same workload
    K64 = max(1, min(K, args.fp64_steps))
    ms64, st64, _, kt64, _ = timed(lgt.solver("fp64", tol=TOL), K64, W, kernel_timing=True)
    ms64 = max_ranks(ms64)
    value64 = world * K64 / (ms64 / 1e3)
    iters64 = statistics.mean(s["iters"] for s in st64)

    # the same workload with the other force arithmetics of the mixed path: FP64, and
    # FP32 (~1e-7 force error, moves Delta H by ~1e-4 relative)
    variants = {}
    fd = None
    for arith in ("fp64", "fp32"):
        apv = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=arith)
        msv, _, _, _, _ = timed(sp_mixed, K, W, a=apv)
        restore()
        Fv, _ = lat.force(apv, phi, sp_mixed)
        if fd is None:
            fd, _ = lat.force(ap, phi, lgt.solver("fp64", tol=TOL))
        variants[arith] = {"value": world * K / (max_ranks(msv) / 1e3), "ms_per_step": msv / K, "steps": K,
                           "force_rel_err_vs_fp64_path": (torch.linalg.norm(Fv - fd) / torch.linalg.norm(fd)).item()}
        del Fv

    # the even-odd clover action (c_sw = 1.0) against the Wilson one on the same MD steps,
    # at kappa = 0.13 (1 + A stays positive definite on this start at the couplings used)
    clover = None
    if not args.no_clover:
        kc, cswc = 0.13, 1.0
        res_c = {}
        for name, csw in (("wilson_eo", 0.0), ("clover_eo", cswc)):
            apc = lgt.action_params(beta=BETA, kappa=kc, even_odd=True, force_arith=FORCE_ARITH, csw=csw)
            msc, stc, _, _, _ = timed(sp_mixed, K, W, a=apc)
            res_c[name] = {"value": world * K / (max_ranks(msc) / 1e3), "ms_per_step": msc / K,
                           "cg_iters_per_step": statistics.mean(x["iters"] for x in stc)}
        clover = {"kappa": kc, "csw": cswc, **res_c,
                  "clover_overhead": res_c["clover_eo"]["ms_per_step"] / res_c["wilson_eo"]["ms_per_step"]}
        restore()   # the force comparison below is on the starting field

    # error of the headline mixed force against the FP64 path on the same field
    Fm, _ = lat.force(ap, phi, sp_mixed)
    force_err = (torch.linalg.norm(Fm - fd) / torch.linalg.norm(fd)).item()
    del Fm, fd

    # dominant kernel: the FP32 hop, timed with CUDA events on its stream inside the
    # timed region; each epilogue variant counts its own algorithmic bytes
    kinds, n32_short = kt
    bytes32 = sum(HOP_BYTES_EPI["fp32"][e] * lat.Vh * n for (p, e), (ms_, n) in kinds.items() if p == "fp32")
    ms32_sum = sum(ms_ for (p, e), (ms_, n) in kinds.items() if p == "fp32")
    n32 = sum(n for (p, e), (ms_, n) in kinds.items() if p == "fp32")
    hop32_ms = ms32_sum / max(n32, 1)
    achieved = bytes32 / (ms32_sum * 1e-3) / 1e9
    per_variant = {e: {"launches": n, "avg_us": 1e3 * ms_ / n,
                       "GBs": HOP_BYTES_EPI["fp32"][e] * lat.Vh / (ms_ / n * 1e-3) / 1e9}
                   for (p, e), (ms_, n) in kinds.items() if p == "fp32"}
    kinds64, _ = kt64
    plain64 = kinds64.get(("fp64", "hop"), (0.0, 0))
    hop64_ms = plain64[0] / max(plain64[1], 1)
    fp64_peak = lgt.measure_fp64_peak()
    peak, peak_kind = measured_peaks()
    traffic = NCU_TRAFFIC["bytes"] if NCU_TRAFFIC["sources_sha256"] == hop_sources_hash() else None

    # end to end through the public API with host buffers: every step uploads the
    # canonical links and phi from pinned host memory and downloads the canonical
    # force; the upload of step k+1 and the download of step k run on a copy stream
    # while step k / k+1 compute (two device staging slots)
    e2e = None
    if not args.no_e2e:
        Ke = max(2, min(K, args.e2e_steps))
        # the gauge configurations of the headline's first timed MD steps (an untimed
        # replay of the same sequence), so that every end-to-end force evaluation is
        # one the headline also timed; at most 4 kept in pinned host memory, cycled
        n_cfg = min(Ke, 4)
        Uhs = []
        restore()
        st_replay = []
        for _ in range(W):
            step(sp_mixed, st_replay)
        for _ in range(n_cfg):
            Uhs.append(lat.get_links().cpu().pin_memory())
            step(sp_mixed, st_replay)
        Uh = Uhs[0]
        phic = lat.unpack_spinor(phi, lgt.EVEN, lgt.FP64).cpu().pin_memory()
        Fh = [torch.empty((lat.V, 4, 8), dtype=torch.float64).pin_memory() for _ in range(2)]
        Ud = [torch.empty_like(Uh, device="cuda") for _ in range(2)]
        phid = [torch.empty_like(phic, device="cuda") for _ in range(2)]
        Fd = [torch.empty((lat.V, 4, 8), dtype=torch.float64, device="cuda") for _ in range(2)]
        # uploads and downloads on streams of their own (the two copy engines run both
        # directions at once, and an upload never queues behind a download)
        copy = torch.cuda.Stream()
        copy_out = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        e2e_iters = []

        def upload(k):
            q = k % 2
            with torch.cuda.stream(copy):
                copy.wait_event(ev_free[q])
                Ud[q].copy_(Uhs[k % n_cfg], non_blocking=True)
                phid[q].copy_(phic, non_blocking=True)
                ev_in[q].record(copy)

        def compute(k):
            q = k % 2
            stream.wait_event(ev_in[q])
            lat.set_links(Ud[q])
            pf = lat.pack_spinor(phid[q], lgt.EVEN, lgt.FP64)
            ev_free[q].record(stream)
            F, fs = lat.force(ap, pf, sp_mixed)
            e2e_iters.append(fs["iters"])
            Fd[q].copy_(lat.unpack_momenta(F))
            ev_out[q].record(stream)

        def download(k):
            q = k % 2
            with torch.cuda.stream(copy_out):
                copy_out.wait_event(ev_out[q])
                Fh[q].copy_(Fd[q], non_blocking=True)

        def pipeline(n):
            upload(0)
            for k in range(n):
                if k + 1 < n:
                    upload(k + 1)
                compute(k)
                download(k)
            torch.cuda.synchronize()

        pipeline(2)
        barrier()
        e2e_iters.clear()
        t0 = time.perf_counter()
        pipeline(Ke)
        barrier()
        te = max_ranks(time.perf_counter() - t0)

        # the host link alone: one upload and one download of a step's bytes
        def copy_time(fn):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) * 1e-3
        h2d_b, d2h_b = Uh.numel() * 16 + phic.numel() * 16, Fh[0].numel() * 8
        t_up = copy_time(lambda: (Ud[0].copy_(Uh, non_blocking=True), phid[0].copy_(phic, non_blocking=True)))
        t_down = copy_time(lambda: Fh[0].copy_(Fd[0], non_blocking=True))
        e2e = {"value": world * Ke / te, "unit": UNIT,
               "h2d_bytes_per_step": h2d_b,
               "d2h_bytes_per_step": d2h_b,
               "h2d_GBs": h2d_b / t_up / 1e9, "d2h_GBs": d2h_b / t_down / 1e9,
               "cg_iters_per_step": statistics.mean(e2e_iters),
               "steps": Ke, "step": "upload canonical links (the configurations of the headline's first "
                                   "timed MD steps) + phi from pinned host memory, force (mixed CG), "
                                   "download canonical force; uploads and downloads overlap the "
                                   "neighbouring steps' compute on copy streams"}
        del Uhs, Uh

    multi = run_multi_rhs(lat, stream) if not args.no_multi else None

    serving = None
    if args.serve_requests > 0:
        free, total = torch.cuda.mem_get_info()
        serving = {"full": run_serving(args.serve_requests, int(0.8 * free)),
                   "tight_8GB": run_serving(args.serve_requests, 8 << 30) if args.serve_tight else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        est, cores, sample = oracle_sample(int(round(iters64)), reps=1)
        cpu = {"value": 1.0 / statistics.mean(est), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 CG + f64 reliable updates + df64 forces (mixed)", "data": "synthetic: seeded links exp(i 0.5 H), Gaussian pseudofermion",
           "config": config_block(args),
           "cg_iters_per_step": iters, "reliable_updates_per_step": rel,
           "fp64": {"value": value64, "ms_per_step": ms64 / K64, "steps": K64, "cg_iters_per_step": iters64,
                    "mixed_speedup": value / value64,
                    "mixed_force_rel_err_vs_fp64_path": force_err},
           "force_arith": FORCE_ARITH, "force_arith_variants": variants,
           "dslash": {"fp32_hop_avg_us": hop32_ms * 1e3, "fp32_hop_GBs_algorithmic": achieved,
                      "fp32_variants": per_variant,
                      "fp32_hop_launches": n32, "skipped_hop_launches": n32_short,
                      "fp64_plain_hop_us": hop64_ms * 1e3,
                      "fp64_hop_TFLOPs": HOP_FLOPS * lat.Vh / (hop64_ms * 1e-3) / 1e12,
                      "fp64_peak_TFLOPs_measured": fp64_peak / 1e12,
                      "fp64_hop_frac_of_fp64_peak": HOP_FLOPS * lat.Vh / (hop64_ms * 1e-3) / fp64_peak},
           "roofline": {"bound": "hbm", "kernel": "hop_kernel<float> (FP32 Wilson hop, two-row links)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": peak_kind,
                        "traffic": traffic, "traffic_kernel": "plain FP32 hop (ncu capture)",
                        "algorithmic_bytes_per_launch": bytes32 / max(n32, 1),
                        "algorithmic_bytes_plain_hop": HOP_BYTES["fp32"] * lat.Vh},
           "clover": clover,
           "multi_rhs": multi,
           "serving": serving,
           "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- several right-hand sides
def run_multi_rhs(lat, stream, reps=50):
    """FP32 hop on K = 1..4 sources with one load of each link (lgt_hop_multi), and
    four mixed-precision solves at once (lgt_cg_solve_multi) against one at a time;
    algorithmic bytes per site of a K-source hop: 8 x 48 + K x (96 + 96)."""
    import torch
    from paper_2602_20516_b300 import lgt
    ins = [lat.pack_spinor(lat.unpack_spinor(lat.gaussian_spinor(SEED + 100 + k, 0, lgt.FIELD_SOURCE, lgt.ODD),
                                             lgt.ODD, lgt.FP64), lgt.ODD, lgt.FP32) for k in range(4)]
    hop = {}
    for K in (1, 2, 3, 4):
        outs = [lat.spinor_field(lgt.EVEN, lgt.FP32) for _ in range(K)]
        for _ in range(3):
            lat.hop_multi(ins[:K], lgt.EVEN, False, outs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lat.hop_multi(ins[:K], lgt.EVEN, False, outs)
        e1.record(stream)
        torch.cuda.synchronize()
        us = 1e3 * e0.elapsed_time(e1) / reps
        hop[K] = {"us": us, "us_per_source": us / K,
                  "GBs_algorithmic": (8 * 48 + K * 192) * lat.Vh / (us * 1e-6) / 1e9}
    del ins, outs
    phis = [lat.gaussian_spinor(SEED + 200 + k, 0, lgt.FIELD_SOURCE, lgt.EVEN) for k in range(4)]
    kap = [0.150, 0.152, 0.154, 0.156]
    sp = lgt.solver("mixed", tol=TOL, delta=DELTA)
    lat.cg_solve_multi(phis, kap, sp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, sts = lat.cg_solve_multi(phis, kap, sp)
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    t_single = 0.0
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.cg_solve(phis[k], kap[k], True, sp)
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t0
    return {"hop_fp32": hop, "solve4": {"kappa": kap, "seconds_together": t_multi, "seconds_one_by_one": t_single,
                                        "iters": [s["iters"] for s in sts], "speedup": t_single / t_multi}}


# ---------------------------------------------------------------- serving (p50/p99 latency)
SERVE_VOLUMES = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 48)]


def run_serving(n_per_rate, budget_bytes, seed=10):
    """Resident pool of 2 gauge fields per volume (alpha ~ U[0.3, 0.6]); requests:
    70% Dirac solves, 30% force evaluations, kappa ~ U[0.14, 0.157], FP64 / mixed
    50/50, tol 1e-10.  Saturated throughput, then open-loop Poisson arrivals at
    0.5, 0.9 and 1.2 x that rate; latency = completion - scheduled arrival."""
    import numpy as np
    from paper_2602_20516_b300 import serve
    rng = np.random.default_rng(seed)
    srv = serve.Server(budget_bytes, max_active=64, batch_iters=8, delta=DELTA)
    gids = []
    for k, d in enumerate(SERVE_VOLUMES):
        for j in range(2):
            gids.append(srv.add_gauge(d, 1000 + 10 * k + j, float(rng.uniform(0.3, 0.6))))
    warm = max(10, n_per_rate // 10)
    serve.saturated(srv, serve.workload(gids, warm, seed=seed))          # warm-up
    thr, done = serve.saturated(srv, serve.workload(gids, n_per_rate, seed=seed + 1))
    out = {"saturated_requests_per_s": thr, "budget_bytes": budget_bytes,
           "requests_per_rate": n_per_rate, "warmup_per_rate": warm, "rates": {}}
    for j, f in enumerate((0.5, 0.9, 1.2)):
        reqs = serve.workload(gids, n_per_rate + warm, seed=seed + 2 + j)
        d = serve.poisson(srv, reqs, f * thr, seed=seed + 20 + j, warmup=warm)
        st = serve.latency_stats(d)
        solves = [c for c in d if c["status"] == 0]
        st["offered_per_s"] = f * thr
        st["completed"] = len(solves)
        out["rates"][f"{f}x"] = st
    srv.close()
    return out


# ---------------------------------------------------------------- HMC on the 32^3 x 64 lattice
def run_hmc(args):
    """Full Nf=2 HMC at 32^3 x 64 (beta 5.8, kappa 0.156, even-odd S_f, Omelyan 2MN,
    20 steps, tau = 1) from the seeded alpha = 0.5 start, mixed-precision solver
    (tol 1e-10 in MD and action).  The first --hmc-fp64 trajectories are replayed on
    the FP64 path from the same starting field and seeds: Delta H is compared
    trajectory by trajectory (free-running chains diverge by MD chaos)."""
    import torch
    from paper_2602_20516_b300 import lgt
    torch.cuda.set_device(0)
    ap = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=FORCE_ARITH)
    mixed = lgt.solver("mixed", tol=TOL, delta=DELTA, chrono=args.chrono)
    fp64 = lgt.solver("fp64", tol=TOL, chrono=args.chrono)
    hp_m = lgt.hmc_params("omelyan", 20, 1.0, mixed, lgt.solver("mixed", tol=TOL, delta=DELTA))
    hp_d = lgt.hmc_params("omelyan", 20, 1.0, fp64, lgt.solver("fp64", tol=TOL))
    lat = lgt.Lattice(DIMS)
    lat.random_links(SEED, ALPHA)
    ref = lgt.Lattice(DIMS) if args.hmc_fp64 > 0 else None
    trajs = []
    for k in range(args.hmc):
        U0 = lat.get_links() if k < args.hmc_fp64 else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = lat.hmc_trajectory(ap, hp_m, SEED, k)
        torch.cuda.synchronize()
        rec = {"traj": k, "dH": r["dH"], "accepted": r["accepted"], "plaquette": r["plaquette"],
               "seconds": time.perf_counter() - t0, "force_evals": r["force_evals"],
               "cg_iters": r["total"]["iters"], "reliable_updates": r["total"]["reliable_updates"]}
        if U0 is not None:
            ref.set_links(U0)
            t1 = time.perf_counter()
            rd = ref.hmc_trajectory(ap, hp_d, SEED, k)
            rec.update({"dH_fp64": rd["dH"], "accepted_fp64": rd["accepted"],
                        "dH_abs_diff": abs(rd["dH"] - r["dH"]), "fp64_seconds": time.perf_counter() - t1})
        trajs.append(rec)
        print(json.dumps({"progress": rec}), file=sys.stderr, flush=True)
        if args.log:   # one JSON line per trajectory
            with open(args.log, "a") as f:
                f.write(json.dumps(rec) + "\n")
        if args.checkpoint:   # the chain's state after trajectory k: links, seed, k + 1
            lat.save_checkpoint(args.checkpoint, SEED, k + 1)
    acc = sum(t["accepted"] for t in trajs) / max(len(trajs), 1)
    mixed_s = statistics.mean(t["seconds"] for t in trajs)
    out = {"metric": "HMC trajectories at 32^3x64 (Omelyan 2MN, 20 steps, tau 1), mixed vs FP64",
           "trajectories": len(trajs), "acceptance": acc, "seconds_per_trajectory_mixed": mixed_s,
           "seconds_per_trajectory_fp64": statistics.mean(t["fp64_seconds"] for t in trajs if "fp64_seconds" in t)
           if args.hmc_fp64 else None,
           "config": {"lattice": list(DIMS), "beta": BETA, "kappa": KAPPA, "alpha_start": ALPHA, "seed": SEED,
                      "tol": TOL, "delta": DELTA, "integrator": "omelyan2mn", "n_steps": 20, "tau": 1.0,
                      "force_arith": FORCE_ARITH, "chrono": args.chrono},
           "per_trajectory": trajs}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    est, cores, sample = oracle_sample(CG_ITERS_FP64, reps=W + K)
    timed = est[W:]
    value = len(timed) / sum(timed)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": K, "warmup": W, "ms_per_step": 1e3 * statistics.mean(timed), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (same seeds)",
           "config": config_block(args),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- single-kernel mode (ncu)
def run_kernel(args):
    import torch
    from paper_2602_20516_b300 import lgt
    lat = lgt.Lattice(DIMS)
    lat.random_links(SEED, ALPHA)
    if args.kernel == "force_df":
        # one mixed-precision force evaluation with double-float force arithmetic
        phi = lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.EVEN)
        ap = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith="df64")
        for _ in range(args.reps):
            lat.force(ap, phi, lgt.solver("mixed", tol=TOL, delta=DELTA))
        torch.cuda.synchronize()
        print(json.dumps({"kernel": args.kernel, "force_evals": args.reps, "lattice": list(DIMS)}))
        return
    if args.kernel == "clover_md":
        # mixed-precision MD steps with the even-odd clover action (kappa 0.13, c_sw 1.0)
        phi = lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.EVEN)
        ap = lgt.action_params(beta=BETA, kappa=0.13, even_odd=True, force_arith=FORCE_ARITH, csw=1.0)
        sp = lgt.solver("mixed", tol=TOL, delta=DELTA)
        mom = lat.momentum_field()
        for _ in range(args.reps):
            st = lat.md_update(mom, EPS, lgt.UPDATE_P, ap, phi, sp)
            lat.md_update(mom, EPS, lgt.UPDATE_U)
        torch.cuda.synchronize()
        print(json.dumps({"kernel": args.kernel, "md_steps": args.reps, "lattice": list(DIMS), "last_solve": st}))
        return
    prec = lgt.FP32 if args.kernel == "hop32" else lgt.FP64
    src = lat.pack_spinor(lat.unpack_spinor(lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.ODD),
                                            lgt.ODD, lgt.FP64), lgt.ODD, prec)
    out = lat.spinor_field(lgt.EVEN, prec)
    for _ in range(args.reps):
        lat.dslash(src, lgt.OP_HOP, lgt.EVEN, False, 0.0, prec, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"kernel": args.kernel, "launches": args.reps, "lattice": list(DIMS)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="timed steps of the FP64 path (the first ones of the same MD sequence)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-multi", action="store_true", help="skip the several-sources measurement")
    ap.add_argument("--no-clover", action="store_true", help="skip the even-odd clover measurement")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests per arrival rate in the serving measurement (0 skips it)")
    ap.add_argument("--serve-tight", action="store_true", help="also run serving under an 8 GB budget")
    ap.add_argument("--hmc", type=int, default=0, help="run this many HMC trajectories instead (own JSON line)")
    ap.add_argument("--hmc-fp64", type=int, default=2, help="trajectories replayed on the FP64 path")
    ap.add_argument("--log", default="", help="HMC mode: append one JSON line per trajectory to this file")
    ap.add_argument("--checkpoint", default="", help="HMC mode: write the chain's checkpoint here after every trajectory")
    ap.add_argument("--chrono", type=int, default=0,
                    help="HMC mode: MD solves start from the last N solutions (chronological guess)")
    ap.add_argument("--kernel", choices=["hop32", "hop64", "force_df", "clover_md"])
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    if args.impl == "ours" and not args.kernel:
        args.warmup = max(3, args.warmup)   # timing rule: at least 3 untimed steps
    if args.kernel:
        run_kernel(args)
    elif args.hmc > 0:
        run_hmc(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
