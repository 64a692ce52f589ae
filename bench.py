#!/usr/bin/env python
"""Benchmark: molecular-dynamics force evaluations per second on a 32^3 x 64
lattice (two-flavour Wilson fermions, even-odd pseudofermion action, beta 5.8,
kappa 0.156), mixed-precision path vs FP64 path, Wilson-hop HBM bandwidth,
end-to-end rate with host buffers, and the FP64 CPU oracle as the baseline.

Workload: four fixed gauge fields, the links (and momenta) at MD steps 0, 10, 20
and 30 of the seeded MD sequence from the exp(i 0.5 H) start (eps = 1/20, built
untimed before the measurement and kept on the device).  Along that sequence the
plaquette swings 0.50 -> 0.61 -> 0.47 and the field at step 20 has a nearly
singular Dhat (about 600 FP64 CG iterations against 110-190 for the others), so
the four span the cost range of the sequence.  One step = one force evaluation
on each of the four fields from a zero CG guess (CG on Dhat^+ Dhat to tol 1e-10,
X/Y vectors, fermion and gauge force fused into the momentum kick) followed by
the link update U <- exp(i eps P) U: the same work whatever --steps is.  The
mixed path runs the CG in FP32 with FP64 reliable updates and the forces in
double-float (FP32-pair) arithmetic accumulated in FP64; the FP64 path is FP64
throughout and is timed on the same four fields.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--detail PATH]
    python bench.py --kernel hop32|hop64|hopdf|force_df|clover_md [--reps R]   # a few launches, for ncu
    python bench.py --hmc N [--hmc-fp64 M] [--log PATH]                  # config-4 HMC record
    python bench.py --cpu-table1                                         # oracle force at 24^4, 1 and all threads

Prints one JSON line (rank 0); --detail also writes the per-field and per-phase
figures to a file.  With torchrun each rank runs an independent replica (no
collective in the data path; weak scaling).
"""
import argparse
import hashlib
import json
import os
import platform
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
# DELTA: reliable-update threshold of the mixed CG (|r| < DELTA max|r| triggers a
# residual replacement, formed in double-float).  Measured on the four fields of the
# workload (iterations on the fields at MD steps 0, 10, 20, 30): DELTA 1e-2 .. 1e-3 needs
# 146 / 111 / 593 / 188 iterations with 4-6 updates each, as many as FP64 CG; 3e-6 needs
# 147 / 111 / 738 / 189 with 2-3 (the nearly singular step-20 field loses 25 %), 1e-6
# 158 / 117 / 950 / 201.  The step takes 657 ms at 3e-3 against 717 ms at 3e-6.
BETA, KAPPA, ALPHA, TOL, DELTA = 5.8, 0.156, 0.5, 1e-10, 3e-3
# force arithmetic of the mixed path: double-float (FP32 pairs, ~48 bits) accumulated
# in FP64; FP64 and FP32 force arithmetic are timed beside it
FORCE_ARITH = "df64"
EPS = 1.0 / 20
SEED = 4
# the workload's gauge fields: MD steps of the seeded sequence
FIELD_STEPS = (0, 10, 20, 30)
# FP64 CG iterations (Dhat^+Dhat, tol 1e-10, zero guess) on those four fields, measured
# on a B300 with this library; the reference arm scales its capped-CG sample with them (the
# default arm uses the counts it measures in the same run, reported beside them)
CG_ITERS_FP64 = {0: 146, 10: 111, 20: 592, 30: 188}
# one oracle force evaluation run to completion (no extrapolation) beside Table I of
# the paper (24^4, Wilson fermions, no smearing; its beta, kappa and tolerance are not
# stated, so these are config 4's)
TABLE1_DIMS = (24, 24, 24, 24)
TABLE1_PAPER_S = {"single_thread_cpu_handwritten": 195.53, "single_thread_cpu_ad": 162.50,
                  "h100_handwritten": 4.61, "h100_ad": 3.39}
# algorithmic (compulsory) bytes per output site of one even-odd hop:
# 8 links + 1 input spinor + 1 output spinor (each array touched once)
HOP_BYTES = {"fp32": 8 * 48 + 96 + 96, "fp64": 8 * 144 + 192 + 192}
# per epilogue: + y read (xpay); the fused CG residual update reads y and r and writes
# r instead of writing the output (x += alpha p is left to the p update)
HOP_BYTES_EPI = {prec: {"hop": b, "xpay": b + s, "xpay_norm": b + s, "cg_update": b - s + s + 2 * s,
                        "residual": b + 2 * s}
                 for prec, b, s in (("fp32", HOP_BYTES["fp32"], 96), ("fp64", HOP_BYTES["fp64"], 192))}
HOP_FLOPS = 1320
# the roofline's CUDA-event timing records every HOP_TIMING_EVERY-th hop launch of the
# timed region
HOP_TIMING_EVERY = 7
# launches shorter than this did no work (a full hop at 32^3 x 64 takes >= 70 us)
HOP_MIN_MS = 0.010
# ncu DRAM traffic (read + write) of one FP32 hop launch at 32^3 x 64, and the hash of
# the kernel sources it was taken from (traffic is reported as null once they change)
NCU_TRAFFIC = {"bytes": 593230848,
               "sources_sha256": "fef8c0ff4d06cd6e8ba8b3265932a3209456a5e487b9973d20f3559a2eb6e0ec"}
HOP_SOURCES = ["paper_2602_20516_b300/csrc/lgt_dirac.cu", "paper_2602_20516_b300/csrc/lgt_spin.cuh",
               "paper_2602_20516_b300/csrc/lgt_common.cuh", "paper_2602_20516_b300/csrc/lgt_clover.cuh"]


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
    return {"workload": "32^3x64 Nf=2 Wilson eo; step = force eval (CG from 0, tol 1e-10) + kick + link update "
                        "on each of 4 fixed fields (MD steps 0,10,20,30 of the seeded sequence)",
            "force_evals_per_step": len(FIELD_STEPS), "field_md_steps": list(FIELD_STEPS),
            "lattice": list(DIMS), "beta": BETA, "kappa": KAPPA, "alpha": ALPHA, "tol": TOL,
            "delta": DELTA, "seed": SEED, "eps": EPS,
            "l2": "inputs > L2 (1.61 GB of links per field)",
            "hop_staging": args.staging,
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


# ---------------------------------------------------------------- CPU oracle
def cpu_info():
    model = platform.processor() or ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count(),
            "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}


_ORACLE_FIELDS = {}


def oracle_step_estimate(iters_by_field):
    """An ESTIMATE of one step of the workload on the FP64 oracle at 32^3 x 64, from a
    bounded sample on the seeded start field: CG capped at 1 iteration (2 operator
    applications with its residual check; per-iteration cost = t/2) plus the X/Y hops,
    gauge force, fermion force and link update, timed once.  One step is estimated as
    sum over the four fields of t_iter (iters + 1) + t_rest with the FP64 CG iteration
    counts of those fields.  Returns (seconds per step, sample description)."""
    import oracle as O
    d = DIMS
    if not _ORACLE_FIELDS:   # generated once per process, outside the sample
        _ORACLE_FIELDS["U"] = O.random_links(d, SEED, ALPHA)
        _ORACLE_FIELDS["phi"] = O.gaussian_spinor(d, SEED, 0, O.FIELD_SOURCE, 1)
        _ORACLE_FIELDS["mom"] = O.gaussian_momenta(d, SEED, 0)
    U, phi, mom = _ORACLE_FIELDS["U"], _ORACLE_FIELDS["phi"], _ORACLE_FIELDS["mom"]
    t0 = time.perf_counter()
    O.cg(d, U, KAPPA, phi, eo=True, tol=TOL, max_iter=1)
    t_iter = (time.perf_counter() - t0) / 2.0
    t1 = time.perf_counter()
    X = O.hop(d, U, phi, out_mask=2)
    Y = O.hop(d, U, X, out_mask=1)
    O.hop(d, U, Y, out_mask=2, dagger=True)
    O.gauge_force(d, U, BETA)
    O.fermion_force_xy(d, U, KAPPA, X, Y)
    O.update_links(d, U, mom, EPS)
    t_rest = time.perf_counter() - t1
    step = sum(t_iter * (iters_by_field[f] + 1) + t_rest for f in FIELD_STEPS)
    sample = (f"ESTIMATE from a sample: oracle (C, OpenMP) on the 32^3x64 start field, CG capped at 1 "
              f"iteration ({t_iter:.2f} s per iteration) scaled to the FP64 iteration counts of the 4 fields "
              f"{[iters_by_field[f] for f in FIELD_STEPS]} (+1 residual apply each), plus X/Y hops, gauge force, "
              f"fermion force and link update ({t_rest:.2f} s) per field")
    return step, sample


def oracle_full_force(dims=TABLE1_DIMS):
    """One complete FP64 oracle force evaluation (no extrapolation): CG on Dhat^+ Dhat
    from zero to tol 1e-10, fermion force, gauge force, at config 4's couplings on
    the seeded exp(i 0.5 H) field of the given lattice.  Threads: OMP_NUM_THREADS."""
    import oracle as O
    U = O.random_links(dims, SEED, ALPHA)
    phi = O.gaussian_spinor(dims, SEED, 0, O.FIELD_SOURCE, 1)
    t0 = time.perf_counter()
    Ff, it = O.pf_force(dims, U, KAPPA, phi, eo=True, tol=TOL)
    Fg = O.gauge_force(dims, U, BETA)
    sec = time.perf_counter() - t0
    del Ff, Fg
    return {"lattice": list(dims), "seconds": sec, "cg_iters": int(it), **cpu_info()}


def cpu_table1(threads_list=(1, None)):
    """The full oracle force at 24^4 with 1 thread and with every core, each in a
    process of its own (OpenMP reads its thread count at start)."""
    out = []
    for th in threads_list:
        env = dict(os.environ)
        if th is None:
            env.pop("OMP_NUM_THREADS", None)
        else:
            env["OMP_NUM_THREADS"] = str(th)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-force-once"], env=env,
                           capture_output=True, text=True, check=True)
        out.append(json.loads(r.stdout.strip().splitlines()[-1]))
    return {"oracle_force_24x4": out, "paper_table1_s": TABLE1_PAPER_S,
            "note": "paper: 24^4 Wilson fermions, no smearing, beta/kappa/tolerance not stated, CPU model not "
                    "stated; here config 4's couplings (beta 5.8, kappa 0.156, tol 1e-10) on the seeded "
                    "exp(i 0.5 H) field"}


def gpu_table1(reps=10, warmup=3):
    """The force evaluation of oracle_full_force (24^4, config 4's couplings, the seeded
    exp(i 0.5 H) field, CG from zero to tol 1e-10, even-odd fermion force + gauge
    force) on this GPU through the public API: the FP64 path and the mixed path
    (double-float forces), each the median of `reps` CUDA-event timings after `warmup`
    untimed evaluations, and the relative difference of the two forces."""
    import torch
    from paper_2602_20516_b300 import lgt
    torch.cuda.set_device(0)
    lat = lgt.Lattice(TABLE1_DIMS)
    lat.random_links(SEED, ALPHA)
    phi = lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    ap = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=FORCE_ARITH)
    stream = torch.cuda.current_stream()
    out, forces = {}, {}
    for name, sp in (("fp64_path", lgt.solver("fp64", tol=TOL)), ("mixed", lgt.solver("mixed", tol=TOL, delta=DELTA))):
        for _ in range(warmup):
            F, st = lat.force(ap, phi, sp)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F, st = lat.force(ap, phi, sp)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        forces[name] = F
        out[name] = {"ms_median": sorted(ms)[len(ms) // 2], "ms_min": min(ms), "cg_iters": st["iters"],
                     "reliable_updates": st["reliable_updates"]}
    out["force_rel_diff"] = (torch.linalg.norm(forces["mixed"] - forces["fp64_path"]) /
                             torch.linalg.norm(forces["fp64_path"])).item()
    return {"lattice": list(TABLE1_DIMS), "gpu": torch.cuda.get_device_name(0), **out, "reps": reps,
            "paper_table1_s": TABLE1_PAPER_S}


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
STAT_KEYS = ("iters", "reliable_updates", "breakdowns", "diverged", "handovers", "fp64_iters", "restarts")


def _round(v, sig=4):
    if isinstance(v, float):
        return float(f"{v:.{sig}g}")
    if isinstance(v, dict):
        return {k: _round(x, sig) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [_round(x, sig) for x in v]
    return v


def summarize_stats(st):
    """Per-field solver counts of one step (the steps repeat the same four solves) and
    their mean over the step."""
    n = len(FIELD_STEPS)
    first = st[:n]
    per_field = {str(f): {k: s[k] for k in STAT_KEYS} for f, s in zip(FIELD_STEPS, first)}
    sums = {k: sum(s[k] for s in st) / (len(st) / n) for k in STAT_KEYS}
    return per_field, sums


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
    lat.set_hop_staging(args.staging)
    lat.random_links(SEED + rank, ALPHA)
    phi = lat.gaussian_spinor(SEED + rank, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    mom = lat.gaussian_momenta(SEED + rank, 0)
    # headline mixed path: FP32 CG with FP64 reliable updates, forces in double-float
    # (FP32-pair) arithmetic accumulated in FP64; the FP64 path ignores force_arith
    ap = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=FORCE_ARITH)
    sp_mixed = lgt.solver("mixed", tol=TOL, delta=DELTA)
    sp64 = lgt.solver("fp64", tol=TOL)
    stream = torch.cuda.current_stream()

    # the workload's fields: links and momenta at the MD steps FIELD_STEPS of the seeded
    # sequence (untimed; every phase below starts each force evaluation from one of them)
    fields = []
    for k in range(max(FIELD_STEPS) + 1):
        if k in FIELD_STEPS:
            fields.append((lat.get_links(), mom.clone()))
        if k < max(FIELD_STEPS):
            lat.md_update(mom, EPS, lgt.UPDATE_P, ap, phi, sp_mixed)
            lat.md_update(mom, EPS, lgt.UPDATE_U)   # FP64: the fields do not depend on the update's arithmetic
    plaq = []
    for U, _ in fields:
        lat.set_links(U)
        plaq.append(lat.plaquette())

    def step(sp, stats, a=ap):
        for U, m in fields:
            lat.set_links(U)
            mom.copy_(m)
            stats.append(lat.md_update(mom, EPS, lgt.UPDATE_P, a, phi, sp))
            lat.md_update(mom, EPS, lgt.UPDATE_U, a, None, sp)

    def timed(sp, K, W, kernel_timing=False, clocks=None, a=ap, label="mixed"):
        st = []
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
            # every 7th hop launch (7 is prime to the 4 hops and 5 launches of a CG
            # iteration, so every kind is sampled): recording all of them slows the
            # step by ~2.4 %
            lgt.kernel_timing_start(1 << 16, every=HOP_TIMING_EVERY)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # an NVTX range per timed region (ncu --nvtx --nvtx-include "timed mixed/" captures it alone)
        torch.cuda.nvtx.range_push(f"timed {label}")
        e0.record(stream)
        for _ in range(K):
            step(sp, st, a)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches = lgt.launch_count()
        # hops enqueued after a solve stopped return at entry (a few us): excluded
        kt = lgt.kernel_timing_stop(HOP_MIN_MS) if kernel_timing else None
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        return ms, st, launches, kt, clk

    nf = len(FIELD_STEPS)
    K, W = args.steps, args.warmup
    sampler = ClockSampler(local)
    ms, st, launches, kt, clk = timed(sp_mixed, K, W, kernel_timing=True, clocks=sampler)
    ms_max = max_ranks(ms)
    value = whole_job_rate(world, nf * K, ms_max / 1e3)
    per_field, sums = summarize_stats(st)

    # FP64 path on the same four fields (each step the same work as a mixed step)
    K64 = max(1, min(K, args.fp64_steps))
    ms64, st64, _, kt64, _ = timed(sp64, K64, 1, kernel_timing=True, label="fp64")
    ms64 = max_ranks(ms64)
    value64 = whole_job_rate(world, nf * K64, ms64 / 1e3)
    per_field64, sums64 = summarize_stats(st64)

    # the other force arithmetics of the mixed path: FP64, and FP32 (~1e-7 force error,
    # moves Delta H by ~1e-4 relative)
    Kv = max(1, min(K, args.variant_steps))
    variants = {}
    for arith in ("fp64", "fp32"):
        apv = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=arith)
        msv, _, _, _, _ = timed(sp_mixed, Kv, 1, a=apv, label=f"arith {arith}")
        variants[arith] = {"value": whole_job_rate(world, nf * Kv, max_ranks(msv) / 1e3),
                           "ms_per_step": msv / Kv, "steps": Kv}

    # force of every arithmetic against the FP64 path's, field by field
    ferr = {"df64": [], "fp64": [], "fp32": []}
    for U, _ in fields:
        lat.set_links(U)
        fd, _ = lat.force(ap, phi, sp64)
        for arith in ferr:
            Fv, _ = lat.force(lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=arith),
                              phi, sp_mixed)
            ferr[arith].append((torch.linalg.norm(Fv - fd) / torch.linalg.norm(fd)).item())
            del Fv
        del fd
    for arith in ("fp64", "fp32"):
        variants[arith]["force_rel_err_vs_fp64_path_max"] = max(ferr[arith])

    # the even-odd clover action (c_sw = 1.0) against the Wilson one on the same fields,
    # at kappa = 0.13 (1 + A stays positive definite on them at the couplings used)
    clover = None
    if not args.no_clover:
        kc, cswc = 0.13, 1.0
        res_c = {}
        for name, csw in (("wilson_eo", 0.0), ("clover_eo", cswc)):
            apc = lgt.action_params(beta=BETA, kappa=kc, even_odd=True, force_arith=FORCE_ARITH, csw=csw)
            msc, stc, _, _, _ = timed(sp_mixed, Kv, 1, a=apc, label=name)
            res_c[name] = {"value": whole_job_rate(world, nf * Kv, max_ranks(msc) / 1e3), "ms_per_step": msc / Kv,
                           "cg_iters_per_step": sum(x["iters"] for x in stc) / Kv}
        clover = {"kappa": kc, "csw": cswc, **res_c,
                  "clover_overhead": res_c["clover_eo"]["ms_per_step"] / res_c["wilson_eo"]["ms_per_step"]}

    # dominant kernel: the FP32 hop, timed with CUDA events on its stream inside the
    # timed region; each epilogue variant counts its own algorithmic bytes
    kinds, n32_short = kt
    bytes32 = sum(HOP_BYTES_EPI["fp32"][e] * lat.Vh * n for (p, e), (ms_, n) in kinds.items() if p == "fp32")
    ms32_sum = sum(ms_ for (p, e), (ms_, n) in kinds.items() if p == "fp32")
    n32 = sum(n for (p, e), (ms_, n) in kinds.items() if p == "fp32")
    achieved = bytes32 / (ms32_sum * 1e-3) / 1e9
    per_variant = {e: {"launches": n, "avg_us": 1e3 * ms_ / n,
                       "GBs": HOP_BYTES_EPI["fp32"][e] * lat.Vh / (ms_ / n * 1e-3) / 1e9}
                   for (p, e), (ms_, n) in kinds.items() if p == "fp32"}
    hop_share = HOP_TIMING_EVERY * ms32_sum / ms   # FP32 hop launches' share of the timed region (sampled)
    # the true-residual hops of the mixed solver (double-float; FP64 before it)
    resid_kinds = {f"{p}:{e}": {"launches": n, "avg_us": 1e3 * ms_ / n}
                   for (p, e), (ms_, n) in kinds.items() if p != "fp32"}
    kinds64, _ = kt64
    plain64 = kinds64.get(("fp64", "hop"), (0.0, 0))
    hop64_ms = plain64[0] / max(plain64[1], 1)
    fp64_peak = lgt.measure_fp64_peak()
    peak, peak_kind = measured_peaks()
    traffic = NCU_TRAFFIC["bytes"] if NCU_TRAFFIC["sources_sha256"] == hop_sources_hash() else None

    # end to end through the public API with host buffers: for every force evaluation the
    # canonical links, momenta and phi are uploaded from pinned host memory, the MD update
    # (force + kick, link update) runs, and the kicked canonical momenta are downloaded;
    # the upload of evaluation j+1 and the download of j run on copy streams of their own
    # while j / j+1 compute (two device staging slots)
    e2e = None
    if not args.no_e2e:
        Ke = max(1, min(K, args.e2e_steps))
        Uhs = [U.cpu().pin_memory() for U, _ in fields]
        Mhs = [lat.unpack_momenta(m).cpu().pin_memory() for _, m in fields]
        phic = lat.unpack_spinor(phi, lgt.EVEN, lgt.FP64).cpu().pin_memory()
        Mout = [torch.empty_like(Mhs[0]).pin_memory() for _ in range(2)]
        Ud = [torch.empty_like(Uhs[0], device="cuda") for _ in range(2)]
        Md = [torch.empty_like(Mhs[0], device="cuda") for _ in range(2)]
        phid = [torch.empty_like(phic, device="cuda") for _ in range(2)]
        Mres = [torch.empty_like(Mhs[0], device="cuda") for _ in range(2)]
        copy_in = torch.cuda.Stream()
        copy_out = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        e2e_st = []

        def upload(j):
            q = j % 2
            with torch.cuda.stream(copy_in):
                copy_in.wait_event(ev_free[q])
                Ud[q].copy_(Uhs[j % nf], non_blocking=True)
                Md[q].copy_(Mhs[j % nf], non_blocking=True)
                phid[q].copy_(phic, non_blocking=True)
                ev_in[q].record(copy_in)

        def compute(j):
            q = j % 2
            stream.wait_event(ev_in[q])
            stream.wait_event(ev_done[q])   # the slot's previous download has finished
            lat.set_links(Ud[q])
            pf = lat.pack_spinor(phid[q], lgt.EVEN, lgt.FP64)
            m = lat.pack_momenta(Md[q])
            ev_free[q].record(stream)
            e2e_st.append(lat.md_update(m, EPS, lgt.UPDATE_P, ap, pf, sp_mixed))
            lat.md_update(m, EPS, lgt.UPDATE_U, ap, None, sp_mixed)
            Mres[q].copy_(lat.unpack_momenta(m))
            ev_out[q].record(stream)

        def download(j):
            q = j % 2
            with torch.cuda.stream(copy_out):
                copy_out.wait_event(ev_out[q])
                Mout[q].copy_(Mres[q], non_blocking=True)
                ev_done[q].record(copy_out)

        def pipeline(n):
            upload(0)
            for j in range(n):
                if j + 1 < n:
                    upload(j + 1)
                compute(j)
                download(j)
            torch.cuda.synchronize()

        pipeline(nf)   # warm-up: one step
        barrier()
        e2e_st.clear()
        t0 = time.perf_counter()
        pipeline(nf * Ke)
        barrier()
        te = max_ranks(time.perf_counter() - t0)
        h2d_b = Uhs[0].numel() * 16 + Mhs[0].numel() * 8 + phic.numel() * 16
        d2h_b = Mout[0].numel() * 8
        e2e = {"value": whole_job_rate(world, nf * Ke, te), "unit": UNIT,
               "h2d_bytes_per_step": nf * h2d_b, "d2h_bytes_per_step": nf * d2h_b, "steps": Ke,
               "cg_iters_per_step": sum(x["iters"] for x in e2e_st) / Ke,
               "step": "per field: upload canonical links, momenta and phi from pinned host memory, MD update "
                       "through the public API (force + kick, link update), download the kicked canonical "
                       "momenta; copies overlap the neighbouring evaluations on copy streams"}
        del Uhs, Mhs, Ud, Md, Mres

    multi = run_multi_rhs(lat, stream) if not args.no_multi else None

    serving = None
    if args.serve_requests > 0:
        free, total = torch.cuda.mem_get_info()
        serving = {"full": run_serving(args.serve_requests, int(0.8 * free), warmup=args.serve_warmup),
                   "mixed_only": run_serving(args.serve_requests, int(0.8 * free), warmup=args.serve_warmup,
                                             rates=(0.5, 0.9), mixed_fraction=1.0),
                   "tight_8GB": run_serving(args.serve_requests, 8 << 30, warmup=args.serve_warmup)
                   if args.serve_tight else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters64 = {f: per_field64[str(f)]["iters"] for f in FIELD_STEPS}
        est, sample = oracle_step_estimate(iters64)
        full = oracle_full_force()
        cpu = {"value": len(FIELD_STEPS) / est, "unit": UNIT, "kind": "oracle", "cores": full["threads"],
               "sample": sample, "cpu_model": full["model"],
               "full_force_24x4": {"seconds": full["seconds"], "cg_iters": full["cg_iters"],
                                   "threads": full["threads"],
                                   "paper_table1_single_thread_s": TABLE1_PAPER_S["single_thread_cpu_handwritten"]}}

    detail = {"plaquette_per_field": dict(zip(map(str, FIELD_STEPS), plaq)),
              "solver_per_field_mixed": per_field, "solver_per_field_fp64": per_field64,
              "force_rel_err_vs_fp64_path_per_field": ferr, "force_arith_variants": variants,
              "dslash_fp32_variants": per_variant, "residual_hops_in_mixed_region": resid_kinds,
              "clover": clover, "multi_rhs": multi, "serving": serving, "e2e": e2e, "cpu_baseline": cpu}

    def serve_summary(sv):
        if not sv:
            return None
        return {"saturated_req_s": sv["saturated_requests_per_s"], "requests_per_rate": sv["requests_per_rate"],
                **{r: [v["p50_ms"], v["p99_ms"], v["failed"]] for r, v in sv["rates"].items()}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 CG + df64 (f32-pair) reliable updates and forces, f64 sums (mixed)",
           "data": "synthetic: seeded exp(i 0.5 H) links evolved by seeded MD, Gaussian phi",
           "config": config_block(args),
           "cg": {"iters_per_step": sums["iters"], "iters_per_field": [per_field[str(f)]["iters"] for f in FIELD_STEPS],
                  "reliable_updates_per_step": sums["reliable_updates"], "breakdowns_per_step": sums["breakdowns"],
                  "diverged_per_step": sums["diverged"], "handovers_per_step": sums["handovers"],
                  "fp64_iters_per_step": sums["fp64_iters"]},
           "fp64": {"value": value64, "ms_per_step": ms64 / K64, "steps": K64,
                    "iters_per_field": [per_field64[str(f)]["iters"] for f in FIELD_STEPS],
                    "mixed_speedup": value / value64,
                    "mixed_force_rel_err_vs_fp64_path_max": max(ferr["df64"])},
           "roofline": {"bound": "hbm", "kernel": "hop_kernel<float> (FP32 Wilson hop, two-row links)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": peak_kind, "traffic": traffic,
                        "algorithmic_bytes_per_launch": bytes32 / max(n32, 1), "launches_timed": n32,
                        "timed_every": HOP_TIMING_EVERY,
                        "share_of_step": hop_share},
           "dslash": {"fp32_plain_hop_us": per_variant.get("hop", {}).get("avg_us"),
                      "df64_hop_us": resid_kinds.get("df64:hop", {}).get("avg_us"),
                      "fp64_plain_hop_us": hop64_ms * 1e3,
                      "fp64_hop_frac_of_fp64_peak": HOP_FLOPS * lat.Vh / (hop64_ms * 1e-3) / fp64_peak},
           "force_arith_variants": {k: round(v["value"], 3) for k, v in variants.items()},
           "clover_overhead": clover["clover_overhead"] if clover else None,
           "multi_rhs_solve4_speedup": multi["solve4"]["speedup"] if multi else None,
           "multi_rhs_same_kappa_speedup": multi["solve4_same_kappa"]["speedup"] if multi else None,
           "serving": serve_summary(serving["full"]) if serving else None,
           "serving_mixed_only": serve_summary(serving["mixed_only"]) if serving else None,
           "serving_tight_8GB": serve_summary(serving["tight_8GB"]) if serving else None,
           "cpu_baseline": ({k: cpu[k] for k in ("value", "unit", "kind", "cores", "cpu_model")} |
                            {"sample": "estimate from a capped-CG sample (see detail)",
                             "full_force_24x4_s": cpu["full_force_24x4"]["seconds"]}) if cpu else None,
           "e2e": ({k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "steps")}
                   if e2e else None),
           "clocks": clk, "gpu_launches": launches}
    # nested figures to 4 significant digits (the line must fit a 3 kB log tail)
    out = {k: (v if k in ("value", "ms_per_step", "config", "metric") else _round(v)) for k, v in out.items()}
    if args.detail and rank == 0:
        os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
        with open(args.detail, "w") as f:
            json.dump({"line": out, "detail": detail}, f, indent=1)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- several right-hand sides
def run_clover_sweep(kappas=(0.13, 0.135, 0.14, 0.145), steps=2):
    """The even-odd clover step (c_sw 1.0) against the Wilson step at several kappa on
    the workload's four fields (force evaluation from a zero guess, kick, link update
    per field; mixed solver, double-float forces): ms per step, CG iterations per step
    and their ratios.  A kappa where a clover solve or the odd-site inverse fails is
    reported with its error."""
    import torch
    from paper_2602_20516_b300 import lgt
    torch.cuda.set_device(0)
    lat = lgt.Lattice(DIMS)
    lat.random_links(SEED, ALPHA)
    phi = lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    mom = lat.gaussian_momenta(SEED, 0)
    ap0 = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith=FORCE_ARITH)
    sp = lgt.solver("mixed", tol=TOL, delta=DELTA)
    fields = []
    for k in range(max(FIELD_STEPS) + 1):
        if k in FIELD_STEPS:
            fields.append((lat.get_links(), mom.clone()))
        if k < max(FIELD_STEPS):
            lat.md_update(mom, EPS, lgt.UPDATE_P, ap0, phi, sp)
            lat.md_update(mom, EPS, lgt.UPDATE_U)
    stream = torch.cuda.current_stream()

    def timed(a):
        iters = 0
        for rep in range(steps + 1):   # the first pass is the warm-up
            if rep == 1:
                iters = 0
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            for U, m in fields:
                lat.set_links(U)
                mom.copy_(m)
                iters += lat.md_update(mom, EPS, lgt.UPDATE_P, a, phi, sp)["iters"]
                lat.md_update(mom, EPS, lgt.UPDATE_U, a, None, sp)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, iters / steps

    out = []
    for kc in kappas:
        row = {"kappa": kc}
        for name, csw in (("wilson", 0.0), ("clover", 1.0)):
            a = lgt.action_params(beta=BETA, kappa=kc, even_odd=True, force_arith=FORCE_ARITH, csw=csw)
            try:
                ms, it = timed(a)
                row[name] = {"ms_per_step": ms, "cg_iters_per_step": it}
            except lgt.LGTError as e:
                row[name] = {"error": str(e)}
        if "ms_per_step" in row["wilson"] and "ms_per_step" in row["clover"]:
            row["overhead"] = row["clover"]["ms_per_step"] / row["wilson"]["ms_per_step"]
            row["iters_ratio"] = row["clover"]["cg_iters_per_step"] / row["wilson"]["cg_iters_per_step"]
        out.append(row)
        print(json.dumps(row), flush=True)
    return {"clover_sweep": out, "csw": 1.0, "steps": steps}


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
    sp = lgt.solver("mixed", tol=TOL, delta=DELTA)

    def solve4(kap):
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
        return {"kappa": kap, "seconds_together": t_multi, "seconds_one_by_one": t_single,
                "iters": [s["iters"] for s in sts], "speedup": t_single / t_multi}
    # four systems at spread kappa, and four sources at one kappa (serving several
    # sources on one field), where the systems converge together
    return {"hop_fp32": hop, "solve4": solve4([0.150, 0.152, 0.154, 0.156]),
            "solve4_same_kappa": solve4([KAPPA] * 4)}


# ---------------------------------------------------------------- serving (p50/p99 latency)
SERVE_VOLUMES = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 48)]


def run_serving(n_per_rate, budget_bytes, seed=10, warmup=None, rates=(0.5, 0.9, 1.2), mixed_fraction=0.5,
                batch_iters=8, max_active=16):
    """Resident pool of 2 gauge fields per volume (alpha ~ U[0.3, 0.6]); requests:
    70% Dirac solves, 30% force evaluations, kappa ~ U[0.14, 0.157], a fraction
    `mixed_fraction` in mixed precision and the rest FP64 (0.5: half FP64; 1.0:
    every request mixed), tol 1e-10.  Saturated throughput, then open-loop Poisson
    arrivals at 0.5, 0.9 and 1.2 x that rate (1.2 x is overload: no steady state);
    latency = completion - scheduled arrival, over the requests after the first
    `warmup`."""
    import numpy as np
    from paper_2602_20516_b300 import serve
    rng = np.random.default_rng(seed)
    srv = serve.Server(budget_bytes, max_active=max_active, batch_iters=batch_iters, delta=DELTA)
    gids, vol = [], {}
    for k, d in enumerate(SERVE_VOLUMES):
        for j in range(2):
            g = srv.add_gauge(d, 1000 + 10 * k + j, float(rng.uniform(0.3, 0.6)))
            gids.append(g)
            vol[g] = "x".join(map(str, d))
    warm = max(10, n_per_rate // 10) if warmup is None else warmup
    serve.saturated(srv, serve.workload(gids, warm, seed=seed, mixed_fraction=mixed_fraction))   # warm-up
    thr, done = serve.saturated(srv, serve.workload(gids, n_per_rate, seed=seed + 1, mixed_fraction=mixed_fraction))
    out = {"saturated_requests_per_s": thr, "budget_bytes": budget_bytes, "mixed_fraction": mixed_fraction,
           "batch_iters": batch_iters, "max_active": max_active,
           "requests_per_rate": n_per_rate, "warmup_per_rate": warm, "rates": {}}

    def label(c):
        return f"{vol[c['gauge_id']]}/{'solve' if c['kind'] == serve.SOLVE else 'force'}/{c['precision']}"
    for j, f in enumerate(rates):
        reqs = serve.workload(gids, n_per_rate + warm, seed=seed + 2 + j, mixed_fraction=mixed_fraction)
        d = serve.poisson(srv, reqs, f * thr, seed=seed + 20 + j, warmup=warm)
        st = serve.latency_stats(d)
        st["offered_per_s"] = f * thr
        st["completed"] = len(d)
        st["overload"] = f > 1.0
        st["by_class"] = serve.latency_breakdown(d, label)
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
    """The oracle on the host cores, on this arm's workload: each step is the
    estimate of one step (four force evaluations with their link updates) from a
    bounded capped-CG sample, scaled with the same FP64 iteration counts of the four
    fields that the default arm measures on the GPU."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    est = []
    for _ in range(W + K):
        t, sample = oracle_step_estimate(CG_ITERS_FP64)
        est.append(t)
    timed = est[W:]
    value = len(FIELD_STEPS) * len(timed) / sum(timed)
    info = cpu_info()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": K, "warmup": W, "ms_per_step": 1e3 * statistics.mean(timed), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (same seeds)",
           "config": config_block(args),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["threads"], "kind": "oracle",
                            "cpu_model": info["model"], "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- serving record (config 5 as stated)
def run_serve_only(args):
    """The serving measurement alone, under the full budget and under 8 GB:
    --serve-requests per arrival rate after --serve-warmup (config 5: 5000 after 200)."""
    import torch
    torch.cuda.set_device(0)
    free, _ = torch.cuda.mem_get_info()
    nt = args.serve_requests if args.serve_tight_requests == 0 else args.serve_tight_requests   # < 0 skips it
    f, bi = args.serve_mixed_fraction, args.serve_batch_iters
    out = {"metric": "serving: p50/p99 latency (arrival -> completion) and requests/s", "mixed_fraction": f,
           "full": run_serving(args.serve_requests, int(0.8 * free), warmup=args.serve_warmup, mixed_fraction=f,
                               batch_iters=bi, max_active=args.serve_max_active),
           "tight_8GB": run_serving(nt, 8 << 30, warmup=min(args.serve_warmup or nt // 10, nt // 5),
                                    mixed_fraction=f, batch_iters=bi) if nt > 0 else None}
    if args.detail:
        with open(args.detail, "w") as f:
            json.dump(out, f, indent=1)
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- single-kernel mode (ncu)
def run_kernel(args):
    import torch
    from paper_2602_20516_b300 import lgt
    dims = tuple(args.lattice) if args.lattice else DIMS
    lat = lgt.Lattice(dims)
    lat.set_hop_staging(args.staging)
    lat.random_links(SEED, ALPHA)
    if args.kernel == "force_df":
        # one mixed-precision force evaluation with double-float force arithmetic
        phi = lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.EVEN)
        ap = lgt.action_params(beta=BETA, kappa=KAPPA, even_odd=True, force_arith="df64")
        for _ in range(args.reps):
            lat.force(ap, phi, lgt.solver("mixed", tol=TOL, delta=DELTA))
        torch.cuda.synchronize()
        print(json.dumps({"kernel": args.kernel, "force_evals": args.reps, "lattice": list(dims)}))
        return
    if args.kernel == "clover_md":
        # mixed-precision MD steps with the even-odd clover action (kappa 0.13, c_sw 1.0)
        phi = lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.EVEN)
        ap = lgt.action_params(beta=BETA, kappa=0.13, even_odd=True, force_arith=FORCE_ARITH, csw=1.0)
        sp = lgt.solver("mixed", tol=TOL, delta=DELTA)
        mom = lat.momentum_field()
        for _ in range(args.reps):
            st = lat.md_update(mom, EPS, lgt.UPDATE_P, ap, phi, sp)
            lat.md_update(mom, EPS, lgt.UPDATE_U, ap, None, sp)
        torch.cuda.synchronize()
        print(json.dumps({"kernel": args.kernel, "md_steps": args.reps, "lattice": list(dims), "last_solve": st}))
        return
    prec = {"hop32": lgt.FP32, "hop64": lgt.FP64, "hopdf": lgt.DF64}[args.kernel]
    src = lat.pack_spinor(lat.unpack_spinor(lat.gaussian_spinor(SEED, 0, lgt.FIELD_SOURCE, lgt.ODD),
                                            lgt.ODD, lgt.FP64), lgt.ODD, prec)
    out = lat.spinor_field(lgt.EVEN, prec)
    # untimed launches for about a second first (clocks ramp up under load)
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        lat.dslash(src, lgt.OP_HOP, lgt.EVEN, False, 0.0, prec, out=out)
        torch.cuda.synchronize()
    lgt.kernel_timing_start(max(args.reps, 1))
    for _ in range(args.reps):
        lat.dslash(src, lgt.OP_HOP, lgt.EVEN, False, 0.0, prec, out=out)
    torch.cuda.synchronize()
    kinds, _ = lgt.kernel_timing_stop()
    us = {f"{p_}:{e}": 1e3 * ms / n for (p_, e), (ms, n) in kinds.items()}
    print(json.dumps({"kernel": args.kernel, "launches": args.reps, "lattice": list(dims), "avg_us": us}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--detail", default="", help="also write the per-field and per-phase figures to this file")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 path (same four fields; each step the same work)")
    ap.add_argument("--variant-steps", type=int, default=3,
                    help="timed steps of the force-arithmetic and clover variants")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-multi", action="store_true", help="skip the several-sources measurement")
    ap.add_argument("--no-clover", action="store_true", help="skip the even-odd clover measurement")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests per arrival rate in the serving measurement (0 skips it)")
    ap.add_argument("--serve-warmup", type=int, default=None,
                    help="warm-up requests per rate (default: a tenth of --serve-requests)")
    ap.add_argument("--serve-tight", action="store_true", help="also run serving under an 8 GB budget")
    ap.add_argument("--serve-tight-requests", type=int, default=0,
                    help="--serve-only: requests per rate under the 8 GB budget (default: --serve-requests; "
                         "negative: skip it)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving measurement (full budget and 8 GB) and print it")
    ap.add_argument("--serve-mixed-fraction", type=float, default=0.5,
                    help="--serve-only: fraction of requests in mixed precision (the rest FP64)")
    ap.add_argument("--serve-batch-iters", type=int, default=8,
                    help="--serve-only: CG iterations per request per scheduling step")
    ap.add_argument("--serve-max-active", type=int, default=16,
                    help="--serve-only: requests running at once")
    ap.add_argument("--hmc", type=int, default=0, help="run this many HMC trajectories instead (own JSON line)")
    ap.add_argument("--hmc-fp64", type=int, default=2, help="trajectories replayed on the FP64 path")
    ap.add_argument("--log", default="", help="HMC mode: append one JSON line per trajectory to this file")
    ap.add_argument("--checkpoint", default="", help="HMC mode: write the chain's checkpoint here after every trajectory")
    ap.add_argument("--chrono", type=int, default=0,
                    help="HMC mode: MD solves start from the last N solutions (chronological guess)")
    ap.add_argument("--staging", type=int, default=0, choices=[0, 1, 2, 3],
                    help="FP32 hops: stage links (1), spinors with halos (2) or both (3) in shared memory")
    ap.add_argument("--kernel", choices=["hop32", "hop64", "hopdf", "force_df", "clover_md"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--lattice", type=int, nargs=4, default=None, metavar=("LX", "LY", "LZ", "LT"),
                    help="--kernel: lattice extents (default 32 32 32 64); small cases for multi-pass profiles")
    ap.add_argument("--cpu-table1", action="store_true",
                    help="one complete oracle force evaluation at 24^4 with 1 thread and with every core")
    ap.add_argument("--cpu-force-once", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--clover-sweep", action="store_true",
                    help="clover / Wilson step time at several kappa (own JSON lines)")
    ap.add_argument("--gpu-table1", action="store_true",
                    help="the 24^4 force evaluation of --cpu-table1 on the GPU (FP64 and mixed paths)")
    args = ap.parse_args()
    if args.impl == "ours" and not args.kernel:
        args.warmup = max(3, args.warmup)   # timing rule: at least 3 untimed steps
    if args.cpu_force_once:
        print(json.dumps(oracle_full_force()))
    elif args.clover_sweep:
        print(json.dumps(run_clover_sweep()))
    elif args.gpu_table1:
        print(json.dumps(gpu_table1()))
    elif args.cpu_table1:
        print(json.dumps(cpu_table1()))
    elif args.kernel:
        run_kernel(args)
    elif args.hmc > 0:
        run_hmc(args)
    elif args.serve_only:
        run_serve_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
