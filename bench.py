"""Benchmark: LJ + ATM molecular-dynamics steps on a homogeneous liquid.

One step = one velocity-Verlet step of the whole hot path through the C ABI:
half kick + drift, wrap + bin + stable sort into linked cells, LJ pair forces,
ATM three-body forces (traversal x truncation x precision), reductions of
energy / virial / counts, second half kick.  The default workload is the
N = 256,000 liquid at rho* = 0.8, T* = 1.0 (fcc start with +-0.05 jitter,
r_c = 2.5, nu = 0.073), 3c08 traversal, pair truncation, FP32C arithmetic.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores on a bounded sample of the same workload instead.

Multi-GPU (torchrun): every rank advances its own independent replica (seeded
by rank); there is no data-path collective ("replicas only", weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2510_21230_gb300 import analysis, synth  # noqa: E402

METRIC = "3-body molecule updates/s at N=256k, FP64 exact vs FP32 vs surrogate at stated error"
UNIT = "molecule updates/s"
NU, RC = 0.073, 2.5
L2_FLUSH_BYTES = 256 << 20

# FP32 / FP64 issue widths per SM per clock on GB300 (152 SMs): 128 FP32 lanes,
# FP64 derived from the nominal 1.25 TFLOP/s at 2070 MHz (about 2 DFMA per clock per SM)
SMS = 152
FP32_FLOPS_PER_CLK_SM = 256.0
FP64_FLOPS_PER_CLK_SM = 1.25e12 / (SMS * 2.07e9)

# Useful flops per interacting triplet, counted from the kernel's evaluate()
# (FMA = 2, the reciprocal square root = 1): 3 displacements 42, ATM terms 49,
# gradient scalars, energy and virial 9, force vectors 27 (3c01: 9).
F3 = {"3c01": 109.0, "3c18": 127.0, "3c08": 127.0, "3c08a": 127.0}

# Useful flops per interacting LJ pair when a step evaluates LJ inside the
# block units (3c08 / 3c18 / 3c08a, pair rule): displacement and square 14,
# the LJ scalar 9, energy and virial 4 (the force vector is the ATM gather's).
F2_FUSED = 27.0
FUSED_TRAV = ("3c08", "3c18", "3c08a")

# DRAM traffic per ATM evaluation (dram__bytes_read.sum + dram__bytes_write.sum
# of its kernels -- the FP32C pair rule's pair-bitmap kernel and the block
# kernel -- from one ncu capture, whose replays start from a flushed L2: the
# bitmaps the block kernel reads count as DRAM bytes there, though a run finds
# them in L2), keyed by (traversal, truncation, precision, workload), with the
# sha256 prefix of the kernel sources it was taken from: a changed kernel
# reports null until it is captured again.  liquid_n256k is the N = 32,000
# capture (2197 units) scaled to 19683 units.
KERNEL_SOURCES = ["atm3_internal.cuh", "atm_common.cuh", "atm_block.cuh", "atm_owner.cuh",
                  "atm_fp32.cu", "atm_fp64.cu", "atm_launch.cuh", "pair_masks.cu"]
TRAFFIC = {("3c08", "pair", "fp32c", "liquid_n256k"): (32.43e6, "86ebe58ae46bedf4"),
           ("3c08", "pair", "fp32c", "liquid_n32k"): (3.620e6, "86ebe58ae46bedf4")}


# Issued FP32 flops (fadd + fmul + 2 ffma thread instructions of the ATM
# evaluation's kernels, from the same ncu capture) over its useful flops,
# with the source hash they belong to: what candidates and bookkeeping add
# in floating point.
ISSUED = {("3c08", "pair", "fp32c"): (0.929, "86ebe58ae46bedf4")}


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2510_21230_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(trav, trunc, prec, workload):
    t = TRAFFIC.get((trav, trunc, prec, workload))
    if t is None or t[1] != kernel_hash():
        return None
    return t[0]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="liquid_n256k", choices=sorted(synth.CONFIGS))
    p.add_argument("--trav", default="3c08", choices=["3c01", "3c18", "3c08", "3c08a", "3cw"])
    p.add_argument("--trunc", default="pair", choices=["pair", "product"])
    p.add_argument("--prec", default="fp32c", choices=["fp64", "fp32c", "surrogate"])
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-tune", action="store_true", help="skip the launch-form autotuner")
    p.add_argument("--no-surrogate", action="store_true", help="skip the surrogate variant")
    p.add_argument("--sur-frames", type=int, default=1000,
                   help="training frames of each of the N=1000 and N=32,000 liquids")
    p.add_argument("--sur-stride", type=int, default=10, help="MD steps between frames")
    p.add_argument("--sur-steps", type=int, default=20000, help="Adam steps")
    p.add_argument("--sur-batch", type=int, default=8192, help="rows per Adam step")
    p.add_argument("--paper-table", action="store_true",
                   help="also time the paper's own runtime workload (context only)")
    p.add_argument("--kernel-case", action="store_true",
                   help="only time repeated force evaluations of one combination (a small "
                        "driver for profilers: cell build, LJ and the chosen ATM or surrogate "
                        "kernel) and print their CUDA-event time")
    p.add_argument("--n", type=int, default=0,
                   help="--kernel-case: a liquid of N molecules at rho 0.8 instead of the "
                        "workload (N = 104052 has the cell edge of the 256,000 liquid)")
    p.add_argument("--reps", type=int, default=3, help="--kernel-case: evaluations per timing")
    p.add_argument("--nwarps", type=int, default=0, help="--kernel-case: warps per CTA")
    p.add_argument("--det", action="store_true", help="--kernel-case: deterministic mode")
    p.add_argument("--train", type=int, default=0,
                   help="--kernel-case with --prec surrogate: instead, time this many Adam "
                        "steps of 8192 rows on exact forces of 20 frames of the 1000 liquid")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device):
    """The largest value over all ranks of the process group (the job's time
    is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name, rank):
    c = synth.CONFIGS[name]
    cfg = synth.homogeneous(c["n"], c["rho"], c["T"], c["seed"] + rank)
    cfg["name"] = name
    return cfg


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ------------------------------------------------------------------ per-phase rooflines

# Algorithmic HBM bytes per molecule and step of the memory-bound phases (the
# minimum each must move, counted from the kernels' loads and stores):
#  cell build: wrap x in place (24 + 24), cell id and arrival rank (4 + 4),
#    scatter (reads cell id and rank 8, writes the slot 4), per-cell order and
#    local coordinates (perm 4 + 4, x 24, FP64 and FP32 local 24 + 12, slot cell 4)
#  two half kicks: forces 24 (LJ part 24, zero when fused), v 24 + 24, x 24 + 24
#    (drift, once), kinetic energy 8, perm 4
CELL_BYTES_PER_MOL = 24 + 24 + 4 + 4 + 8 + 4 + 4 + 4 + 24 + 24 + 12 + 4
CELL_BYTES_PER_CELL = 4 * 4
KICK_BYTES_PER_MOL = 2 * (24 + 24 + 24 + 24 + 8 + 4) + (24 + 24)


def ncell_of(cfg):
    from paper_2510_21230_gb300 import atm3
    return int(np.prod(atm3.cell_grid(cfg["box"], RC)))


def kernel_rooflines(prof, steps, n, ncell, atm_roof, pk):
    """Achieved fraction of the bounding roofline for each phase of a step:
    the ATM kernel against the FP32 pipe (from `roofline`, the timed steps),
    the cell build and the kicks (from prof, the split pass) against the
    measured HBM bandwidth (algorithmic bytes)."""
    hbm = pk.get("hbm_gbs")
    out = {"atm_triplets": {"bound": "alu", "frac": atm_roof["frac"],
                            "ms_per_step": atm_roof["ms_per_launch"]}}
    per_step = max(1, steps)
    for name, key, nbytes in (("cell_build", "ms_cells", CELL_BYTES_PER_MOL * n + CELL_BYTES_PER_CELL * ncell),
                              ("kicks_and_reductions", "ms_md", KICK_BYTES_PER_MOL * n)):
        ms = prof[key] / per_step
        gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else None
        out[name] = {"bound": "hbm", "ms_per_step": ms, "bytes_per_step": nbytes,
                     "achieved_gbs": gbs, "peak_gbs": hbm,
                     "frac": (gbs / hbm) if (gbs and hbm) else None}
    return out


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.offset = 0

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self):
        """Only samples written after this call count (the timed region starts)."""
        if self.proc is not None:
            self.offset = os.path.getsize(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        with open(self.path) as fh:
            fh.seek(self.offset)
            for line in fh:
                parts = [t.strip() for t in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                      "sw_power_cap"], parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2510_21230_gb300 import atm3, build

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # one build per node (ranks of a node share the build folder), then all load it
    if local == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    atm3.load()
    cfg = workload(args.workload, rank)
    n = cfg["n"]
    stream = torch.cuda.current_stream()
    sysm = atm3.AtmSystem(cfg["box"], n, rc=RC, nu=NU, dt=0.002, device=local,
                          stream=stream.cuda_stream)
    sysm.set_state(cfg["x"], cfg["v"])
    tuning = None
    if not args.no_tune:
        # the library's autotuner picks the launch form (one CTA per unit or
        # persistent, warps per CTA) for the measured combination
        sysm.build_cells()
        tuning = sysm.autotune(args.trav, args.trunc, args.prec, reps=3)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(trav, trunc, prec, steps, warmup, clocks=None, forces_only=True):
        # the timed steps record timestamps around the force evaluations only
        # (the roofline's kernel time); the other phases' split comes from an
        # untimed pass with every launch group bracketed
        sysm.step(warmup, trav, trunc, prec)
        torch.cuda.synchronize()
        sysm.set_profiling(True, forces_only=forces_only)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
            clocks.mark()
        evs = []
        t_host = time.perf_counter()
        for _ in range(steps):
            flush.fill_(1.0)  # evict L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sysm.step(1, trav, trunc, prec, sync=False)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        t_host = time.perf_counter() - t_host
        clk = clocks.stop() if clocks else None
        ms = sum(a.elapsed_time(b) for a, b in evs)
        prof = sysm.get_profile()
        res = sysm.step(0, trav, trunc, prec)
        if ws > 1:
            ms = max_over_ranks(ms, "cuda")
        return dict(ms=ms, host_s=t_host, prof=prof, res=res, clocks=clk)

    clocks = ClockSampler(local) if rank == 0 else None
    main = timed(args.trav, args.trunc, args.prec, args.steps, args.warmup, clocks)
    ms_step = main["ms"] / args.steps
    value = n * ws * args.steps / (main["ms"] * 1e-3)
    split_steps = max(3, min(args.steps, 50))
    split = timed(args.trav, args.trunc, args.prec, split_steps, 1, None, forces_only=False)

    # roofline of the dominant kernel (ATM triplets): useful flops per launch / launch time
    prof = main["prof"]
    atm_ms = prof["ms_atm"] / max(1, prof["n_atm_launches"])
    fused = args.trav in FUSED_TRAV and args.trunc == "pair"
    flops = F3[args.trav] * main["res"]["n_int3"]
    if fused:
        flops += F2_FUSED * main["res"]["n_int2"]
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    per_clk = FP32_FLOPS_PER_CLK_SM if args.prec == "fp32c" else FP64_FLOPS_PER_CLK_SM
    derived = SMS * per_clk * sm_max * 1e6 / 1e12
    # the roof is the device's measured FMA throughput in the path's precision
    # (independent FMA chains on every SM, same clocks, this run)
    measured = atm3.measure_fma_peak(local, args.prec == "fp64")
    peak = measured if measured and measured > 0 else derived
    achieved = flops / (atm_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_for(args.trav, args.trunc, args.prec, args.workload),
                "kernel": ("atm_owner_kernel<%s,%s,%s>" if args.trav == "3c01" else "atm_block_kernel<%s,%s,%s>") % (args.trav, args.trunc, args.prec)
                          + (" (LJ of the c08 pairs inside)" if fused else "")
                          + (" after k_pair_masks" if args.prec == "fp32c" and args.trunc == "pair"
                             and args.trav in ("3c08", "3c18", "3c08a") else ""),
                "peak_source": ("measured: atm_measure_fma_peak, %s FMA chains on every SM"
                                % ("FP32" if args.prec == "fp32c" else "FP64"))
                               if peak == measured else "derived (measurement failed)",
                "derived_peak_tflops": derived,
                "derived_peak_source": "%d SMs x %.2f flops/clk x %.0f MHz (%s pipe)"
                                       % (SMS, per_clk, sm_max,
                                          "FP32" if args.prec == "fp32c" else "FP64, nominal"),
                "flops_per_interacting_triplet": F3[args.trav],
                "flops_per_interacting_pair": F2_FUSED if fused else None,
                "ms_per_launch": atm_ms,
                "measured_fma_peak_tflops": measured,
                "measured_rsqrt_peak_gops": atm3.measure_rsqrt_peak(local),
                "rsqrt_per_s_needed_gops": main["res"]["n_int3"] / (atm_ms * 1e-3) / 1e9}
    tr = roofline["traffic"]
    hbm = pk.get("hbm_gbs")
    if tr is not None and hbm:
        # the kernel's DRAM bytes per launch over its time, against measured HBM copy bandwidth
        roofline["hbm_achieved_gbs"] = tr / (atm_ms * 1e-3) / 1e9
        roofline["hbm_peak_gbs"] = hbm
        roofline["hbm_frac"] = roofline["hbm_achieved_gbs"] / hbm
    iss = ISSUED.get((args.trav, args.trunc, args.prec))
    if iss is not None and iss[1] == kernel_hash():
        roofline["issued_over_useful_flops"] = iss[0]
        roofline["issued_frac"] = roofline["frac"] * iss[0]

    # paper-style 3-body MUPS: N / (ATM force time)
    mups_3body = n / (atm_ms * 1e-3)

    # force error of FP32C against the FP64 GPU path on the same state
    force_err = None
    if args.prec == "fp32c":
        sysm.build_cells()
        r64 = sysm.compute_forces(args.trav, args.trunc, "fp64")
        f64 = sysm.get_forces("atm")
        r32 = sysm.compute_forces(args.trav, args.trunc, "fp32c")
        f32 = sysm.get_forces("atm")
        scale = float(np.sqrt(np.mean(f64 ** 2)))
        d = np.abs(f32 - f64)
        # a pair within FP32 rounding of r_c can be decided differently in
        # the two precisions; every triplet on it then changes the force of
        # its three molecules by a term of the size of a triplet at the cutoff
        force_err = {"vs": "fp64 GPU path, same state", "max_abs_over_rms": float(d.max() / scale),
                     "p99_99_abs_over_rms": float(np.quantile(d, 0.9999) / scale),
                     "rms_rel": float(np.sqrt(np.mean(d ** 2)) / scale),
                     "n_int3_fp32c": int(r32["n_int3"]), "n_int3_fp64": int(r64["n_int3"])}

    # variants (same state, fewer steps)
    variants = []
    vpeak = {args.prec: measured}  # measured FMA peaks per precision
    if not args.no_variants and rank == 0:
        for tv, tr, pr, det in [("3c08", "pair", "fp64", False), ("3c18", "pair", "fp32c", False),
                                ("3c08", "product", "fp32c", False), ("3c18", "pair", "fp64", False),
                                ("3c08a", "pair", "fp32c", False), ("3c08", "pair", "fp32c", True)]:
            if (tv, tr, pr) == (args.trav, args.trunc, args.prec) and not det:
                continue
            k = max(2, min(5, args.steps))
            if det:
                sysm.set_deterministic(True)
            r = timed(tv, tr, pr, k, 2)
            if det:
                sysm.set_deterministic(False)
            am = r["prof"]["ms_atm"] / max(1, r["prof"]["n_atm_launches"])
            # useful flops over the ATM evaluation's time, against the measured
            # FMA peak of the variant's precision
            vflops = F3[tv] * r["res"]["n_int3"]
            if tv in FUSED_TRAV and tr == "pair":
                vflops += F2_FUSED * r["res"]["n_int2"]
            if pr not in vpeak:
                vpeak[pr] = atm3.measure_fma_peak(local, pr == "fp64")
            vach = vflops / (am * 1e-3) / 1e12
            variants.append({"traversal": tv, "truncation": tr, "precision": pr,
                             "deterministic": det,
                             "value": n * k / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / k,
                             "atm_ms_per_launch": am, "mups_3body": n / (am * 1e-3),
                             "n_int3": r["res"]["n_int3"],
                             "roofline": {"bound": "alu", "achieved": vach, "peak": vpeak[pr],
                                          "unit": "TFLOP/s",
                                          "frac": vach / vpeak[pr] if vpeak[pr] else None,
                                          "peak_source": "measured: atm_measure_fma_peak, %s FMA "
                                          "chains on every SM" % ("FP64" if pr == "fp64" else "FP32")}})
            if det and tuning is not None:
                # the mode switch reset the tuned launch form: tune again
                sysm.build_cells()
                sysm.autotune(args.trav, args.trunc, args.prec, reps=3)
            if tv == "3c08a" and (args.trav, args.trunc) == ("3c08", "pair"):
                # the corner-anchored 3c08 omits the triplets of cornerless
                # block triples: its share of the complete 3c08's, same state
                full = sysm.compute_forces("3c08", "pair", "fp32c")
                variants[-1]["found_fraction_vs_3c08"] = r["res"]["n_int3"] / full["n_int3"]
    # batched ensemble: 64 independent replicas in one context (one launch per
    # kernel for the whole batch), autotuned ATM launch form, graph-captured step
    batch = None
    if not args.no_variants and rank == 0:
        batch = batch_variant(atm3, local, stream, flush)

    # vapour-liquid slab with the density profile rho(z) accumulated every step
    slab = None
    if not args.no_variants and rank == 0:
        slab = slab_variant(atm3, local, stream, flush)

    # product-rule completeness: the wide traversal finds every product-rule
    # triplet of the N = 32,000 liquid; the paper's block traversals a subset
    completeness = None
    if not args.no_variants and rank == 0:
        completeness = completeness_variant(atm3, local, stream)

    # the paper's own runtime workload (its node-level table): all six
    # traversal / truncation combinations, three-body force time only
    paper_table = None
    if args.paper_table and rank == 0:
        paper_table = paper_table_variant(atm3, local, stream)

    # learned surrogate: trained on exact forces of smaller liquids, then
    # timed and checked on this workload's state
    surrogate = None
    if not args.no_surrogate and rank == 0:
        P, mean, scale, info = train_surrogate(atm3, args, local, stream.cuda_stream)
        sysm.surrogate_set_model(P, mean, scale)
        sysm.build_cells()
        sysm.compute_forces("3c08", "pair", "fp64")
        f64 = sysm.get_forces("atm")
        sysm.compute_forces("3c08", "pair", "surrogate")
        fsur = sysm.get_forces("atm")
        scale_f = float(np.sqrt(np.mean(f64 ** 2)))
        d = fsur - f64
        # surrogate kernel alone (no exact steps), then the amortised step with
        # the exact FP32C traversal every 50 steps
        sysm.surrogate_options(exact_every=0)
        r0 = timed("3c08", "pair", "surrogate", 10, 3)
        sm = r0["prof"]["ms_atm"] / max(1, r0["prof"]["n_atm_launches"])
        sysm.surrogate_options(exact_every=50)
        sysm.surrogate_error(reset=True)
        r1 = timed("3c08", "pair", "surrogate", 50, 3)
        ed, ee, ek = sysm.surrogate_error()
        surrogate = {
            "precision": "surrogate (FP32 descriptors + LJ in one neighbour pass, bf16 tcgen05 MLP)",
            "value": n * 50 / (r1["ms"] * 1e-3), "ms_per_step": r1["ms"] / 50,
            "steps": "50 timed, exact FP32C 3c08 traversal every 50 (one in the timed run)",
            "ms_per_step_surrogate_only": r0["ms"] / 10,
            "sur_ms_per_launch": sm, "mups_3body": n / (sm * 1e-3),
            "force_error": {"vs": "fp64 exact ATM force (3c08, pair), same state",
                            "rms_rel": float(np.sqrt(np.mean(d ** 2)) / scale_f),
                            "max_abs_over_rms": float(np.abs(d).max() / scale_f)},
            "online_check": {"rms_diff_over_rms_exact": ed / ee if ee > 0 else None,
                             "checks": ek},
            "training": info,
            "observables": surrogate_observables(atm3, P, mean, scale, local, stream),
        }

    # end to end through the public API with host buffers: per step H2D of
    # the state (x, v) and its force F from pinned memory, one velocity-Verlet
    # step (one force evaluation, at the new positions), D2H of (x, v, F)
    e2e = None
    if rank == 0:
        xh = torch.empty((3, n), dtype=torch.float64).pin_memory()
        vh = torch.empty((3, n), dtype=torch.float64).pin_memory()
        fh = torch.empty((3, n), dtype=torch.float64).pin_memory()
        xh.numpy()[:] = cfg["x"]
        vh.numpy()[:] = cfg["v"]
        sysm.set_state(xh.numpy(), vh.numpy())
        sysm.step(0, args.trav, args.trunc, args.prec)   # the force of the start state
        sysm.get_forces("total", out=fh.numpy())
        k = max(3, min(args.steps, 10))
        xs, vs, fs = xh.numpy(), vh.numpy(), fh.numpy()
        for it in range(k + 2):
            if it == 2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            # state and force in, one step, state and force out (atm_step_host)
            sysm.step_host(xs, vs, fs, 1, args.trav, args.trunc, args.prec)
        dt = time.perf_counter() - t0
        e2e = {"value": n * k / dt, "unit": UNIT, "h2d_bytes_per_step": 3 * 3 * n * 8,
               "d2h_bytes_per_step": 3 * 3 * n * 8 + 72,
               "note": "atm_step_host from pinned host buffers: state (x, v) and its force in, "
                       "one velocity-Verlet step (one force evaluation), state, force and "
                       "scalars out"}
        # the same round trip through the separate calls (each synchronises)
        for it in range(k + 2):
            if it == 2:
                torch.cuda.synchronize()
                t1 = time.perf_counter()
            sysm.set_state(xs, vs)
            sysm.set_forces(fs, args.trav, args.trunc, args.prec)
            sysm.step(1, args.trav, args.trunc, args.prec)
            sysm.get_state(xs, vs)
            sysm.get_forces("total", out=fs)
        e2e["separate_calls_value"] = n * k / (time.perf_counter() - t1)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            cpu = cpu_baseline(cfg, args.trav, args.trunc, args.cpu_seconds)
        launches_per_step = prof["n_launches"] / max(1, args.steps + 1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "fp32c" else "f64", "data": "synthetic",
            "config": {"workload": "liquid N=%d rho=0.8 T=1.0 fcc+-0.05 (%s)" % (n, cfg["name"]),
                       "n": n, "box": float(cfg["box"][0]), "rc": RC, "nu": NU,
                       "traversal": args.trav, "truncation": args.trunc,
                       "precision": args.prec, "dt": 0.002, "integrator": "velocity Verlet NVE",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "launch": tuning or "default (one CTA per unit)"},
            "mups_3body": mups_3body,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(prof["n_launches"]),
            "gpu_launches_per_step": launches_per_step,
            "clocks": main["clocks"],
            "force_error": force_err,
            "profile_ms": dict({k: split["prof"][k] for k in ("ms_cells", "ms_lj", "ms_atm", "ms_md")},
                               steps=split_steps,
                               note="every launch group timed, an untimed pass after the timed steps"),
            "kernels": kernel_rooflines(split["prof"], split_steps, n, ncell_of(cfg), roofline, pk),
            "counts": {k: int(main["res"][k]) for k in ("n_cand3", "n_int3", "n_cand2", "n_int2")},
            "variants": variants,
            "surrogate": surrogate,
            "batch": batch,
            "slab": slab,
            "product_completeness": completeness,
            "paper_runtime_workload": paper_table,
        }
        print(json.dumps(line))
    sysm.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return line


# ------------------------------------------------------------------ batch

def batch_variant(atm3, device, stream, flush, count=64, steps=10, warmup=5):
    """64 replicas, N log-uniform in [500, 20000], rho in [0.1, 0.85], T in
    [0.7, 1.3] (fcc starts), 3c08 + pair + FP32C, in one context: autotuned
    ATM launch form, CUDA-graph steps, L2 flushed between timed steps."""
    import torch
    reps = synth.replicas(count=count)
    ns = [r["n"] for r in reps]
    x = np.ascontiguousarray(np.concatenate([r["x"] for r in reps], axis=1))
    v = np.ascontiguousarray(np.concatenate([r["v"] for r in reps], axis=1))
    with atm3.AtmSystem([r["box"] for r in reps], ns, rc=RC, nu=NU, dt=0.002, device=device,
                        stream=stream.cuda_stream) as b:
        b.set_state(x, v)
        b.build_cells()
        # options first: setting them resets an autotuned choice
        b.set_options(graph=True)
        tuning = b.autotune("3c08", "pair", "fp32c", reps=3)
        b.step(warmup, "3c08", "pair", "fp32c")
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(1, "3c08", "pair", "fp32c", sync=False)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in evs)
        res = b.results()
    ntot = int(sum(ns))
    # the same replicas as 64 separate contexts, each stepped with its own
    # launches (graph steps too), one after another on the same stream
    seps = []
    try:
        for r in reps:
            s = atm3.AtmSystem(r["box"], r["n"], rc=RC, nu=NU, dt=0.002, device=device,
                               stream=stream.cuda_stream)
            seps.append(s)
            s.set_state(r["x"], r["v"])
            s.set_options(graph=True)
            s.step(warmup, "3c08", "pair", "fp32c")
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s in seps:
                s.step(1, "3c08", "pair", "fp32c", sync=False)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms_sep = sum(a.elapsed_time(c) for a, c in evs)
    finally:
        for s in seps:
            s.close()
    return {"workload": "%d replicas, N log-uniform [500, 20000] (total %d), rho U(0.1, 0.85), "
                        "T U(0.7, 1.3), fcc starts" % (count, ntot),
            "traversal": "3c08", "truncation": "pair", "precision": "fp32c",
            "launch": tuning, "graph": True, "value": ntot * steps / (ms * 1e-3),
            "unit": UNIT, "ms_per_step": ms / steps,
            "n_int3": int(sum(r["n_int3"] for r in res)),
            "separate_contexts": {"ms_per_step": ms_sep / steps,
                                  "value": ntot * steps / (ms_sep * 1e-3),
                                  "note": "the same replicas in %d contexts stepped one after "
                                          "another (graph steps each)" % count}}


# ------------------------------------------------------------------ completeness

# The paper's runtime table (section 5.3): 10 iterations of the three-body
# force computation on 64 cores of an AMD EPYC 7763, per traversal and cutoff
# (seconds), for the workload below; context only (another machine and a CPU).
PAPER_RUNTIME_64C = {("3c01", "product"): 18.3553, ("3c01", "pair"): 12.7049,
                     ("3c18", "product"): 3.8193, ("3c18", "pair"): 2.5725,
                     ("3c08", "product"): 2.0499, ("3c08", "pair"): 1.3221}


def paper_table_variant(atm3, device, stream, iters=10):
    """The paper's runtime workload: N = 37,000 in a cubic box of edge 37.5
    (rho* = 0.70, 15^3 cells), simple cubic start, T* = 1.2, r_c = 2.5; for
    every traversal and cutoff, `iters` velocity-Verlet steps with the ATM
    kernel's own time of a force evaluation at each visited state (the
    paper's time counts the three-body forces only).  Three-body molecule
    updates/s = N iters / time, FP64 and FP32C, beside the paper's 64-core
    figure."""
    n, box = 37000, 37.5
    rng = np.random.default_rng(7100)
    x = synth.simple_cubic_positions(n, box, rng)
    v = synth.maxwell_boltzmann(n, 1.2, rng)
    out = {"workload": "N=37000, box 37.5 (rho 0.70, 15^3 cells), simple cubic start, T 1.2, "
                       "%d iterations" % iters, "unit": UNIT, "rows": []}
    for trav in ("3c01", "3c18", "3c08"):
        for trunc in ("product", "pair"):
            row = {"traversal": trav, "truncation": trunc}
            for prec in ("fp64", "fp32c"):
                with atm3.AtmSystem(box, n, rc=RC, nu=NU, dt=0.002, device=device,
                                    stream=stream.cuda_stream) as s:
                    s.set_state(x, v)
                    s.build_cells()
                    s.compute_forces(trav, trunc, prec)  # warm-up
                    ms = 0.0
                    for _ in range(iters):
                        s.step(1, trav, trunc, prec)
                        s.set_profiling(True)
                        s.compute_forces(trav, trunc, prec)
                        prof = s.get_profile()
                        s.set_profiling(False)
                        ms += prof["ms_atm"]
                row[prec] = {"ms_per_iteration": ms / iters,
                             "value": n * iters / (ms * 1e-3)}
            t64 = PAPER_RUNTIME_64C[(trav, trunc)]
            row["paper_64_cores"] = {"s_per_10_iterations": t64, "value": n * 10 / t64}
            out["rows"].append(row)
    return out


def completeness_variant(atm3, device, stream, workload="liquid_n32k"):
    """Product rule on the N = 32,000 liquid: interacting triplets found by the
    wide traversal (3cw: all of them, since the liquid's closest pair, about
    one sigma apart, bounds every side by 4.5 sigma, below twice the cell
    edge) and by 3c18 / 3c08, FP32C."""
    import torch
    cfg = synth.config(workload)
    out = {"workload": "liquid N=%d rho=0.8 (%s), product rule, FP32C" % (cfg["n"], workload)}
    with atm3.AtmSystem(cfg["box"], cfg["n"], rc=RC, nu=NU, device=device,
                        stream=stream.cuda_stream) as s:
        s.set_state(cfg["x"])
        s.build_cells()
        found = {}
        for trav in ("3cw", "3c18", "3c08", "3c08a"):
            s.compute_forces(trav, "product", "fp32c")
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = s.compute_forces(trav, "product", "fp32c")
            e1.record(stream)
            torch.cuda.synchronize()
            unique = r["n_int3"] // 3 if trav == "3cw" else r["n_int3"]
            found[trav] = unique
            out[trav] = {"triplets": int(unique), "e3": r["e3"], "ms": e0.elapsed_time(e1)}
        for trav in ("3c18", "3c08", "3c08a"):
            out[trav]["found_fraction"] = found[trav] / found["3cw"]
    return out


# ------------------------------------------------------------------ slab

def slab_variant(atm3, device, stream, flush, steps=20, warmup=5, nbins=600, compare_steps=500,
                 fit_equil=5000, fit_sample=5000, fit_bins=240):
    """Vapour-liquid slab: 30 x 30 x 120 box, a 30-sigma fcc liquid slab at
    rho 0.73 with vapour at rho 0.02 (random sequential insertion), T 0.85,
    3c08 + pair + FP32C; every step also adds the 600-bin histogram of z.  Then
    Eq. tanh is fitted to the profile of an NVT run from the same start, and the
    same start is run 500 steps in FP32C and in FP64 and the two density
    profiles are compared."""
    import torch
    cfg = synth.slab()
    n = cfg["n"]
    with atm3.AtmSystem(cfg["box"], n, rc=RC, nu=NU, dt=0.002, device=device,
                        stream=stream.cuda_stream) as b:
        b.set_state(cfg["x"], cfg["v"])
        b.step(warmup, "3c08", "pair", "fp32c")
        b.density_reset()
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(1, "3c08", "pair", "fp32c", sync=False)
            b.density_accumulate(axis=2, nbins=nbins)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in evs)
        counts, samples = b.density_get(nbins)
    L = cfg["box"]
    z, rho = analysis.density_profile(counts[0], samples, L)
    mid = rho[nbins // 2 - 50: nbins // 2 + 50].mean()
    edge = np.concatenate([rho[:50], rho[-50:]]).mean()
    # Eq. tanh fitted to an equilibrated profile: NVT (velocity rescaling to
    # T 0.85 every 10 steps) for fit_equil steps from the lattice start, then
    # fit_sample steps with the histogram (fit_bins bins) added every 10 steps
    fit = {"equilibration_steps": fit_equil, "sample_steps": fit_sample, "bins": fit_bins,
           "thermostat": "velocity rescaling to T 0.85 every 10 steps"}
    with atm3.AtmSystem(cfg["box"], n, rc=RC, nu=NU, dt=0.002, device=device,
                        stream=stream.cuda_stream) as b:
        b.set_state(cfg["x"], cfg["v"])
        b.set_options(graph=True)
        for k in range((fit_equil + fit_sample) // 10):
            b.step(10, "3c08", "pair", "fp32c", sync=False)
            if k >= fit_equil // 10:
                b.density_accumulate(axis=2, nbins=fit_bins)
            b.thermostat([cfg["T"]])
        c, smp = b.density_get(fit_bins)
    try:
        zf, rf = analysis.density_profile(c[0], smp, L)
        res = analysis.fit_interfaces(zf, rf, L[2])
        for side in ("left", "right"):
            fit[side] = {k: round(v, 4) for k, v in res[side].items()}
    except ImportError:
        fit = None
    # the same start run 500 steps in FP32C and in FP64 with rho(z) sampled
    # every step: the two profiles must agree to within sampling noise
    profiles = {}
    for prec in ("fp32c", "fp64"):
        with atm3.AtmSystem(cfg["box"], n, rc=RC, nu=NU, dt=0.002, device=device,
                            stream=stream.cuda_stream) as b:
            b.set_state(cfg["x"], cfg["v"])
            b.set_options(graph=True)
            for _ in range(compare_steps):
                b.step(1, "3c08", "pair", prec, sync=False)
                b.density_accumulate(axis=2, nbins=nbins)
            c, smp = b.density_get(nbins)
            profiles[prec] = analysis.density_profile(c[0], smp, L)[1]
    d = np.abs(profiles["fp32c"] - profiles["fp64"])
    # counting noise of one bin: sqrt(mean count per sample / samples) / bin volume
    bin_vol = L[0] * L[1] * L[2] / nbins
    noise = np.sqrt(np.maximum(profiles["fp64"], 1e-12) / (bin_vol * compare_steps))
    compare = {"steps": compare_steps, "max_abs_diff": float(d.max()),
               "mean_abs_diff": float(d.mean()),
               "rho_centre_fp32c": float(profiles["fp32c"][nbins // 2 - 50: nbins // 2 + 50].mean()),
               "rho_centre_fp64": float(profiles["fp64"][nbins // 2 - 50: nbins // 2 + 50].mean()),
               "max_diff_over_bin_noise": float((d / np.maximum(noise, 1e-12)).max())}
    return {"workload": "slab 30x30x120, liquid rho 0.73 (30 sigma) + vapour rho 0.02, N=%d, T 0.85"
                        % n,
            "traversal": "3c08", "truncation": "pair", "precision": "fp32c",
            "value": n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "density_bins": nbins, "density_samples": samples,
            "rho_centre": float(mid), "rho_edges": float(edge), "tanh_fit": fit,
            "fp32c_vs_fp64_profile": compare}


# ------------------------------------------------------------------ surrogate

def surrogate_observables(atm3, P, mean, scale, device, stream, steps=1000, every=10, nbins=125):
    """What the surrogate's force error costs in the observables of section 5:
    the N = 32,000 liquid stepped 'steps' velocity-Verlet steps (NVE) from the
    same state with the exact FP32C 3c08 traversal and with the surrogate
    alone; mean kinetic temperature over the second half, the total-energy
    drift of the exact run, and the pair-distance histogram g(r) sampled
    every 'every' steps over the second half (first peak, largest difference)."""
    cfg = synth.config("liquid_n32k")
    out = {"workload": "liquid N=32000 rho 0.8, %d NVE steps dt 0.002 from the same state" % steps}
    g = {}
    for mode in ("fp32c", "surrogate"):
        with atm3.AtmSystem(cfg["box"], cfg["n"], rc=RC, nu=NU, dt=0.002, device=device,
                            stream=stream.cuda_stream) as s:
            s.set_state(cfg["x"], cfg["v"])
            if mode == "surrogate":
                s.surrogate_set_model(P, mean, scale)
                s.surrogate_options(exact_every=0)
            s.step(steps // 2, "3c08", "pair", mode)
            s.rdf_reset()
            temps, etot = [], []
            for _ in range(steps // 2 // every):
                r = s.step(every, "3c08", "pair", mode)
                s.build_cells()
                s.rdf_accumulate(2.5, nbins)
                temps.append(2 * r["ekin"] / (3 * cfg["n"] - 3))
                etot.append(r["e2"] + r["e3"] + r["ekin"])
            counts, samples = s.rdf_get(nbins)
        vol = float(np.prod(cfg["box"]))
        edges = np.linspace(0.0, 2.5, nbins + 1)
        shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
        gr = counts[0] / (samples * 0.5 * cfg["n"] * (cfg["n"] / vol) * shell)
        g[mode] = gr
        k = int(np.argmax(gr))
        out[mode] = {"T_mean": float(np.mean(temps)), "g_peak_r": float(0.5 * (edges[k] + edges[k + 1])),
                     "g_peak": float(gr[k])}
        if mode == "fp32c":
            out[mode]["e_total_drift_per_molecule"] = float((etot[-1] - etot[0]) / cfg["n"])
    out["g_max_abs_diff"] = float(np.max(np.abs(g["surrogate"] - g["fp32c"])))
    return out


def train_surrogate(atm3, args, device, stream):
    """Training recipe of the surrogate: exact FP32C ATM forces (3c08, pair)
    on `sur_frames` frames each of the N=1000 and N=32,000 liquids (rho 0.8,
    T 1.0), run together as a batch of two replicas, frames `sur_stride`
    velocity-Verlet steps apart; Adam on minibatches of `sur_batch` rows,
    learning rate 2e-3 for the first half of the steps, 5e-4 after."""
    c1 = synth.config("liquid_n1000")
    c2 = synth.config("liquid_n32k")
    t0 = time.perf_counter()
    with atm3.AtmSystem([c1["box"], c2["box"]], [c1["n"], c2["n"]], rc=RC, nu=NU, dt=0.002,
                        device=device, stream=stream) as tr:
        tr.set_state(np.concatenate([c1["x"], c2["x"]], axis=1),
                     np.concatenate([c1["v"], c2["v"]], axis=1))
        tr.set_options(graph=True)
        for _ in range(args.sur_frames):
            tr.step(args.sur_stride, "3c08", "pair", "fp32c", sync=False)
            tr.surrogate_add_frame("3c08", "pair", "fp32c")
        rows, sigma2 = tr.surrogate_dataset()
        t1 = time.perf_counter()
        tr.surrogate_init(seed=1)
        h = args.sur_steps // 2
        l1 = tr.surrogate_train(h, batch=args.sur_batch, lr=2e-3, seed=2)
        l2 = tr.surrogate_train(args.sur_steps - h, batch=args.sur_batch, lr=5e-4, seed=3)
        t2 = time.perf_counter()
        P, mean, scale = tr.surrogate_get_model()
    loss = np.concatenate([l1, l2])
    tail = loss[-min(200, len(loss)):]
    info = {"frames": 2 * args.sur_frames, "rows": int(rows), "stride_steps": args.sur_stride,
            "adam_steps": args.sur_steps, "batch": args.sur_batch,
            "loss_first": float(loss[0]) if len(loss) else None,
            "loss_last200_mean": float(tail.mean()) if len(loss) else None,
            "collect_s": t1 - t0, "train_s": t2 - t1}
    return P, mean, scale, info


# ------------------------------------------------------------------ CPU oracle

def cpu_baseline(cfg, trav, trunc, seconds):
    """The oracle (linked-cell, FP64, OpenMP over units) on a bounded sample of
    units of the same workload; molecule updates/s = molecules of the sampled
    base cells / time."""
    import oracle
    prm = oracle.params(cfg["box"], RC, NU)
    cells = oracle.build_cells(prm, cfg["x"])
    occ = np.diff(cells["cell_start"])
    ncell = len(occ)
    u = 16
    t0 = time.perf_counter()
    oracle.atm_cells(prm, cfg["x"], trav, trunc, "fp64", 0, u)
    t = time.perf_counter() - t0
    while t < 0.5 and u < ncell:
        u = min(ncell, u * 4)
        t0 = time.perf_counter()
        oracle.atm_cells(prm, cfg["x"], trav, trunc, "fp64", 0, u)
        t = time.perf_counter() - t0
    per_unit = t / u
    units = int(min(ncell, max(u, seconds / max(per_unit, 1e-9))))
    t0 = time.perf_counter()
    oracle.atm_cells(prm, cfg["x"], trav, trunc, "fp64", 0, units)
    t = time.perf_counter() - t0
    mol = int(occ[:units].sum())
    return {"value": mol / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "ATM forces (%s, %s, FP64 linked-cell oracle) of the first %d of %d units "
                      "(%d molecules) of the N=%d liquid, %.1f s; LJ and integration excluded"
                      % (trav, trunc, units, ncell, mol, cfg["n"], t)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    cfg = workload(args.workload, 0)
    prm = oracle.params(cfg["box"], RC, NU)
    cells = oracle.build_cells(prm, cfg["x"])
    occ = np.diff(cells["cell_start"])
    ncell = len(occ)
    # size one step's sample to about 4 s of CPU work, less when there are
    # many steps, so that the whole run stays near two minutes
    per_step_s = min(4.0, 120.0 / max(1, args.steps))
    # the cost of one unit from two sample sizes (a call also bins all
    # molecules into cells, a fixed cost the difference cancels)
    ts = []
    for hi in (min(16, ncell), min(272, ncell)):
        t0 = time.perf_counter()
        oracle.atm_cells(prm, cfg["x"], args.trav, args.trunc, "fp64", 0, hi)
        ts.append(time.perf_counter() - t0)
    per_unit = max((ts[1] - ts[0]) / max(1, min(272, ncell) - min(16, ncell)), 1e-9)
    units = int(min(ncell, max(16, per_step_s / per_unit)))
    for _ in range(args.warmup if args.warmup < 2 else 1):
        oracle.atm_cells(prm, cfg["x"], args.trav, args.trunc, "fp64", 0, min(units, 16))
    total, mol = 0.0, 0
    for s in range(args.steps):
        lo = (s * units) % ncell
        hi = min(ncell, lo + units)
        t0 = time.perf_counter()
        oracle.atm_cells(prm, cfg["x"], args.trav, args.trunc, "fp64", lo, hi)
        total += time.perf_counter() - t0
        mol += int(occ[lo:hi].sum())
    value = mol / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "liquid N=%d rho=0.8 T=1.0 fcc+-0.05 (%s)"
                                   % (cfg["n"], cfg["name"]),
                       "n": cfg["n"], "traversal": args.trav, "truncation": args.trunc,
                       "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "per step the ATM forces of %d consecutive units of %d "
                                       "(FP64 linked-cell oracle, OpenMP)" % (units, ncell)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def kernel_case(args):
    """Repeated force evaluations of one (traversal, truncation, precision) on
    a workload, with their CUDA-event time and the ATM kernel's own time from
    the library's launch profiler.  With --prec surrogate the model is random
    (seeded) with the descriptor normalisation of the workload's descriptors."""
    import torch

    from paper_2510_21230_gb300 import atm3, build
    build.build()
    if args.train > 0:
        stream = torch.cuda.current_stream()
        c = synth.config("liquid_n1000")
        with atm3.AtmSystem(c["box"], c["n"], rc=RC, nu=NU, dt=0.002, stream=stream.cuda_stream) as s:
            s.set_state(c["x"], c["v"])
            for _ in range(20):
                s.step(10, "3c08", "pair", "fp32c")
                s.surrogate_add_frame("3c08", "pair", "fp32c")
            s.surrogate_init(seed=1)
            s.surrogate_train(2, batch=8192, lr=1e-3, seed=1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.surrogate_train(args.train, batch=8192, lr=1e-3, seed=2)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        print(json.dumps({"kernel_case": "surrogate training", "adam_steps": args.train,
                          "batch": 8192, "ms_per_step": 1e3 * dt / args.train}))
        return
    cfg = synth.homogeneous(args.n, 0.8, 1.0, seed=7000) if args.n > 0 else synth.config(args.workload)
    name = "liquid_n%d" % args.n if args.n > 0 else args.workload
    stream = torch.cuda.current_stream()
    with atm3.AtmSystem(cfg["box"], cfg["n"], rc=RC, nu=NU, stream=stream.cuda_stream) as s:
        s.set_state(cfg["x"], cfg["v"])
        s.build_cells()
        if args.prec == "surrogate":
            D, _ = s.surrogate_descriptors()
            sd = D.std(axis=0)
            s.surrogate_set_model(synth.sur_params(7), D.mean(axis=0),
                                  np.where(sd > 1e-12, sd, 1.0).astype(np.float32))
        if args.nwarps:
            s.set_options(nwarps=args.nwarps)
        if args.det:
            s.set_deterministic(True)
        s.compute_forces(args.trav, args.trunc, args.prec)
        torch.cuda.synchronize()
        s.set_profiling(True)
        times = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.reps):
                s.compute_forces(args.trav, args.trunc, args.prec, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / args.reps)
        r = s.results()[0]
        prof = s.get_profile()
    atm = prof["ms_atm"] / max(1, prof["n_atm_launches"])
    print(json.dumps({"kernel_case": name, "traversal": args.trav, "truncation": args.trunc,
                      "precision": args.prec, "deterministic": bool(args.det),
                      "ms_per_evaluation": sorted(times)[1],
                      "atm_ms_per_launch": atm, "n_int3": int(r["n_int3"]),
                      "note": "median of 3 x %d evaluations, cell build excluded" % args.reps}))


def main():
    args = parse()
    if args.kernel_case:
        kernel_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
