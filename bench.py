"""Benchmark of the FMM force solve on GB300.

A step is one pass of the whole hot path over one box of synthetic particles: Morton keys,
radix sort, radix tree, upward pass, checklist walk with local expansions, PP, PC and L2P
evaluation (fmm_compute_forces).  Partial sums are added per particle in FP64 (the paper's double
accumulation, fmm_params.accumulate = 1) unless --accumulate 0.

The default workload is the largest configuration: 512^3 particles clustered like the 4096-particle
set (half uniform, half in Plummer spheres), eps = 1/50 of the mean separation, solved with the
learned opening criterion at the rms force error of fixed theta = 0.55 (see Learned).  Other
workloads: the 128^3 NFW box (nfw2m, with a rung-0 kick-drift per step), 64 batched boxes, the
256^3 rung hierarchy, the 4096-particle set, and the 128^3 NFW box as a periodic box (periodic2m).

metric: interactions/s = (PP pairs + PC pairs) of one solve / seconds per step, over the
whole job (all ranks).  Inputs are resident in HBM when the timed region starts; the box is
larger than L2 for the tree-build phase and every step rebuilds the tree from the drifted
positions, so no state is reused across steps.  ``e2e`` repeats the measurement through
fmm_compute_forces_host with host buffers (copies inside the timed region).

With the CPU baseline (rank 0, one GPU), ``force_error`` reports one more, untimed solve of
the synthetic input against the oracle's FP64 direct sum at random sinks (rms, nearest-rank
99th percentile, maximum of the relative error); the learned workload reports its errors in its
"learned" entry instead.

``--impl reference`` times the CPU oracle (plain FP64 FMM, OpenMP) on a bounded sample of
the same workload and prints the same JSON line with "impl": "reference".

Under torchrun each rank solves an independent box (its own seed): weak scaling, no
collective on the data path; rank 0 prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# FP32 FMA peak of the part: SMs x lanes x 2 flops x max SM clock (TFLOP/s)
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
PP_FLOPS = 19.0  # FP32 flops of one PP pair in the kernel (3 sub, 3 fma, 3 mul, 3 fma, 1 add)

# DRAM bytes (read + write) of the interaction kernels with buckets of 16, groups of 64 and work
# items of 128 list entries, stored from one earlier ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of the timed solve's launch), not measured by this run, and reported
# labelled as stored only for runs with those settings; set back to None whenever a kernel changes
# after that capture.
# - the 128^3 NFW box: bytes per launch;
# - the 512^3 box: bytes per (sink, source) pair of the kernel, from the full-size fixed-theta solve
#   (k_pc 54,254,844,416 B for 31,659,347,808 PC pairs, k_pp 18,396,550,144 B for 128,335,887,451
#   PP pairs); a learned solve runs the same kernels over fewer pairs, so its traffic is that rate
#   times its own pair count.
NCU_TRAFFIC = {"k_pc": 204893440 + 52785664, "k_pp": 94600448 + 20952576}
NCU_TRAFFIC_PER_PAIR_512 = {"k_pc": 54254844416 / 31659347808, "k_pp": 18396550144 / 128335887451}
NCU_TRAFFIC_PARAMS = (16, 64, 128)

def stored_traffic(workload, n_override, tuning, kernel, stats):
    """(DRAM bytes per launch of `kernel`, where the figure comes from) for the roofline: a stored ncu
    capture for the 128^3 NFW box, a stored per-pair rate times this solve's pairs for the 512^3 box,
    both only at the captured settings; else (None, why)."""
    tun = tuning or {}
    stored = (tun.get("bucket"), tun.get("group"), tun.get("list_chunk")) == NCU_TRAFFIC_PARAMS and n_override is None
    if stored and workload == "nfw2m" and NCU_TRAFFIC and kernel in NCU_TRAFFIC:
        return (NCU_TRAFFIC[kernel],
                "stored from an earlier ncu capture of this kernel and these settings, not measured in this run")
    if stored and workload == "learned134m" and NCU_TRAFFIC_PER_PAIR_512 and kernel in NCU_TRAFFIC_PER_PAIR_512:
        pairs = int(stats.get("n_pc_pairs" if kernel == "k_pc" else "n_pp_pairs", 0) or 0)
        if pairs > 0:
            return (NCU_TRAFFIC_PER_PAIR_512[kernel] * pairs,
                    "stored: bytes per pair from an earlier ncu capture of this kernel on the fixed-theta solve of "
                    "this box at these settings, times this solve's pairs; not measured in this run")
    return None, "no ncu capture of the current kernel at these settings"


# Algorithmic DRAM bytes of the tree phase (keys, radix sort, gather, radix tree, cells, upward
# pass, exact b_max, walk nodes), the reads and writes a streaming implementation cannot avoid:
# per particle keys 40 (positions and mass in, key and index out), 8 sort passes of 24 (key and
# index in and out), gather 89 (positions and mass in; sorted FP64 positions, mass, active flag and
# the FP32 pairs out), radix tree 40 (keys in, nodes out), bucket flags 4, upward 44 (sorted
# positions and mass in, FP32 offsets out), b_max 16 (FP32 positions in); per cell 500: the cell
# arrays 20, the upward pass's centre, box, b_max, active count and 44-float record (268), and the
# walk node, centre pair and multipole norms with their inputs (212).
TREE_BYTES_PER_PARTICLE = 40 + 8 * 24 + 89 + 40 + 4 + 44 + 16
TREE_BYTES_PER_CELL = 20 + 268 + 212


def measured_peak(key, fallback):
    """A peak from MEASURED_PEAKS.json at the repository root (written by the harness that
    measured the GB300s), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="learned134m",
                    choices=["nfw2m", "plummer4096", "batch64", "rungs16m", "learned134m", "periodic2m",
                             "compressed704"])
    ap.add_argument("--accumulate", type=int, default=1, choices=[0, 1],
                    help="1: partial sums added in FP64 per particle (the paper's double accumulation)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (buckets 16, groups 64)")
    ap.add_argument("--no-graphs", action="store_true", help="solve eagerly instead of replaying a CUDA graph")
    ap.add_argument("--params", default=None, help="bucket,group,list_chunk instead of autotuning")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fixed", action="store_true",
                    help="learned134m: time the fixed-theta solve of the same box only (no training, no judge)")
    ap.add_argument("--levels", action="store_true",
                    help="add the walk's counts per level of the last timed solve (sinks, checklist entries, "
                         "largest of one sink)")
    ap.add_argument("--cpu-sample", type=float, default=None, help="active fraction of the CPU sample")
    ap.add_argument("--dual", type=int, default=None,
                    help="rungs16m: fixed rung of the dual-tree scheme (rungs <= it form the fixed tree)")
    ap.add_argument("--n", type=int, default=None,
                    help="particle count override (profiling a smaller box of the same structure)")
    return ap.parse_args()


L2_FLUSHED = "flushed before every step (256 MB write, not timed)"
L2_NOTE = {
    "batch64": "inputs and trees larger than L2 are rebuilt every step",
    "rungs16m": "inputs and tree larger than L2 are rebuilt every substep",
}


def fits_l2(n):
    """Inputs plus tree of n particles well inside the 129 MB L2 (about 64 bytes per particle)."""
    return n * 64 < (128 << 20)


def static_config(name, n=None, extra=None):
    """The workload as both arms describe it (what is solved, not how): name, size, softening,
    opening angle, accumulation, and how L2 is kept from carrying data between timed steps."""
    from paper_1609_08621_gb300 import synth

    w = synth.WORKLOADS[name]
    nn = n if n is not None else w["n"]
    eps = w["eps"] if (n is None or w["eps"] == 1e-3) else synth.paper_softening(nn)
    cfg = {"workload": name, "n": nn, "eps": eps, "theta": w["theta"],
           "l2": L2_FLUSHED if (name != "batch64" and fits_l2(nn)) else
                 L2_NOTE.get(name, "inputs and tree larger than L2 are rebuilt every step"),
           "combine": "fp64 per particle (the paper's double accumulation)"}
    if name == "periodic2m":
        cfg["nrep"] = w["nrep"]
    if name == "rungs16m":
        cfg["max_rung"] = 5
    if name == "learned134m":
        cfg["criterion"] = "learned, tau set to the rms error of fixed theta 0.55 against the FP64 direct sum"
    if name == "compressed704":
        cfg["positions"] = "3 x uint32 fixed point (x = u 2^-32), fmm_compute_forces_i32"
    if extra:
        cfg.update(extra)
    return cfg


def workload(name, rank, n=None):
    from paper_1609_08621_gb300 import synth

    w = synth.WORKLOADS[name]
    seed = w["seed"] + 1000 * rank
    if n is None:
        pos, mass = synth.make(w["kind"], w["n"], seed)
        return pos, mass, w["eps"], w["theta"]
    pos, mass = synth.make(w["kind"], n, seed)
    return pos, mass, (w["eps"] if w["eps"] == 1e-3 else synth.paper_softening(n)), w["theta"]


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons in the background during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.rows.append([x.strip() for x in ln.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 8:
                for nm, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_totals(ms, interactions, world, device):
    """Whole-job numbers of a weak-scaling run: the slowest rank's time per step (max) and the
    interactions of all ranks (sum), through torch.distributed when world > 1."""
    if world <= 1:
        return ms, interactions
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([interactions], device=device, dtype=torch.float64)
    dist.all_reduce(tot)
    return float(t.item()), float(tot.item())


def cpu_baseline(pos, mass, eps, theta, frac=None, target_s=15.0):
    """The oracle's plain FP64 FMM on a bounded sample: the full tree, forces for a random
    subset of active sinks.  Returns interactions/s over the sample."""
    import oracle

    n = mass.size
    rng = np.random.default_rng(123)
    if frac is None:
        frac = min(1.0, 4096.0 / n)
    act = (rng.random(n) < frac).astype(np.uint8)
    t0 = time.perf_counter()
    f = oracle.FMM(pos, mass, eps, theta, active=act)
    f.forces()
    dt = time.perf_counter() - t0
    c = f.counts()
    inter = c["pp_pairs"] + c["pc_pairs"]
    return {"value": inter / dt, "unit": "interactions/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"N={n} tree + walk + FP64 PP/PC/local for {int(act.sum())} random active sinks "
                      f"({frac:.4f} of N); {inter} interactions in {dt:.2f} s",
            "seconds": dt}


def error_stats(a, ref):
    """rms, nearest-rank 99th percentile and maximum of |a - ref| / |ref| over the columns."""
    e = np.sort(np.linalg.norm(np.asarray(a, np.float64) - ref, axis=0) / np.linalg.norm(ref, axis=0))
    return {"rms": float(np.sqrt(np.mean(e * e))), "p99": float(e[int(np.ceil(0.99 * e.size)) - 1]),
            "max": float(e[-1])}


def periodic_cpu_sample(pos, mass, eps, theta, frac, nrep):
    """The oracle's periodic plain FMM on a bounded sample: the full tree, the walk over the root's
    copies and the FP64 PP/PC/local/Ewald terms for a random subset of active sinks."""
    import oracle

    n = mass.size
    act = (np.random.default_rng(123).random(n) < (frac or 1024.0 / n)).astype(np.uint8)
    t0 = time.perf_counter()
    f = oracle.FMM(pos, mass, eps, theta, active=act, nrep=nrep)
    f.forces()
    dt = time.perf_counter() - t0
    c = f.counts()
    inter = c["pp_pairs"] + c["pc_pairs"]
    return {"value": inter / dt, "unit": "interactions/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"periodic N={n} tree + walk over the root's copies + FP64 PP/PC/local/Ewald for "
                      f"{int(act.sum())} random active sinks; {inter} interactions in {dt:.2f} s",
            "seconds": dt}


def force_error(pos, mass, eps, acc, nsinks=1024, seed=7):
    """Relative force error |a - a_ref| / |a_ref| of a solve's accelerations acc (3, N) against
    the oracle's FP64 direct sum at random sinks: rms, nearest-rank 99th percentile and maximum."""
    import oracle

    n = mass.size
    sinks = np.sort(np.random.default_rng(seed).choice(n, min(nsinks, n), replace=False))
    t0 = time.perf_counter()
    ref, _ = oracle.direct(pos, mass, eps, sinks)
    dt = time.perf_counter() - t0
    r = error_stats(np.asarray(acc, np.float64)[:, sinks], ref)
    r.update(sinks=int(sinks.size), reference="FP64 direct sum (oracle) of the synthetic input, %.1f s on %d threads"
             % (dt, oracle.num_threads()))
    return r


def run_reference(args, rank, world):
    """The CPU oracle as it stands, timed on the host cores on bounded samples of the workload: the
    same config as the GPU arm's line; each step is a few seconds of the oracle's plain FP64 FMM."""
    if rank != 0:
        return
    from paper_1609_08621_gb300 import synth

    if args.workload == "batch64":
        w = synth.WORKLOADS["batch64"]
        boxes, off = synth.batch_boxes(w["boxes"], w["seed"])
        b = int(np.argmax(np.diff(off)))
        pos, mass = boxes[b]
        eps, theta = w["eps"], w["theta"]
        frac = args.cpu_sample or min(1.0, 1024.0 / mass.size)
        cfg = static_config("batch64", extra={"boxes": int(w["boxes"]), "n": int(off[-1])})

        def sample():
            r = cpu_baseline(pos, mass, eps, theta, frac=frac)
            r["sample"] = f"the largest box ({b}) of the batch; " + r["sample"]
            return r
    else:
        pos, mass, eps, theta = workload(args.workload, 0, args.n)
        cfg = static_config(args.workload, args.n)
        if args.workload in ("learned134m", "compressed704"):
            def sample():
                return learned_cpu_sample(pos, mass, eps, theta, args.cpu_sample)
        else:
            frac = args.cpu_sample or min(1.0, 1024.0 / mass.size)
            nrep = synth.WORKLOADS[args.workload].get("nrep")

            def sample():
                if nrep:
                    return periodic_cpu_sample(pos, mass, eps, theta, frac, nrep)
                return cpu_baseline(pos, mass, eps, theta, frac=frac)
    steps = []
    for k in range(args.warmup + args.steps):
        r = sample()
        if k >= args.warmup:
            steps.append(r)
    v = float(np.mean([s["value"] for s in steps]))
    sec = float(np.mean([s["seconds"] for s in steps]))
    line = {"impl": "reference", "metric": "interactions/s (PP + PC) per force solve", "value": v,
            "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {k: steps[-1][k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    line["cpu_baseline"]["value"] = v
    print(json.dumps(line), flush=True)


def tune(args, ctx, tpos, tmass, eps, theta, acc, box_offsets=None, buckets=(16,)):
    """Autotune group size and work-item size (and the bucket sizes given) before the timed region;
    returns the chosen settings for the config.  --no-tune keeps buckets of 16, groups of 64."""
    if args.params:
        b, g, ch = (int(x) for x in args.params.split(","))
        ctx.set_params(bucket=b, group=g, list_chunk=ch)
        return {"bucket": b, "group": g, "list_chunk": ch, "tuned": False}
    if args.no_tune:
        ctx.set_params(bucket=16, group=64, list_chunk=0)
        return {"bucket": 16, "group": 64, "list_chunk": 64, "tuned": False}
    cands = [(b, g, ch) for b in buckets for g in (32, 48, 64) for ch in (32, 64, 128) if g >= b]
    best, ms = ctx.autotune(tpos, tmass, eps, theta, acc, candidates=cands, reps=2, box_offsets=box_offsets)
    return {"bucket": best.bucket, "group": best.group, "list_chunk": best.list_chunk, "tuned": True,
            "tuned_over": "bucket %s x group {32,48,64} x list_chunk {32,64,128}" % (list(buckets),)}


class Box:
    """One box (nfw2m, plummer4096): a step is one force solve plus one rung-0 kick-drift."""

    def __init__(self, args, rank, dev, ctx):
        import torch

        self.pos, self.mass, self.eps, self.theta = workload(args.workload, rank, args.n)
        n = self.n = self.mass.size
        self.ctx, self.dev = ctx, dev
        self.tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(dev)
        self.tmass = torch.from_numpy(self.mass).to(dev)
        self.vel = torch.zeros(3 * n, dtype=torch.float64, device=dev)
        self.acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)
        self.rung = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.act = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.dt0 = 1e-5  # tiny base step: the box barely changes, so every step solves the same workload
        self.config = static_config(args.workload, args.n)
        ctx.set_params(accumulate=args.accumulate)
        self.tuning = tune(args, ctx, self.tpos, self.tmass, self.eps, self.theta, self.acc)
        self.small = fits_l2(n)

    def step(self, k):
        self.ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)
        self.ctx.kick_drift(self.tpos, self.vel, self.acc, self.rung, self.act, self.eps, self.dt0, 0, 0,
                            1 if k > 0 else 0)

    def e2e(self, steps):
        """Through fmm_compute_forces_host: host inputs in, host results out, copies timed."""
        import torch

        hpos = torch.from_numpy(self.pos.reshape(-1).copy()).pin_memory().numpy()
        hmass = torch.from_numpy(self.mass.copy()).pin_memory().numpy()
        # the last solve's accelerations: the estimate the learned criterion reads on entry
        hacc = self.acc.cpu().pin_memory().numpy()
        hpot = torch.zeros(self.n, dtype=torch.float32).pin_memory().numpy()
        for _ in range(2):
            self.ctx.compute_forces_host(hpos, hmass, self.eps, self.theta, hacc, hpot)
        t0 = time.perf_counter()
        for _ in range(steps):
            self.ctx.compute_forces_host(hpos, hmass, self.eps, self.theta, hacc, hpot)
        dt = (time.perf_counter() - t0) / steps
        h2d = hpos.nbytes + hmass.nbytes + (hacc.nbytes if self.ctx.get_params().criterion == 1 else 0)
        return dt, int(h2d), int(hacc.nbytes + hpot.nbytes)

    def cpu_sample(self, frac):
        return cpu_baseline(self.pos, self.mass, self.eps, self.theta, frac)

    def force_error(self, nsinks=8192):
        """One more solve, outside the timed region, of the synthetic input as generated (the timed
        steps drift the particles), checked against the FP64 direct sum at random sinks (8192 of
        the 128^3 box; every particle of the 4096-particle set)."""
        import torch

        tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(self.dev)
        acc = torch.zeros_like(self.acc)
        self.ctx.compute_forces(tpos, self.tmass, self.eps, self.theta, acc, None)
        return force_error(self.pos, self.mass, self.eps, acc.cpu().numpy().reshape(3, self.n), nsinks)


class Periodic(Box):
    """The 128^3 NFW box as a periodic box (Sec. 3.1): the root's 26 copies on the checklist and the
    Ewald correction for the copies beyond; a step is one force solve."""

    def __init__(self, args, rank, dev, ctx):
        from paper_1609_08621_gb300 import synth

        args.workload = "periodic2m"
        ctx.set_params(nrep=synth.WORKLOADS["periodic2m"]["nrep"])
        super().__init__(args, rank, dev, ctx)

    def step(self, k):
        self.ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)

    def cpu_sample(self, frac):
        return periodic_cpu_sample(self.pos, self.mass, self.eps, self.theta, frac, 1)

    def force_error(self, nsinks=256):
        """One more solve of the box as generated, against the oracle's periodic FP64 direct sum (the
        softened shell, Ewald beyond it) at 256 random sinks."""
        import oracle
        import torch

        tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(self.dev)
        acc = torch.zeros_like(self.acc)
        self.ctx.compute_forces(tpos, self.tmass, self.eps, self.theta, acc, None)
        a = acc.cpu().numpy().reshape(3, self.n)
        sinks = np.sort(np.random.default_rng(7).choice(self.n, nsinks, replace=False))
        t0 = time.perf_counter()
        ref, _ = oracle.direct_periodic(self.pos, self.mass, self.eps, sinks, nrep=1)
        dt = time.perf_counter() - t0
        r = error_stats(np.asarray(a, np.float64)[:, sinks], ref)
        r.update(sinks=int(sinks.size), reference="periodic FP64 direct sum (oracle), %.1f s on %d threads"
                 % (dt, oracle.num_threads()))
        return r


class Compressed(Box):
    """704^3 = 348,913,664 particles clustered like the 4096-particle set, positions stored as
    32-bit fixed-point coordinates (Sec. 3.4: 12 bytes per particle), fixed theta = 0.55: the
    largest box the context's buffers let one GB300 hold.  A step is one fmm_compute_forces_i32."""

    def __init__(self, args, rank, dev, ctx):
        import torch

        from paper_1609_08621_gb300 import synth

        args.workload = "compressed704"
        pos, self.mass, self.eps, self.theta = workload("compressed704", rank, args.n)
        n = self.n = self.mass.size
        u = synth.to_fixed(pos)
        del pos
        self.ipos = u  # the FP64 positions the solve sees are u 2^-32 (force_error)
        self.ctx, self.dev = ctx, dev
        self.tu = torch.from_numpy(u.reshape(-1).view(np.int32)).to(dev)
        self.tmass = torch.from_numpy(self.mass).to(dev)
        self.acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)
        self.config = static_config("compressed704", args.n)
        ctx.set_params(accumulate=args.accumulate, bucket=16, group=64, list_chunk=128)
        self.tuning = {"bucket": 16, "group": 64, "list_chunk": 128, "tuned": False,
                       "note": "the bench's tuned settings of the 512^3 box (autotuning would hold a second box)"}
        self.small = False
        ctx.compute_forces_i32(self.tu, self.tmass, self.eps, self.theta, self.acc, self.pot)
        d, _ = ctx.memory_info()
        free, total = torch.cuda.mem_get_info(dev)
        self.detail = {"context_device_bytes": d, "context_bytes_per_particle": d / n,
                       "device_used_gib": (total - free) / 2 ** 30, "device_total_gib": total / 2 ** 30}

    def step(self, k):
        self.ctx.compute_forces_i32(self.tu, self.tmass, self.eps, self.theta, self.acc, self.pot)

    def e2e(self, steps):
        return None

    def cpu_sample(self, frac):
        return learned_cpu_sample(self.ipos.astype(np.float64) * (1.0 / 4294967296.0), self.mass, self.eps,
                                  self.theta, frac)

    def force_error(self, nsinks=256):
        """The last step's solve against the FP64 direct sum at 256 random sinks (about 45 s of host
        time over 3.5e8 sources)."""
        x = self.ipos.astype(np.float64) * (1.0 / 4294967296.0)
        return force_error(x, self.mass, self.eps, self.acc.cpu().numpy().reshape(3, self.n), nsinks)


class Batch:
    """64 independent boxes of N ~ U[32^3, 96^3] (Plummer-clustered): one batched solve per step."""

    def __init__(self, args, rank, dev, ctx):
        import torch

        from paper_1609_08621_gb300 import synth

        w = synth.WORKLOADS["batch64"]
        boxes, self.off = synth.batch_boxes(w["boxes"], w["seed"] + 1000 * rank)
        self.boxes = boxes
        self.pos = np.concatenate([b[0] for b in boxes], axis=1)
        self.mass = np.concatenate([b[1] for b in boxes])
        self.eps, self.theta = w["eps"], w["theta"]
        n = self.n = self.mass.size
        self.ctx, self.dev = ctx, dev
        self.tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(dev)
        self.tmass = torch.from_numpy(self.mass).to(dev)
        self.acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)
        self.config = static_config("batch64", extra={"boxes": int(w["boxes"]), "n": int(n)})
        ctx.set_params(accumulate=args.accumulate)
        self.tuning = tune(args, ctx, self.tpos, self.tmass, self.eps, self.theta, self.acc, box_offsets=self.off,
                           buckets=(8, 12, 16))

    def step(self, k):
        self.ctx.compute_forces_batch(self.tpos, self.tmass, self.off, self.eps, self.theta, self.acc, self.pot)

    def e2e(self, steps):
        """Pinned host inputs copied in and results copied out around the batched call, every step."""
        import torch

        hpos = torch.from_numpy(self.pos.reshape(-1).copy()).pin_memory()
        hmass = torch.from_numpy(self.mass.copy()).pin_memory()
        hacc = torch.zeros(3 * self.n, dtype=torch.float32).pin_memory()
        hpot = torch.zeros(self.n, dtype=torch.float32).pin_memory()

        def one():
            self.tpos.copy_(hpos, non_blocking=True)
            self.tmass.copy_(hmass, non_blocking=True)
            self.step(0)
            hacc.copy_(self.acc, non_blocking=True)
            hpot.copy_(self.pot, non_blocking=True)
            torch.cuda.current_stream(self.dev).synchronize()

        one()
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        dt = (time.perf_counter() - t0) / steps
        return dt, int(hpos.numel() * 8 + hmass.numel() * 4), int(hacc.numel() * 4 + hpot.numel() * 4)

    def cpu_sample(self, frac):
        # one box of the batch (the largest), a random subset of its particles as sinks
        b = int(np.argmax(np.diff(self.off)))
        p, m = self.boxes[b]
        return cpu_baseline(p, m, self.eps, self.theta, frac if frac else min(1.0, 4096.0 / m.size))

    def force_error(self, nsinks=4096):
        """One more batched solve of the boxes as generated, outside the timed region; the largest
        box is checked against its own FP64 direct sum at 4096 random sinks (the boxes are
        independent)."""
        import torch

        tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(self.dev)
        acc = torch.zeros_like(self.acc)
        pot = torch.zeros_like(self.pot)
        self.ctx.compute_forces_batch(tpos, self.tmass, self.off, self.eps, self.theta, acc, pot)
        b = int(np.argmax(np.diff(self.off)))
        p, m = self.boxes[b]
        a = acc.cpu().numpy().reshape(3, self.n)[:, int(self.off[b]):int(self.off[b + 1])]
        r = force_error(p, m, self.eps, a, nsinks)
        r["box"] = b
        return r


def dual_role(t, max_rung, fixed_rung):
    """Role of the force solve at substep t (counted from the run's start) under dual trees
    (Sec. 3.2) with the rungs <= fixed_rung fixed over intervals of m = 2^(max_rung - fixed_rung)
    substeps: ("full", None, None) on an interval's boundary, where the slow rungs are active as
    well; else ("dual", interval, to_mid), to_mid being the substeps from t to the interval's
    middle, where the fixed particles are drifted to."""
    m = 1 << (max_rung - fixed_rung)
    j = t % m
    if j == 0:
        return "full", None, None
    return "dual", t // m, 0.5 * m - j


class Rungs:
    """256^3 Plummer-clustered box on rungs 0-5 (Sec. 3.2): a step is one substep of the KDK
    hierarchy -- kick-drift of the active particles and drift of all, then the force solve of the
    particles active at the next substep (about 10% on average)."""

    R = 5

    def __init__(self, args, rank, dev, ctx):
        import torch

        self.pos, self.mass, self.eps, self.theta = workload("rungs16m", rank, args.n)
        n = self.n = self.mass.size
        self.ctx, self.dev = ctx, dev
        self.tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(dev)
        self.tmass = torch.from_numpy(self.mass).to(dev)
        self.vel = torch.zeros(3 * n, dtype=torch.float64, device=dev)
        self.acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)
        self.rung = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.act = torch.ones(n, dtype=torch.uint8, device=dev)
        ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)
        a = self.acc.cpu().numpy().reshape(3, n).astype(np.float64)
        dtp = 0.2 * np.sqrt(self.eps / np.maximum(np.linalg.norm(a, axis=0), 1e-30))
        # base step such that about 10% of the particles sit on the finest rung: rung R holds the
        # particles with Delta T < dt0 / 2^(R-1)
        self.dt0 = float(np.ldexp(np.quantile(dtp, 0.10), self.R - 1))
        ctx.assign_rungs(self.acc, self.rung, self.eps, self.dt0, self.R)
        hist = np.bincount(self.rung.cpu().numpy(), minlength=self.R + 1)
        self.config = static_config("rungs16m", args.n)
        self.detail = {"dt0": self.dt0, "rung_hist": hist.tolist()}
        ctx.set_params(accumulate=args.accumulate)
        self.tuning = tune(args, ctx, self.tpos, self.tmass, self.eps, self.theta, self.acc)
        ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)
        self.active_frac = []
        # dual trees (Sec. 3.2): inside each interval of 2^(R - dual) substeps only rungs > dual are
        # active; the particles of rungs <= dual are drifted to the interval's middle once and kept
        # in a fixed tree, and each inner substep solves the active particles against both trees
        self.dual = args.dual
        self.fixed_interval = None
        self.extra_launches = 0
        if self.dual is not None:
            if not 0 <= self.dual < self.R:
                raise SystemExit(f"--dual must be in [0, {self.R - 1}]")
            self.config["dual_fixed_rung"] = self.dual
            self.config["dual_interval_substeps"] = 1 << (self.R - self.dual)
            # dual trees take the fixed criterion with FP32 sums per work item as a plain solve does
            ctx.set_params(accumulate=args.accumulate)

    def step(self, k):
        s = k % (1 << self.R)
        self.ctx.kick_drift(self.tpos, self.vel, self.acc, self.rung, self.act, self.eps, self.dt0, self.R, s,
                            1 if k > 0 else 0)
        if self.dual is None:
            self.ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot, self.act)
            return
        # the substep whose forces are solved (positions are there after the drift)
        role, interval, to_mid = dual_role(k + 1, self.R, self.dual)
        if role == "full":  # interval boundary: the slow rungs are active too
            self.ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot, self.act)
            return
        if self.fixed_interval != interval:
            h = self.dt0 / (1 << self.R)
            self.ctx.set_fixed_sources(self.tpos, self.tmass, self.rung, self.dual, self.vel, to_mid * h)
            self.extra_launches += self.ctx.stats()["n_launches"]
            self.fixed_interval = interval
        self.ctx.compute_forces_dual(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot, self.act)

    def e2e(self, steps):
        return None

    def cpu_sample(self, frac):
        return cpu_baseline(self.pos, self.mass, self.eps, self.theta, frac if frac else min(1.0, 4096.0 / self.n))

    def force_error(self, nsinks=4096):
        """One more solve of the box as generated (every particle active), outside the timed region,
        against the FP64 direct sum at 4096 random sinks (about 30 s of host time over 16.8M
        sources)."""
        import torch

        tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(self.dev)
        acc = torch.zeros_like(self.acc)
        self.ctx.compute_forces(tpos, self.tmass, self.eps, self.theta, acc, None)
        return force_error(self.pos, self.mass, self.eps, acc.cpu().numpy().reshape(3, self.n), nsinks)


class Learned(Box):
    """512^3 Plummer-clustered box solved with the learned opening criterion, compared with the
    fixed criterion (theta = 0.55) at equal rms force error against the FP64 direct sum.

    Set-up, outside the timed region:
    - the oracle's FP64 direct sum at 4096 random sinks starts on the host cores in a thread (the C
      call releases the GIL) and runs while the GPU prepares;
    - the network is trained on the GPU from audit walks of the 4096-particle box, the 128^3 NFW
      box and two boxes of the 64-box batch (labels are the method's own cell-cell errors,
      normalised by each particle's acceleration from a theta = 0.3 solve);
    - a fixed-theta solve gives the acceleration estimate a time step carries over; its error
      against the direct sum sets the target, and the budget tau of the network is bisected to the
      largest value whose error does not exceed it;
    - both criteria are timed (3 solves each, CUDA events), and their errors reported.
    A step is one learned solve, with the previous step's accelerations as its estimate."""

    N_JUDGE = 4096
    force_error = None  # the line's "learned" entry reports both criteria's errors against the direct sum

    def __init__(self, args, rank, dev, ctx):
        import torch

        import oracle
        from paper_1609_08621_gb300 import synth

        args.workload = "learned134m"
        # the direct sum starts first: it is the longest part of the set-up
        self.pos, self.mass, self.eps, self.theta = workload("learned134m", rank, args.n)
        n = self.n = self.mass.size
        rng = np.random.default_rng(12345 + rank)
        self.judge_sinks = np.sort(rng.choice(n, min(self.N_JUDGE, n), replace=False))
        self._judge = {}

        def judge():
            t0 = time.perf_counter()
            self._judge["ref"] = oracle.direct(self.pos, self.mass, self.eps, self.judge_sinks)[0]
            self._judge["seconds"] = time.perf_counter() - t0

        th = threading.Thread(target=judge, daemon=True)
        th.start()
        self.ctx, self.dev = ctx, dev
        self.tpos = torch.from_numpy(self.pos.reshape(-1).copy()).to(dev)
        self.tmass = torch.from_numpy(self.mass).to(dev)
        self.acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)
        self.config = static_config("learned134m", args.n)
        self.small = False
        t0 = time.perf_counter()
        self._train(ctx, synth, dev)
        t_train = time.perf_counter() - t0
        ctx.set_params(criterion=0, accumulate=args.accumulate)
        self.tuning = tune(args, ctx, self.tpos, self.tmass, self.eps, self.theta, self.acc)
        ctx.set_params(criterion=0)
        ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)
        self.estimate = self.acc.clone()
        self.ts = torch.from_numpy(self.judge_sinks).to(dev)
        th.join()
        self.ref = self._judge["ref"]
        e_fixed = self._err(0, None)
        # tau: the largest budget whose error does not exceed the fixed criterion's
        lo, hi = -7.0, -3.5
        e_lo = self._err(1, lo)
        for _ in range(9):
            mid = 0.5 * (lo + hi)
            e = self._err(1, mid)
            if e["rms"] <= e_fixed["rms"]:
                lo, e_lo = mid, e
            else:
                hi = mid
        self.tau = lo
        t_fixed, st_fixed = self._time(0, None)
        t_learned, st_learned = self._time(1, lo)
        ctx.set_params(criterion=1, mlp_tau=self.tau)
        self.acc.copy_(self.estimate)
        margin = ctx.get_params().mlp_margin
        self.detail = {"tau": self.tau, "mlp_margin": margin}
        self.learned = {
            "error_reference": "FP64 direct sum (oracle) at %d random sinks, %.1f s on %d threads" %
                               (self.judge_sinks.size, self._judge["seconds"], oracle.num_threads()),
            "train_pairs": self.train_pairs, "train_loss": self.train_loss, "train_seconds": t_train,
            "fixed": {"theta": self.theta, "rms_err": e_fixed["rms"], "p99_err": e_fixed["p99"],
                      "ms_per_solve": t_fixed, "interactions": st_fixed["n_pp_pairs"] + st_fixed["n_pc_pairs"],
                      "n_cc": st_fixed["n_cc"], "ms_walk": st_fixed["ms_walk"]},
            "learned": {"tau": self.tau, "mlp_margin": margin, "rms_err": e_lo["rms"], "p99_err": e_lo["p99"],
                        "ms_per_solve": t_learned, "interactions": st_learned["n_pp_pairs"] + st_learned["n_pc_pairs"],
                        "n_cc": st_learned["n_cc"], "ms_walk": st_learned["ms_walk"],
                        "network_calls": st_learned["n_learned"]},
            "speedup_at_equal_error": t_fixed / t_learned if t_learned > 0 else None,
        }

    def _train(self, ctx, synth, dev):
        import torch

        sets = []
        w1 = synth.WORKLOADS["plummer4096"]
        sets.append(synth.make("plummer", w1["n"], w1["seed"]) + (w1["eps"], w1["theta"]))
        w2 = synth.WORKLOADS["nfw2m"]
        sets.append(synth.make("nfw", w2["n"], w2["seed"]) + (w2["eps"], w2["theta"]))
        w3 = synth.WORKLOADS["batch64"]
        boxes, _ = synth.batch_boxes(w3["boxes"], w3["seed"])
        for b in boxes[:2]:
            sets.append(tuple(b) + (w3["eps"], w3["theta"]))
        fs, ls = [], []
        for p, m, eps, theta in sets:
            n = m.size
            tp = torch.from_numpy(np.ascontiguousarray(p).reshape(-1)).to(dev)
            tm = torch.from_numpy(m).to(dev)
            ref = torch.zeros(3 * n, dtype=torch.float32, device=dev)
            ctx.set_params(criterion=0)
            ctx.compute_forces(tp, tm, eps, 0.3, ref)
            f, l = ctx.mlp_audit(tp, tm, eps, theta, 0.35, 1.0, ref, 4 * n + 4096)
            fs.append(f.clone())
            ls.append(l.clone())
        feats, labels = torch.cat(fs).contiguous(), torch.cat(ls).contiguous()
        self.train_pairs = int(labels.numel())
        self.train_loss = ctx.mlp_train(feats, labels, epochs=10, batch=4096, lr=4e-3, seed=1)

    def _solve(self, criterion, tau):
        if criterion == 1:
            self.ctx.set_params(criterion=1, mlp_tau=tau)
        else:
            self.ctx.set_params(criterion=0)
        self.acc.copy_(self.estimate)  # the estimate a time step carries over
        self.ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)

    def _err(self, criterion, tau):
        self._solve(criterion, tau)
        a = self.acc.view(3, self.n).index_select(1, self.ts).double().cpu().numpy()
        return error_stats(a, self.ref)

    def _time(self, criterion, tau, reps=3):
        import torch

        self._solve(criterion, tau)
        s = torch.cuda.current_stream(self.dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            self._solve(criterion, tau)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, self.ctx.stats()

    def step(self, k):
        self.ctx.compute_forces(self.tpos, self.tmass, self.eps, self.theta, self.acc, self.pot)

    def cpu_sample(self, frac):
        return learned_cpu_sample(self.pos, self.mass, self.eps, self.theta, frac)


def learned_cpu_sample(pos, mass, eps, theta, frac=None, k=1 << 20):
    """The oracle (fixed theta) on a random 2^20-particle subset of the 512^3 box, masses rescaled to
    a total of 1: the full tree alone would take the host minutes."""
    n = mass.size
    k = min(n, k)
    idx = np.sort(np.random.default_rng(7).choice(n, k, replace=False))
    m = (mass[idx].astype(np.float64) * (n / k)).astype(np.float32)
    r = cpu_baseline(np.ascontiguousarray(pos[:, idx]), m, eps, theta, frac if frac else min(1.0, 1024.0 / k))
    r["sample"] = f"random {k}-particle subset of the box; " + r["sample"]
    return r


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    from paper_1609_08621_gb300 import binding

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(local, stream)
    kind = {"batch64": Batch, "rungs16m": Rungs, "learned134m": Learned, "periodic2m": Periodic,
            "compressed704": Compressed}.get(args.workload, Box)
    if args.fixed and args.workload == "learned134m":
        kind = Box  # the same box and settings, fixed theta only (a profiling aid: no judge, no baseline)
        args.no_cpu_baseline = True
    wl = kind(args, rank, dev, ctx)
    if kind is Box and args.workload == "learned134m":
        wl.config["criterion"] = "fixed theta 0.55 only (--fixed)"
    ctx.set_graphs(not args.no_graphs)
    wl.tuning["cuda_graph"] = not args.no_graphs

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for k in range(args.warmup):
        wl.step(k)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kt = {"pp": 0.0, "pc": 0.0, "tree": 0.0, "walk": 0.0, "l2p": 0.0}
    flops = {"pp": 0.0, "pc": 0.0}
    inter = []
    launches = 0
    retries = 0
    active = []
    # workloads smaller than L2 get L2 flushed (a 256 MB write, outside the step's events) before
    # every step; larger ones rebuild a tree bigger than L2 each step
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if getattr(wl, "small", False) else None
    step_ms = []
    e0.record(stream)
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        wl.step(args.warmup + k)
        s1.record(stream)
        step_ms.append((s0, s1))
        st = ctx.stats()
        for key in kt:
            kt[key] += st["ms_" + key]
        flops["pp"] += st["kernel_flops_pp"]
        flops["pc"] += st["kernel_flops_pc"]
        inter.append(st["n_pp_pairs"] + st["n_pc_pairs"])
        retries += st["retries"]
        active.append(st["n_active"])
        launches += st["n_launches"] + (1 if args.workload != "batch64" else 0) + getattr(wl, "extra_launches", 0)
        if hasattr(wl, "extra_launches"):
            wl.extra_launches = 0
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if flush is not None:
        ms = float(np.mean([a.elapsed_time(b) for a, b in step_ms]))
    inter_mean = float(np.mean(inter))
    ms, inter_job = job_totals(ms, inter_mean, world, dev)
    value = inter_job / (ms * 1e-3)
    st = ctx.stats()
    # roofline of the dominant interaction kernel (FP32 ALU bound), CUDA events on the context's stream
    pp_ms, pc_ms = kt["pp"] / args.steps, kt["pc"] / args.steps
    fpp, fpc = flops["pp"] / args.steps, flops["pc"] / args.steps
    dom = "k_pc" if pc_ms >= pp_ms else "k_pp"
    dom_ms, dom_flops = (pc_ms, fpc) if dom == "k_pc" else (pp_ms, fpp)
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS,
            "traffic": None,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
            "pp_pc_frac": ((fpp + fpc) / ((pp_ms + pc_ms) * 1e-3) / 1e12) / FP32_PEAK_TFLOPS
            if pp_ms + pc_ms > 0 else 0.0}
    roof["traffic"], roof["traffic_source"] = stored_traffic(args.workload, args.n, getattr(wl, "tuning", None), dom, st)
    # the tree phase against the HBM roofline (algorithmic bytes; CUDA events of the phase)
    hbm, hbm_src = measured_peak("hbm_gbs", 6800.0)
    tree_ms = kt["tree"] / args.steps
    n_tree = int(wl.config.get("n", 0) or 0)
    tree_bytes = TREE_BYTES_PER_PARTICLE * n_tree + TREE_BYTES_PER_CELL * int(st["n_cells"])
    tree_gbs = tree_bytes / (tree_ms * 1e-3) / 1e9 if tree_ms > 0 else 0.0
    tree_hbm = {"bound": "hbm", "bytes": tree_bytes, "ms": tree_ms, "achieved": tree_gbs, "peak": hbm,
                "unit": "GB/s", "frac": tree_gbs / hbm, "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_particle": TREE_BYTES_PER_PARTICLE, "bytes_per_cell": TREE_BYTES_PER_CELL}
    line = {"metric": "interactions/s (PP + PC) per force solve", "value": value, "unit": "interactions/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": wl.config, "tuning": wl.tuning, "detail": getattr(wl, "detail", {}),
            "phase_ms": {k: v / args.steps for k, v in kt.items()},
            "interactions_per_step": inter_job, "n_pp_pairs": st["n_pp_pairs"], "n_pc_pairs": st["n_pc_pairs"],
            "n_cc": st["n_cc"], "n_cp": st["n_cp"], "n_groups": st["n_groups"], "n_levels": st["n_levels"],
            "active_per_step": float(np.mean(active)), "walk_retries": retries, "roofline": roof,
            "tree_hbm": tree_hbm, "tree_hbm_frac": tree_hbm["frac"], "clocks": ck,
            "gpu_launches": launches}
    if args.levels:
        line["walk_levels"] = [[int(v) for v in row] for row in ctx.export_walk_levels()]
    if hasattr(wl, "learned"):
        line["learned"] = wl.learned
    if not args.no_e2e:
        barrier()
        r = wl.e2e(args.steps)
        if r is not None:
            dt, hb, db = r
            dt, _ = job_totals(dt, 0.0, world, dev)
            line["e2e"] = {"value": inter_job / dt, "unit": "interactions/s", "ms_per_step": dt * 1e3,
                           "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in wl.cpu_sample(args.cpu_sample).items() if k != "seconds"}
        fe = getattr(wl, "force_error", None)
        if fe is not None:
            try:
                line["force_error"] = fe()
            except Exception as ex:  # the accuracy report is auxiliary: keep the line
                line["force_error"] = {"error": repr(ex)}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
