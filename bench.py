"""Benchmark: RelRes vs FG-only Lennard-Jones MD on one GB300 (atom-steps/s).

Workload: neopentane-like liquid, 200 000 molecules = 1 000 000 united atoms
(central C hybrid + 4 CH3), 0.58 g/cm^3 (L = 345.7 A), RelRes radii r_s 6-7 A,
r_c 13-14 A, CG parameters from the multipole sum rule, skin 2 A, FP32 pair
terms with FP64 totals and integration, dt = 2 fs, CSVR thermostat at 260 K.
A step is one full velocity-Verlet step: drift, rebuild check (and rebuild when
an atom moved more than skin/2), RelRes pair forces over the FG and CG lists,
bonded terms, kinetic energy and thermostat.

The same system is then run as the plain FG reference (LJ smoothed to zero
over [13, 14) A, no CG term) for the speedup; and the oracle (FP64, O(N^2)) is
timed on a bounded sample of the same workload on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s RelRes vs FG-only LJ (same GB300, 1M atoms); pair-kernel % roofline"
FALLBACK_HBM_GBS = 6800.0
PAIR_SRC = os.path.join(ROOT, "paper_2104_10231_gb300", "csrc", "pair.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pair_neopentane_1M.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-mol", type=int, default=200_000)
    ap.add_argument("--equil", type=int, default=200, help="untimed equilibration steps")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the step kernels one by one on the stream instead of CUDA graphs "
                         "(same kernels; ncu cannot list kernels inside graphs with conditional nodes)")
    ap.add_argument("--thermo-every", type=int, default=100,
                    help="energy/virial/temperature row every this many timed steps (0: none)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-fg-only", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiable (backward) leg")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the full-step timings of the two small systems (GPU and oracle)")
    ap.add_argument("--batch-replicas", type=int, default=128,
                    help="replicas of the batched leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--prune", type=float, default=0.5,
                    help="pruning margin of the neighbour lists in Angstrom (0: pair kernels walk the full lists)")
    ap.add_argument("--pair-config", type=int, default=-1,
                    help="fix the pair-kernel launch configuration (0..6) instead of autotuning")
    ap.add_argument("--force-acc", type=int, default=-1,
                    help="per-atom pair-force sums: 0 FP32, 1 compensated float-float, 2 FP64 "
                         "(default: the library's)")
    return ap.parse_args()


def workload_config(args, n_atoms, box):
    return {
        "workload": (f"neopentane-like liquid, {args.n_mol} molecules ({n_atoms} atoms), "
                     f"L={box:.2f} A, RelRes r_s 6-7 A / r_c 13-14 A, CG by Eq. 13 sum rule, "
                     "skin 2 A, dt 2 fs, CSVR 260 K"),
        "n_atoms": n_atoms,
        "precision": "FP32 pair terms from exact fixed-point differences; FP64 totals, "
                     "velocities; 64-bit fixed-point positions",
        "l2": "inputs larger than L2 (neighbour lists ~0.5 GB, state 64 MB)",
        "parallelism": "replicas only (one independent system per GPU)",
        "thermo_every": args.thermo_every,
        "execution": "stream launches" if args.no_graphs else "CUDA graph per 100 steps, conditional rebuild node",
        "lists": (f"rebuilt at skin/2 = 1 A displacement; pair kernels walk lists pruned to the cutoff + "
                  f"{args.prune} A, re-pruned at {args.prune / 2} A displacement") if args.prune > 0 else
                 "rebuilt at skin/2 = 1 A displacement; pair kernels walk the full lists",
        "seed": 2104,
    }


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


COUNTER_ATOMS = 1_000_000  # the summary's counters are scaled to the 1M-atom workload


def recorded_pair_counters(p_prune, n_atoms):
    """ncu counters of one pair-kernel launch from the committed summary, if
    it was taken on the current pair.cu (sha256 prefix recorded there) and the
    run is the workload they were scaled to: DRAM bytes and warp instructions
    executed, each the mean over plain launches and pruning launches (a
    fraction p_prune)."""
    out = {}
    if n_atoms != COUNTER_ATOMS:
        return out
    try:
        src_sha = hashlib.sha256(open(PAIR_SRC, "rb").read()).hexdigest()[:16]
        vals = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("pair_cu_sha256_16") != src_sha:
            return out
        for key, name in (("dram_bytes", "dram_bytes_%s_launch_full_size"),
                          ("inst_executed", "inst_executed_%s_launch_full_size")):
            if name % "plain" in vals and name % "pruning" in vals:
                out[key] = ((1.0 - p_prune) * float(vals[name % "plain"]) +
                            p_prune * float(vals[name % "pruning"]))
    except Exception:
        pass
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region.  A region
    shorter than the 200 ms sampling period may hold no sample: then the
    samples on both sides of it (the last before, the first after) stand for
    it, and the summary says so."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []  # (time read, csv line)
        self.t_start = self.t_end = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi's start-up (driver and NVML initialisation) delays this
            # process's own driver calls for tens of milliseconds: the timed
            # region starts after its first sample, once it only samples
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 10.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t_start = time.perf_counter()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *exc):
        self.t_end = time.perf_counter()
        if self.proc:
            # a region without a sample of its own: wait for the one after it
            t0 = time.perf_counter()
            while (not any(self.t_start <= t for t, _ in self.lines) and self.proc.poll() is None
                   and time.perf_counter() - t0 < 2.0):
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        inside = [ln for t, ln in self.lines if self.t_start <= t <= self.t_end]
        window = "samples inside the timed region"
        if not inside:
            before = [ln for t, ln in self.lines if t < self.t_start][-1:]
            after = [ln for t, ln in self.lines if t > self.t_end][:1]
            inside = before + after
            window = ("the samples just before and just after the timed region (shorter than the "
                      "200 ms sampling period)")
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


_THERMO = {}


def max_over_ranks(dist, secs, device="cuda"):
    """The largest of the ranks' times (every rank gets it); secs when not distributed."""
    if dist is None:
        return secs
    import torch

    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, secs_max):
    """Units processed by all ranks per second of the slowest rank (replicas:
    every rank advances its own system of units_per_rank atoms)."""
    return world * units_per_rank * steps / secs_max


def run_md_timed(torch, R, ctx, pos, vel, steps, dt, t_target, seed, thermo_every):
    """K steps of relres_step bracketed by CUDA events on the context stream,
    with a thermo row (energies, virial, temperature) every `thermo_every`
    steps.  The thermo buffer is kept per context, so that a warm-up call with
    the same arguments leaves the captured step graph in place."""
    stream = ctx.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rows = max(1, 100000 // thermo_every) if thermo_every > 0 else 1
    key = id(ctx)
    if key not in _THERMO:
        _THERMO[key] = torch.zeros((rows, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
    thermo = _THERMO[key]
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(steps, dt, pos, vel, t_target=t_target, tau_fs=100.0, seed=seed,
             thermo_every=thermo_every if thermo_every > 0 else 0, d_thermo=thermo)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def ours(args):
    import numpy as np
    import torch

    from paper_2104_10231_gb300 import relres as R
    from paper_2104_10231_gb300 import systems as S
    from paper_2104_10231_gb300.build import build_library

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        build_library()
    if dist:
        dist.barrier()
    R.load()

    # rates of this GPU (probe kernels of the library): FLOP side of the roofline
    scratch = torch.empty(2 << 30, dtype=torch.uint8, device="cuda")
    rates = R.relres_measure_rates(scratch)
    del scratch
    torch.cuda.empty_cache()

    s = S.neopentane(n_mol=args.n_mol, seed=2104 + rank, temperature=260.0)
    n = s.n_atoms
    dt, temp = 2.0, 260.0
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s), stream=stream)
        ctx.set_graphs(not args.no_graphs)
        ctx.set_pair_config(args.pair_config)
        if args.force_acc >= 0:
            ctx.set_force_accumulation(args.force_acc)
        ctx.set_prune(args.prune)
        pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        vel = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
        ctx.build_neighbors(pos, s.box)
        # untimed: relax the lattice start, then warm up
        if args.equil:
            ctx.step(args.equil, dt, pos, vel, t_target=temp, tau_fs=100.0, seed=7)
        ctx.step(args.warmup, dt, pos, vel, t_target=temp, tau_fs=100.0, seed=8)
        # the timed call, untimed once: every block shape it runs (blocks of 100
        # steps and the remainder) is captured and instantiated here, so no graph
        # capture falls inside the timed region
        ctx.set_timing(False)
        run_md_timed(torch, R, ctx, pos, vel, args.steps, dt, temp, 9, args.thermo_every)
        st0 = ctx.stats()
        if dist:
            dist.barrier()
        with ClockSampler(local) as clk:
            secs = run_md_timed(torch, R, ctx, pos, vel, args.steps, dt, temp, 9, args.thermo_every)
        st1 = ctx.stats()
        # roofline pass: every forces-only pair launch of ROOF_STEPS further steps
        # timed with CUDA events (no energy steps, so every launch is of that
        # class); the bytes are weighted by the pruning launches of the same pass
        roof = pair_pass(torch, R, ctx, pos, vel, dt, temp)
        # every kernel class timed on every step: a separate, shorter run
        ctx.set_timing(True)
        run_md_timed(torch, R, ctx, pos, vel, min(200, args.steps), dt, temp, 10, args.thermo_every)
        tim = ctx.timings()
        ctx.set_timing(False)
        secs = max_over_ranks(dist, secs)
        if dist:
            dist.barrier()

        # end to end through the C ABI with host buffers: per step, copy the
        # state in from pinned host memory, one relres_step, copy the new state
        # (the step's result) out
        hp = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hv = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hp.copy_(pos.cpu())
        hv.copy_(vel.cpu())
        ke = max(1, args.e2e_steps)
        ctx.step(1, dt, pos, vel, t_target=temp, tau_fs=100.0, seed=10)  # one-step graph captured here
        torch.cuda.synchronize()
        # positions and velocities travel on two streams (two copy engines)
        side = torch.cuda.Stream()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            side.wait_stream(stream)
            pos.copy_(hp, non_blocking=True)
            with torch.cuda.stream(side):
                vel.copy_(hv, non_blocking=True)
            stream.wait_stream(side)
            ctx.step(1, dt, pos, vel, t_target=temp, tau_fs=100.0, seed=10)
            side.wait_stream(stream)
            hp.copy_(pos, non_blocking=True)
            with torch.cuda.stream(side):
                hv.copy_(vel, non_blocking=True)
            stream.wait_stream(side)
        torch.cuda.synchronize()
        e2e_secs = max_over_ranks(dist, time.perf_counter() - t0)
        e2e_value = whole_job_rate(world, n, ke, e2e_secs)

    value = whole_job_rate(world, n, args.steps, secs)
    ms_step = secs / args.steps * 1e3

    # FG-only reference on the same configuration
    fg = None
    if not args.no_fg_only:
        sf = S.fg_only(s)
        with torch.cuda.stream(stream):
            ctxf = R.Context(R.params_for(sf, R.RELRES_PREC_FP32), R.topology_for(sf), stream=stream)
            ctxf.set_graphs(not args.no_graphs)
            if args.force_acc >= 0:
                ctxf.set_force_accumulation(args.force_acc)
            ctxf.set_prune(args.prune)
            posf = pos.clone()
            velf = vel.clone()
            ctxf.build_neighbors(posf, s.box)
            ctxf.step(args.warmup, dt, posf, velf, t_target=temp, tau_fs=100.0, seed=8)
            run_md_timed(torch, R, ctxf, posf, velf, args.steps, dt, temp, 9, args.thermo_every)  # captures
            if dist:
                dist.barrier()
            secs_f = run_md_timed(torch, R, ctxf, posf, velf, args.steps, dt, temp, 9, args.thermo_every)
            secs_f = max_over_ranks(dist, secs_f)
            roof_f = pair_pass(torch, R, ctxf, posf, velf, dt, temp)
            stf = ctxf.stats()
            ctxf.close()
        fg = {"value": whole_job_rate(world, n, args.steps, secs_f), "ms_per_step": secs_f / args.steps * 1e3,
              "long_run_ms_per_step": roof_f["ms_per_step"],
              "pair_ms_per_launch": roof_f["ms_per_launch"], "pair_launches_timed": roof_f["launches"],
              "pruning_launch_fraction": roof_f["p_prune"],
              "mean_list": stf["mean_fg"], "mean_list_pruned": roof_f["mean_fg_walked"], "rebuilds": stf["n_builds"]}
    ctx_stats = st1
    ctx.close()

    # roofline of the dominant kernel: the RelRes pair kernel (FG and CG lists,
    # one launch) as it runs on every step that needs no energy
    n_h = ctx_stats["n_hybrid"]
    prunes = ctx_stats["n_prunes"] - st0["n_prunes"]
    full = ctx_stats["mean_fg"] * n + ctx_stats["mean_cg"] * n_h
    walked = roof["mean_fg_walked"] * n + roof["mean_cg_walked"] * n_h
    pair_ms = roof["ms_per_launch"]
    p_prune = roof["p_prune"]
    alg_bytes = pair_alg_bytes(n, n_h, roof["mean_fg_full"] * n + roof["mean_cg_full"] * n_h, walked, p_prune)
    clk_sum = clk.summary()
    roofline = pair_roofline(alg_bytes, pair_ms, p_prune, peaks(), rates, clk_sum, n, n_h, walked,
                             roof["mean_fg_full"] * n + roof["mean_cg_full"] * n_h, float(s.box[0]) ** 3)
    roofline["launches_timed"] = roof["launches"]
    kernel_ms = {k: round(v[0] / max(1, v[1]), 5) for k, v in tim.items()}
    kernel_share = {k: round(v[0] / max(1e-12, sum(x[0] for x in tim.values())), 4) for k, v in tim.items()}

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "atom-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded neopentane-like liquid; the paper's systems are not available)",
        "config": workload_config(args, n, float(s.box[0])),
        "ns_per_day": dt * 1e-6 * (args.steps / secs) * 86400.0,
        "fg_only": fg,
        "speedup_vs_fg_only": (value / fg["value"]) if fg else None,
        "eq21": efficiency_eq21(fg, pair_ms, ms_step, full / n, walked / n) if fg else None,
        "roofline": roofline,
        "kernel_ms_per_launch": kernel_ms,
        "kernel_time_share": kernel_share,
        "kernel_breakdown_run": f"{min(200, args.steps)} further steps with every kernel class timed (events slow "
                                "the steps by ~8 %, so the headline run records no events inside its steps)",
        "lists": {"mean_fg": ctx_stats["mean_fg"], "mean_cg": ctx_stats["mean_cg"],
                  "cap_fg": ctx_stats["cap_fg"], "cap_cg": ctx_stats["cap_cg"],
                  "rebuilds_in_timed_region": ctx_stats["n_builds"] - st0["n_builds"],
                  "rebuild_ms_per_step": kernel_ms.get("rebuild"),
                  "rebuild_share_of_step": kernel_share.get("rebuild"),
                  "rebuilds_per_step_long_run": roof["rebuilds"] / ROOF_STEPS,
                  "long_run_context": {"steps": ROOF_STEPS, "ms_per_step": roof["ms_per_step"],
                                       "rebuilds": roof["rebuilds"],
                                       "how": "the same system continued for ROOF_STEPS steps after the timed "
                                              "region, CUDA events around the call, a CUDA-event pair around "
                                              "every pair launch (no energy steps); a short timed region holds "
                                              "0 or 1 list rebuilds, this one the long-run share"},
                  "prune_delta": ctx_stats["prune_delta"], "prunes_in_timed_region": prunes,
                  "mean_fg_walked": roof["mean_fg_walked"], "mean_cg_walked": roof["mean_cg_walked"]},
        "pair_launch": {"threads_per_atom": ctx_stats["pair_tpa"], "block": ctx_stats["pair_block"],
                        "chosen_by": "autotuner (first relres_step)",
                        "force_accumulation": ["FP32", "compensated float-float", "FP64"][ctx_stats["force_acc"]]},
        "gpu_launches": ctx_stats["n_launches"] - st0["n_launches"],
        "device_rates": {k: (round(v, 2) if isinstance(v, float) else v) for k, v in rates.items()},
        "clocks": clk_sum,
        "e2e": {"value": e2e_value, "unit": "atom-steps/s", "h2d_bytes_per_step": 2 * 24 * n,
                "d2h_bytes_per_step": 2 * 24 * n,
                "steps": ke, "how": "relres_step(1) per step with H2D/D2H of positions+velocities (pinned; the two "
                                    "arrays on two streams)"},
    }
    if not args.no_diff:
        out["differentiable"] = differentiable_leg(torch, R, S, stream)
    if args.batch_replicas > 0:
        out["batched"] = batched_leg(torch, R, S, args.batch_replicas, args.batch_steps)
        out["batched_small"] = small_batch_leg(torch, R, S, args.batch_replicas, args.batch_steps)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(s, args.cpu_seconds)
    if rank == 0 and world == 1 and not args.no_small:
        out["small_systems"] = small_systems_leg(torch, R, S, with_oracle=not args.no_cpu)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


ROOF_STEPS = 300


def pair_pass(torch, R, ctx, pos, vel, dt, temp, steps=ROOF_STEPS):
    """ROOF_STEPS MD steps with a CUDA-event pair around every forces-only pair
    launch (no energy steps).  The launches that prune (rebuild or pruning
    trigger) walk the full lists, the others the pruned lists of the last
    pass; the pass reports the mean time per launch, the fraction of pruning
    launches and the list sizes of the same launches."""
    st_a = ctx.stats()
    ctx.set_timing_sampled(["pair"], 1)
    secs = run_md_timed(torch, R, ctx, pos, vel, steps, dt, temp, 11, 0)
    tim = ctx.timings()
    st_b = ctx.stats()
    ctx.set_timing(False)
    prunes = st_b["n_prunes"] - st_a["n_prunes"]
    if st_b["prune_delta"] > 0 and prunes > 0:
        mfg = (st_b["mean_fg_pruned"] * st_b["n_prunes"] - st_a["mean_fg_pruned"] * st_a["n_prunes"]) / prunes
        mcg = (st_b["mean_cg_pruned"] * st_b["n_prunes"] - st_a["mean_cg_pruned"] * st_a["n_prunes"]) / prunes
        p_prune = prunes / steps
    else:
        mfg, mcg, p_prune = st_b["mean_fg"], st_b["mean_cg"], 0.0
    launches = tim["pair"][1]
    return {"ms_per_launch": tim["pair"][0] / max(1, launches), "launches": launches, "p_prune": p_prune,
            "mean_fg_walked": mfg, "mean_cg_walked": mcg, "mean_fg_full": st_b["mean_fg"],
            "mean_cg_full": st_b["mean_cg"], "rebuilds": st_b["n_builds"] - st_a["n_builds"],
            "ms_per_step": secs / steps * 1e3}


def pair_alg_bytes(n, n_h, full, walked, p_prune):
    """Algorithmic bytes of one forces-only pair launch, the mean over plain
    launches (pruned lists: 4 B index + 16 B gathered position per entry; per
    slot 16 B own position, 4 B count, 4 B slot map, 16 B force) and pruning
    launches (full lists, plus 4 B per kept entry, 4 B per slot count and
    16 B per atom of the pruning reference)."""
    alg_plain = walked * 20.0 + (n + n_h) * 40.0
    alg_prune = full * 20.0 + walked * 4.0 + (n + n_h) * 44.0 + n * 16.0
    return (1.0 - p_prune) * alg_plain + p_prune * alg_prune


def pair_roofline(alg_bytes, pair_ms, p_prune, peak_info, rates, clk, n, n_h, walked, full, vol):
    """Roofline record of the pair kernel.  frac: algorithmic bytes over HBM
    copy bandwidth (gathers are L1/L2 hits, so it can pass 1); dram_frac:
    measured DRAM bytes per launch over the same peak; issue_frac: warp
    instructions per launch over the issue peak (one per clock per scheduler,
    4 per SM); flop_side: FP32 FLOPs over the FFMA peak."""
    peak, peak_kind = peak_info
    secs = pair_ms * 1e-3
    achieved = alg_bytes / secs / 1e9
    rec = recorded_pair_counters(p_prune, n)
    traffic = rec.get("dram_bytes")
    insts = rec.get("inst_executed")
    mhz = (clk or {}).get("sm_mhz") or rates.get("clock_mhz")
    sms = rates.get("sm_count") or 152
    pairs_in = (4.0 * math.pi / 3.0) * (7.0 ** 3 * n * n / vol + 14.0 ** 3 * n_h * n_h / vol)
    walked_entries = (1.0 - p_prune) * walked + p_prune * full
    flops = 10.0 * walked_entries + 30.0 * pairs_in
    flop_side = {"flops_per_launch": flops, "achieved_tflops": flops / secs / 1e12,
                 "fp32_peak_tflops": rates["fp32_tflops"],
                 "frac": flops / secs / 1e12 / rates["fp32_tflops"],
                 "peak_source": "measured here (FFMA probe, relres_measure_rates)"}
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_source": peak_kind + " (hbm_gbs, copy)",
           "kernel": "k_pair<float, forces only> (FG + CG lists)",
           "alg_bytes_per_launch": alg_bytes, "ms_per_launch": pair_ms, "pruning_launch_fraction": p_prune,
           "how": "frac = alg_bytes_per_launch / (ms_per_launch * 1e-3) / 1e9 / peak; every forces-only pair "
                  "launch of a separate 300-step pass timed with CUDA events on the context stream, bytes "
                  "weighted by that pass's pruning launches (full lists) and plain launches (pruned lists)",
           "flop_side": flop_side}
    if traffic is not None:
        out["dram_frac"] = traffic / secs / 1e9 / peak
        out["dram_how"] = ("traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, plain and "
                           "pruning launches weighted alike) / (ms_per_launch * 1e-3) / 1e9 / peak")
    if insts is not None and mhz:
        out["issue_frac"] = insts / (secs * mhz * 1e6 * sms * 4)
        out["inst_executed_per_launch"] = insts
        out["issue_how"] = (f"inst_executed_per_launch (ncu smsp__inst_executed.sum) / (ms_per_launch * 1e-3 * "
                            f"{mhz:.0f} MHz * {sms} SMs * 4 schedulers)")
    return out


def efficiency_eq21(fg, pair_ms, step_ms, entries_full, entries_walked):
    """The paper's efficiency analysis (Section 2.6): the pair-time speedup
    against the FG reference, eta~* = 1 / tau~*, set beside 1 / N* (Eq. 21),
    N* the RelRes list size over the reference's, per atom; and the total
    speedup eta*_tot beside chi / N* (Eq. 22), which gives chi.  N* is given
    for the lists with the skin (the paper's list size) and for the pruned
    lists the pair kernel walks."""
    try:
        n_full = entries_full / fg["mean_list"]
        n_walked = entries_walked / fg["mean_list_pruned"]
        eta_pair = fg["pair_ms_per_launch"] / pair_ms
        eta_tot = fg["ms_per_step"] / step_ms
        return {"n_star_lists": round(n_full, 4), "n_star_walked": round(n_walked, 4),
                "one_over_n_star_lists": round(1.0 / n_full, 3), "one_over_n_star_walked": round(1.0 / n_walked, 3),
                "eta_pair": round(eta_pair, 3), "eta_pair_times_n_star_walked": round(eta_pair * n_walked, 3),
                "eta_tot": round(eta_tot, 3), "chi_walked": round(eta_tot * n_walked, 3)}
    except (KeyError, TypeError, ZeroDivisionError):
        return None


def small_systems_leg(torch, R, S, with_oracle=True):
    """Full MD steps of the two small systems the parity tests use: 216
    propane-like molecules (648 atoms, FP64, NVE, dt 1 fs) and 4000
    neopentane-like molecules (20 000 atoms, FP32, CSVR 260 K, dt 2 fs), on
    the GPU (CUDA events around relres_step) and, for the same systems, the
    oracle's own velocity Verlet over all host cores (whole steps, O(N^2))."""
    out = {}
    cases = (("propane_648_fp64_nve", S.propane(), R.RELRES_PREC_FP64, 0.0, 1000, 100),
             ("neopentane_20000_fp32_csvr", S.neopentane(n_mol=4000, seed=2104), R.RELRES_PREC_FP32, 260.0, 1000, 2))
    for name, s, prec, temp, gpu_steps, cpu_steps in cases:
        ctx = R.Context(R.params_for(s, prec), R.topology_for(s))
        pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        vel = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
        ctx.build_neighbors(pos, s.box)
        ctx.step(100, s.dt, pos, vel, t_target=temp, tau_fs=100.0, seed=3)  # warm-up, graphs captured
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ctx.step(gpu_steps, s.dt, pos, vel, t_target=temp, tau_fs=100.0, seed=4)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ctx.close()
        row = {"n_atoms": s.n_atoms, "steps": gpu_steps, "gpu_ms_per_step": ms / gpu_steps,
               "gpu_atom_steps_per_s": s.n_atoms * gpu_steps / (ms * 1e-3)}
        if with_oracle:
            from oracle import core as O

            O.build_oracle()
            t0 = time.perf_counter()
            O.md(s.pos, s.vel, s.box, s.masses, s.types, O.table_for(s), s.n_types, s.excl, s.topo, cpu_steps,
                 s.dt, t_target=temp, tau=100.0, seed=4)
            el = time.perf_counter() - t0
            row.update({"oracle_steps": cpu_steps, "oracle_ms_per_step": el / cpu_steps * 1e3,
                        "oracle_atom_steps_per_s": s.n_atoms * cpu_steps / el, "oracle_cores": os.cpu_count()})
        out[name] = row
    return out


def batched_leg(torch, R, S, n_rep, steps, seed=4242):
    """Independent replicas of uneven sizes advanced together (relres_batch:
    one CUDA graph per block of steps for all of them) against the same
    replicas advanced one after the other (one relres_step call each)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    sizes = rng.integers(1000, 50001, size=n_rep)
    temps = rng.uniform(200.0, 300.0, size=n_rep)
    systems = []
    for k in range(n_rep):
        if k % 2 == 0:  # propane-like (3 sites), k^3 molecules on the lattice spacing of 216 in 31.8 A
            kk = max(7, int(round((int(sizes[k]) / 3) ** (1 / 3))))
            systems.append(S.propane(n_mol=kk ** 3, box=31.8 * kk / 6, temperature=temps[k], seed=seed + k))
        else:  # neopentane-like (5 sites)
            systems.append(S.neopentane(n_mol=max(200, int(sizes[k]) // 5), temperature=temps[k], seed=seed + k))
    n_atoms = int(sum(s.n_atoms for s in systems))

    def make():
        ctxs = []
        for s in systems:
            ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
            p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
            v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
            ctx.build_neighbors(p, s.box)
            ctxs.append((ctx, p, v))
        return ctxs

    seeds = list(range(n_rep))

    def timed(stream, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    # batched, three forms on the same replicas: one graph branch per replica
    # (its own kernels), shared launches covering every replica, and the
    # automatic split (small replicas shared, the others on branches)
    ctxs = make()
    bstream = torch.cuda.Stream()
    batch = R.Batch([c for c, _, _ in ctxs], stream=bstream)
    pos = [p for _, p, _ in ctxs]
    vel = [v for _, _, v in ctxs]
    forms = {}
    for mode, name in ((0, "graph_branches"), (1, "all_shared"), (-1, "automatic")):
        batch.set_mode(mode)
        batch.step(20, 2.0, pos, vel, temps, 100.0, seeds)  # warm-up: autotuning, graph capture
        batch.step(steps, 2.0, pos, vel, temps, 100.0, seeds)  # capture of the timed block shape
        secs = timed(bstream, lambda: batch.step(steps, 2.0, pos, vel, temps, 100.0, seeds))
        forms[name] = {"value": n_atoms * steps / secs, "ms_per_step": secs / steps * 1e3,
                       "replicas_in_shared_launches": batch.n_shared()}
    t_batch = n_atoms * steps / forms["automatic"]["value"]
    batch.close()
    for c, _, _ in ctxs:
        c.close()
    # one after the other (each context on the legacy default stream)
    ctxs = make()
    for (c, p, v), t, sd in zip(ctxs, temps, seeds):
        c.step(20, 2.0, p, v, t_target=t, seed=sd)
        c.step(steps, 2.0, p, v, t_target=t, seed=sd)

    def seq():
        for (c, p, v), t, sd in zip(ctxs, temps, seeds):
            c.step(steps, 2.0, p, v, t_target=t, seed=sd)

    t_seq = timed(torch.cuda.default_stream(), seq)
    for c, _, _ in ctxs:
        c.close()
    return {"workload": f"{n_rep} replicas, seeded sizes 1k-50k atoms ({n_atoms} atoms in all), alternately "
                        "propane-like (k^3 molecules) and neopentane-like, T in U[200, 300] K, CSVR, dt 2 fs, FP32",
            "steps": steps, "value": n_atoms * steps / t_batch, "unit": "atom-steps/s",
            "ms_per_step": t_batch / steps * 1e3, "form": "automatic", "forms": forms,
            "one_after_the_other": {"value": n_atoms * steps / t_seq, "ms_per_step": t_seq / steps * 1e3},
            "timing": "CUDA events on the batch stream around one relres_batch_step call (the per-call set-up "
                      "of every replica included); the sequential run: events on the default stream around "
                      "one relres_step per replica"}


def small_batch_leg(torch, R, S, n_rep=128, steps=200):
    """Many small replicas (648-atom propane-like liquids, seeded), where the
    launch overhead of separate systems dominates: the batch in its two forms
    (single launches covering every replica, one graph branch per replica)."""
    systems = [S.propane(seed=100 + k) for k in range(n_rep)]
    n_atoms = sum(s.n_atoms for s in systems)
    ctxs = []
    for s in systems:
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
        p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
        ctx.build_neighbors(p, s.box)
        ctxs.append((ctx, p, v))
    st = torch.cuda.Stream()
    batch = R.Batch([c for c, _, _ in ctxs], stream=st)
    pos, vel = [p for _, p, _ in ctxs], [v for _, _, v in ctxs]
    temps, seeds = [s.temperature for s in systems], list(range(n_rep))
    out = {"workload": f"{n_rep} replicas of the 648-atom propane-like liquid ({n_atoms} atoms), FP32, CSVR, dt 2 fs",
           "steps": steps, "unit": "atom-steps/s"}
    for mode, name in ((1, "all_shared"), (0, "graph_branches")):
        batch.set_mode(mode)
        batch.step(steps, 2.0, pos, vel, temps, 100.0, seeds)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        batch.step(steps, 2.0, pos, vel, temps, 100.0, seeds)
        e1.record(st)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) * 1e-3
        out[name] = {"value": n_atoms * steps / secs, "ms_per_step": secs / steps * 1e3}
    batch.close()
    for c, _, _ in ctxs:
        c.close()
    return out


def differentiable_leg(torch, R, S, stream, n_snap=64, n_mol=4000):
    """Forward (forces + energy) and backward (force-matching loss: dL/dF =
    2 (F - F_ref), dL/dE = 1) of the RelRes pair interaction through the C ABI
    on seeded snapshots of the 20 000-atom neopentane-like liquid (FP32 with
    FP64 totals): one context, lists rebuilt per snapshot as needed."""
    import numpy as np

    base = S.neopentane(n_mol=n_mol, seed=2104)
    rng = np.random.default_rng(11)
    n = base.n_atoms
    with torch.cuda.stream(stream):
        ctx = R.Context(R.params_for(base, R.RELRES_PREC_FP32),
                        R.make_topology(base.types, base.mass_by_type, base.excl, None), stream=stream)
        snaps = [torch.tensor(base.pos + rng.normal(scale=0.15, size=base.pos.shape), dtype=torch.float64,
                              device="cuda") for _ in range(n_snap)]
        f = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        f_ref = torch.zeros_like(f)
        e = torch.zeros(4, dtype=torch.float64, device="cuda")
        gx = torch.empty_like(f)
        ctx.build_neighbors(snaps[0], base.box)
        for p in snaps[:3]:  # warm-up
            ctx.compute(p, f, e)
            ctx.backward(p, 2.0 * (f - f_ref), 1.0, gx)
        torch.cuda.synchronize()
        t_fwd = t_bwd = 0.0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for p in snaps:
            ev[0].record(stream)
            ctx.compute(p, f, e)
            ev[1].record(stream)
            g = 2.0 * (f - f_ref)
            ctx.backward(p, g, 1.0, gx)
            ev[2].record(stream)
            torch.cuda.synchronize()
            t_fwd += ev[0].elapsed_time(ev[1])
            t_bwd += ev[1].elapsed_time(ev[2])
        ctx.close()
    return {"workload": f"{n_snap} seeded snapshots of the {n}-atom neopentane-like liquid (0.15 A noise), "
                        "FP32 forward with energies, force-matching backward",
            "ms_per_snapshot_forward": t_fwd / n_snap, "ms_per_snapshot_backward": t_bwd / n_snap,
            "snapshots_per_s": n_snap / ((t_fwd + t_bwd) * 1e-3)}


def _oracle_rows_rate(s, seconds, rng_seed=0):
    """Oracle (FP64, all-pairs) force rows of the full system on all host
    cores: rows/s = atom-steps/s of a full force evaluation."""
    import numpy as np

    from oracle import core as O

    table = O.table_for(s)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(rng_seed)
    probe = rng.choice(s.n_atoms, size=cores, replace=False)
    t0 = time.perf_counter()
    O.pair_forces_rows(s.pos, s.box, s.types, table, s.n_types, probe, s.excl, n_threads=cores)
    dt_probe = time.perf_counter() - t0
    n_rows = max(cores, int(cores * seconds / max(dt_probe, 1e-6)))
    n_rows = min(n_rows, s.n_atoms)
    rows = rng.choice(s.n_atoms, size=n_rows, replace=False)
    t0 = time.perf_counter()
    O.pair_forces_rows(s.pos, s.box, s.types, table, s.n_types, rows, s.excl, n_threads=cores)
    el = time.perf_counter() - t0
    return n_rows, el, cores


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(s, seconds):
    n_rows, el, cores = _oracle_rows_rate(s, seconds)
    # the same oracle on one core, on a smaller sample
    import numpy as np

    from oracle import core as O

    table = O.table_for(s)
    rows1 = np.random.default_rng(3).choice(s.n_atoms, size=max(1, n_rows // max(1, cores) // 4), replace=False)
    t0 = time.perf_counter()
    O.pair_forces_rows(s.pos, s.box, s.types, table, s.n_types, rows1, s.excl, n_threads=1)
    el1 = time.perf_counter() - t0
    return {"value": n_rows / el, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 all-pairs Eq. 20 force rows of {n_rows} random atoms of the "
                      f"{s.n_atoms}-atom system ({el:.1f} s); one step needs all rows",
            "single_core": {"value": len(rows1) / el1, "rows": int(len(rows1)), "seconds": round(el1, 2)},
            "cpu_model": _cpu_model(), "nproc": os.cpu_count()}


def reference(args):
    """The oracle as the reference arm: each step is a bounded sample of force
    rows of the same 1M-atom workload, on the host cores (rank 0 only)."""
    import numpy as np

    from oracle import core as O
    from paper_2104_10231_gb300 import systems as S

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.core import build_oracle

    build_oracle()
    s = S.neopentane(n_mol=args.n_mol, seed=2104, temperature=260.0)
    table = O.table_for(s)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    rows_per_step = cores

    def one():
        rows = rng.choice(s.n_atoms, size=rows_per_step, replace=False)
        O.pair_forces_rows(s.pos, s.box, s.types, table, s.n_types, rows, s.excl, n_threads=cores)

    for _ in range(max(0, args.warmup)):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    value = rows_per_step * args.steps / el
    print(json.dumps({
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "atom-steps/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded neopentane-like liquid)",
        "config": workload_config(args, s.n_atoms, float(s.box[0])),
        "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows_per_step} random full force rows per step of the "
                                   f"{s.n_atoms}-atom system"},
        "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        ours(a)
