#!/usr/bin/env python
"""Throughput of the SRD (MPCD) time step on GB300: particle updates per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One step = stream + shift + bin + counting sort + per-cell sums + rotation of every
particle (the whole hot path) on one box of the named workload (default: FP64, 128^3 cells,
10 particles per cell, 20,971,520 particles, full re-sort every 10 steps).  The state
(1 GB) is larger than L2, so no flush is needed between steps.  Prints one JSON line.

With N > 1 (launched by torch.distributed.run) every rank advances its own independent
replica box (the single-box path has no exchange step); `value` is the sum over ranks of
updates divided by the slowest rank's time.

Beside an FP64 run the same process times the mixed-precision form (256^3 cells, 167,772,160
particles) and the 256-box ensemble the same way and reports them under `forms`, each with
its speedup over the FP64 run (--no-forms skips them).

--impl reference times the FP64 CPU oracle (the plain statement the library is checked
against) on the same workload on the host cores, on rank 0 only.
"""
from __future__ import annotations

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
sys.path.insert(0, ROOT)

METRIC = "particle updates/sec/GPU and % of HBM roofline; mixed/batched vs FP64"
UNIT = "particle updates/s"

# Algorithmic HBM bytes per launch of each kernel, as (bytes per particle, bytes per cell):
# what the kernel must read and write once (state, keys, ranks, perm, counts, offsets).
FP64_BYTES = {
    "zero_counts": (0.0, 8.0),   # counts and cursors
    "stream_bin": (48.0 + 24.0 + 8.0, 4.0),
    "scan": (0.0, 12.0),
    "scatter": (12.0, 4.0),
    "collide": (4.0 + 24.0, 8.0 + 128.0),   # cell_frame: v through perm, offsets, 16-double frame
    "rotate": (24.0 + 24.0 + 4.0 + 8.0, 0.0),  # v read + written, key, frame gather (amortised)
    # the rotation of step t fused with the streaming of step t + 1: r, v read and written,
    # key of step t read and of step t + 1 written, rank written, frame gather (amortised)
    "rotate_stream": (48.0 + 48.0 + 4.0 + 4.0 + 4.0 + 8.0, 4.0),
    "end_step": (0.0, 0.0),
}
# on re-sort steps each slot gathers its particle through perm (4 B) and moves its id (4 + 4);
# the separate rotation also moves r (24 + 24), the fused pass moves r anyway
FP64_RESORT_EXTRA = 24.0 + 24.0 + 8.0 + 4.0
FP64_RESORT_EXTRA_FUSED = 8.0 + 4.0
# FP64-pipe instructions (DFMA, DADD, DSUB, DMUL) per launch, as (per particle, per cell), on
# GB300's narrow FP64 pipe (2 per clock per SM), as counted by ncu
# (sm__thread_inst_executed_pipe_fp64_pred_on, profiles/fp64_L64_fp64_instruction_counts.md):
# streaming 3 DFMA (r - s is taken in fixed point, in FP64 only next to a cell face); the frame
# applied in float-float arithmetic joins each component with one DADD; cell_frame 44 per cell
# (u and the axis; R and b are built in float-float arithmetic).
FP64_OPS = {"stream_bin": (3.0, 0.0), "collide": (0.0, 44.0), "rotate": (3.0, 0.0), "rotate_stream": (6.0, 0.0)}
SMS, FP64_PER_CLK, SM_MAX_MHZ = 152, 2, 2070.0
FP64_PEAK_GOPS = SMS * FP64_PER_CLK * SM_MAX_MHZ / 1e3   # 629.3 G FP64 instructions/s
ALGO_STEP_BYTES_FP64 = 96.0             # state read + written once per step
# mixed form: 32-byte records; collide_stream gathers through perm, writes in cell order and
# writes the next step's keys and ranks
MIXED_BYTES = {
    "zero_counts": (0.0, 8.0),   # counts and cursors
    "stream_bin": (32.0 + 8.0, 4.0),     # first step only
    "scan": (0.0, 12.0),
    "scatter": (12.0, 4.0),
    "collide": (4.0 + 32.0 + 32.0 + 8.0, 8.0),
    "end_step": (0.0, 0.0),
    # the one-launch step: collide, plus the scatter (key, perm, offset) and per cell the
    # zeroing of counts and cursors, two count reads of the scan, the offsets, the cursors
    "step": (4.0 + 32.0 + 32.0 + 8.0 + 12.0, 24.0),
}
ALGO_STEP_BYTES_MIXED = 64.0
# DRAM bytes (read + write) per particle of a kernel from one ncu capture of the current build,
# scaled to a launch by the particle count; a kernel changed since its capture has none.
NCU_TRAFFIC = {("mixed", "collide"): (72.07, "profiles/mixed_L128_collide_stream_full.md (128^3 capture)"),
               ("fp64", "rotate_stream"): (111.0, "profiles/fp64_L64_rotate_stream_full.md (64^3 capture of an "
                                                  "ordinary, non-re-sort launch, scaled by the particle count)")}
# timed beside an FP64 run: the mixed form at 256^3, the 256-box ensemble, the walled
# channel with each cell thermostat, the angular-momentum-conserving collision and per-particle
# masses
FORMS = ("mixed_L256", "batched_256", "poiseuille_256x64x64", "poiseuille_256x64x64_mbs", "fp64_L128_angular",
         "mixed_L128_angular", "fp64_L128_masses", "mixed_L128_masses")


# What each form reaches against the FP64 oracle (the parity and error-report tests), stated
# beside its speed-up over the plain FP64 form (which matches the oracle to 1e-12).
FORM_ACCURACY = {
    "mixed_L256": "mixed: one step from identical states v within 8.9e-7 relative, positions 6e-8 cells, "
                  "per-cell momentum 1.3e-7 and energy 3e-7 per collision (64^3 error report)",
    "batched_256": "mixed, per box as mixed_L256; every box bit-identical to the box alone",
    "poiseuille_256x64x64": "mixed with walls; Poiseuille profile within 1.8% rms of the FP64 form",
    "poiseuille_256x64x64_mbs": "mixed with walls and MBS thermostat; canonical cell energies (KS)",
    "fp64_L128_angular": "FP64: 1e-12 against the oracle (omega scaled by the inertia tensor's condition)",
    "mixed_L128_angular": "mixed: per-cell momentum and angular momentum conserved to FP32 rounding",
    "fp64_L128_masses": "FP64: 1e-12 against the oracle",
    "mixed_L128_masses": "mixed with FP32 masses: one-step bounds as mixed_L256 against the mass-weighted oracle",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fp64_L128")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the mixed and ensemble forms")
    ap.add_argument("--form-steps", type=int, default=100)
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            if self.bus_id and self.bus_id[-12:] not in f[1].lower():
                continue
            rows.append(f)
        os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(nm)
        power = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][3]) if rows[0][3].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(power) if power else None}


def cpu_oracle_run(w, steps, sample_note, all_cores=False):
    """Time the FP64 oracle as it stands on the workload on the host: its serial build on one
    core, or (all_cores) the same source built with OpenMP on every core of the host."""
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    orc.use_openmp(all_cores)
    try:
        p = orc.make_params(w.L, a=w.a, dt=w.dt, alpha_deg=w.alpha_deg, kT=w.kT, mass=w.mass, ppc=w.ppc, seed=w.seed,
                            resort_k=w.resort_k, walls_z=w.walls_z, g=w.g, thermostat=w.thermostat,
                            angular=getattr(w, "angular", 0))
        r, v = orc.init(p, w.n_particles)
        st = orc.presort(p, orc.State(r, v))
        orc.step(p, st)   # untimed first step (page-in)
        t0 = time.perf_counter()
        for _ in range(steps):
            orc.step(p, st)
        dt = time.perf_counter() - t0
    finally:
        orc.use_openmp(False)
    value = w.n_particles * steps / dt
    how = ("OpenMP build of the same source, %d threads" % cores) if all_cores else "serial build, single thread"
    return {"value": value, "unit": UNIT, "cores": cores if all_cores else 1, "kind": "oracle",
            "sample": "%s: %d oracle steps of the full %d-particle box (%.1f s), %s" % (
                sample_note, steps, w.n_particles, dt, how)}


REF_TIME_LIMIT_S = 150.0  # the reference arm stops its timed steps after this much CPU time


def run_reference(args, w):
    """The reference arm: the FP64 oracle as it stands (its OpenMP build, every host core) on
    the full workload box, from the same initial state as the library; the timed steps stop
    early once REF_TIME_LIMIT_S of wall time is spent (stated in `sample`)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    orc.use_openmp(True)
    n = w.n_particles
    p = orc.make_params(w.L, a=w.a, dt=w.dt, alpha_deg=w.alpha_deg, kT=w.kT, mass=w.mass, ppc=w.ppc, seed=w.seed,
                        resort_k=w.resort_k, walls_z=w.walls_z, g=w.g, thermostat=w.thermostat,
                        angular=getattr(w, "angular", 0))
    r, v = orc.init(p, n)
    st = orc.presort(p, orc.State(r, v))
    for _ in range(max(1, args.warmup)):
        orc.step(p, st)
        if st.t >= 3:
            break
    done, t_cpu = 0, 0.0
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        orc.step(p, st)
        t_cpu += time.perf_counter() - t0
        done += 1
        if t_cpu > REF_TIME_LIMIT_S:
            break
    value = n * done / t_cpu
    sample = ("%d oracle steps (of %d asked; %d warm-up) of the full %s box (%d particles); OpenMP build of the "
              "oracle source, %d threads; %.1f s" % (done, args.steps, min(max(1, args.warmup), 3), w.name, n,
                                                      int(os.environ["OMP_NUM_THREADS"]), t_cpu))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "L": list(w.L), "particles": n, "precision": w.precision},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


class EnsembleWorkload:
    """Adapter so that an ensemble recipe looks like a single workload to the bench."""

    def __init__(self, name, rec):
        self.name = name
        self.rec = rec
        self.L = (len(rec.sides), 0, 0)
        self.n_particles = rec.n_particles
        self.precision = "mixed"
        self.ppc = float(np.mean(rec.ppc)) if rec.nbox else 0.0
        self.resort_k = 1
        self.alpha_deg = None
        self.dt = None
        self.seed = rec.seeds[0] if rec.nbox else 0


def open_box(abi, inputs, name, rank):
    """The box (or ensemble) of a named workload; rank r draws its own seeds."""
    from paper_2212_11878_gb300 import replicas
    ensemble = name in inputs.BATCH_WORKLOADS
    w = EnsembleWorkload(name, inputs.batch_workload(name)) if ensemble else inputs.WORKLOADS[name]
    if ensemble:
        plist = abi.params_from_recipe(w.rec)
        for q in plist:
            q.seed = replicas.ensemble_seed(q.seed, rank)
        return w, plist[0], abi.Box(batch=plist), True
    p = abi.params_from_workload(w, seed=replicas.box_seed(w.seed, rank))
    box = abi.Box(p)
    if getattr(w, "mass_range", ()):
        box.set_masses(inputs.particle_masses(box.n, p.seed, *w.mass_range, mass=p.mass))
    return w, p, box, False


def timed_steps(abi, torch, dist, box, stream, steps, world, sampler=None):
    """K steps bracketed by barrier + synchronize, timed with CUDA events on the launching
    stream (per-kernel events inside); returns (updates/s of all ranks over the slowest
    rank's time, that time in ms, launches, kernel times, clocks)."""
    h = box.h
    abi.mpcd_timing(h, True)
    l0 = abi.mpcd_launch_count(h)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    box.step(steps)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    launches = abi.mpcd_launch_count(h) - l0
    ktimes = abi.mpcd_timing_read(h)
    abi.mpcd_timing(h, False)
    from paper_2212_11878_gb300 import replicas
    value, ms, _ = replicas.job_throughput(box.n * steps, ms, dist if world > 1 else None, device="cuda")
    if world > 1:
        dist.barrier()
    return value, ms, launches, ktimes, clocks


def kernel_table(p, mixed, n, C, ktimes, steps):
    """Per-kernel device time per step, share, algorithmic HBM bytes and GB/s, and for the
    FP64 kernels their FP64 instruction rate.  Rates are per launch of the kernel (its bytes
    or instructions over its average launch time); the FP64 dense pair launches stream_bin and
    rotate once per mpcd_step call and the fused rotate_stream on every other step."""
    kernels = {}
    total_kernel_ms = sum(v[0] for v in ktimes.values()) or 1.0
    model = MIXED_BYTES if mixed else FP64_BYTES
    once_per_call = ("stream_bin", "rotate", "rotate_stream") if not mixed else ()
    for name, (kms, cnt) in ktimes.items():
        per_p, per_c = model.get(name, (0.0, 0.0))
        invocations = cnt if name in once_per_call else steps   # slot invocations in the timed region
        bytes_inv = per_p * n + per_c * C
        if name in ("rotate", "rotate_stream") and p.resort_k > 0 and not mixed:
            extra = FP64_RESORT_EXTRA if name == "rotate" else FP64_RESORT_EXTRA_FUSED
            bytes_inv += extra * n / p.resort_k
        ms_inv = kms / max(invocations, 1)
        k = {"ms_per_step": kms / steps, "ms_per_invocation": ms_inv, "invocations": invocations, "launches": cnt,
             "share": kms / total_kernel_ms, "algo_bytes_per_invocation": bytes_inv,
             "gbs": bytes_inv / (ms_inv / 1e3) / 1e9 if kms > 0 else None}
        if not mixed and name in FP64_OPS:
            ops = FP64_OPS[name][0] * n + FP64_OPS[name][1] * C
            k["fp64_ops_per_invocation"] = ops
            k["fp64_gops"] = ops / (ms_inv / 1e3) / 1e9 if kms > 0 else None
        kernels[name] = k
    return kernels


def roofline_of(kernels, mixed, hbm_peak, peak_src, n, captured=True, fp64_probe=None):
    """The dominant kernel against its bound: HBM bytes (mixed form) or the FP64 pipe (FP64
    form: measured traffic stays far below HBM; the FP64 instruction count sets the floor).
    `captured`: the kernel variant is the one the ncu traffic figure was taken on (periodic,
    no force, no thermostat); other variants report no traffic."""
    if mixed:
        dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
        d = kernels[dom]
        per_launch = d["algo_bytes_per_invocation"]
        tr = NCU_TRAFFIC.get(("mixed", dom)) if captured else None
        return dict(traffic_rates(tr[0] * n if tr else None, d, hbm_peak), **{"kernel": dom, "bound": "hbm", "achieved": d["gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": d["gbs"] / hbm_peak, "traffic": tr[0] * n if tr else None,
                "traffic_source": tr[1] if tr else None, "peak_source": peak_src + " (hbm_gbs)",
                "algo_bytes_per_launch": per_launch})
    fp64k = [k for k in kernels if "fp64_gops" in kernels[k]]
    dom = max(fp64k, key=lambda k: kernels[k]["ms_per_step"])
    d = kernels[dom]
    tr = NCU_TRAFFIC.get(("fp64", dom))
    alu_frac, hbm_frac = d["fp64_gops"] / FP64_PEAK_GOPS, d["gbs"] / hbm_peak
    alu = {"fp64_achieved": d["fp64_gops"], "fp64_peak": FP64_PEAK_GOPS, "fp64_unit": "G FP64 instructions/s",
           "fp64_frac": alu_frac,
           "fp64_peak_source": "derived: %d SMs x %d FP64 instructions/clock x %.0f MHz" % (SMS, FP64_PER_CLK,
                                                                                              SM_MAX_MHZ),
           "algo_fp64_ops_per_launch": d["fp64_ops_per_invocation"],
           "fp64_peak_measured": fp64_probe, "fp64_frac_of_measured": d["fp64_gops"] / fp64_probe if fp64_probe else None,
           "fp64_peak_measured_source": "mpcd_measure_fp64_rate: chains of independent DFMAs on every SM, this run"}
    # the bound is the nearer of the two ceilings (HBM bytes or FP64-pipe instructions)
    if hbm_frac >= alu_frac:
        out = {"kernel": dom, "bound": "hbm", "achieved": d["gbs"], "peak": hbm_peak, "unit": "GB/s",
               "frac": hbm_frac, "peak_source": peak_src + " (hbm_gbs)",
               "algo_bytes_per_launch": d["algo_bytes_per_invocation"]}
    else:
        out = {"kernel": dom, "bound": "alu", "achieved": d["fp64_gops"], "peak": FP64_PEAK_GOPS,
               "unit": "G FP64 instructions/s", "frac": alu_frac, "peak_source": alu["fp64_peak_source"],
               "algo_bytes_per_launch": d["algo_bytes_per_invocation"]}
    out.update(traffic=tr[0] * n if tr else None, traffic_source=tr[1] if tr else None, **alu)
    out.update(traffic_rates(out["traffic"], d, hbm_peak))
    return out


def traffic_rates(traffic, d, hbm_peak):
    """The measured-traffic fraction beside the algorithmic one: ncu's DRAM bytes of a launch
    over the same CUDA-event launch time."""
    if not traffic or not d.get("ms_per_invocation"):
        return {"traffic_gbs": None, "traffic_frac": None}
    gbs = traffic / (d["ms_per_invocation"] / 1e3) / 1e9
    return {"traffic_gbs": gbs, "traffic_frac": gbs / hbm_peak}


def main():
    args = parse()
    from paper_2212_11878_gb300 import inputs
    ensemble = args.workload in inputs.BATCH_WORKLOADS
    if args.impl == "reference":
        if ensemble:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle times single-box workloads"}))
            return
        run_reference(args, inputs.WORKLOADS[args.workload])
        return

    import torch
    import torch.distributed as dist
    from paper_2212_11878_gb300 import abi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0

    fp64_probe = abi.mpcd_measure_fp64_rate() / 1e9   # G FP64 FMAs/s of this GPU, measured now
    stream = torch.cuda.Stream()
    w, p, box, ensemble = open_box(abi, inputs, args.workload, rank)
    h = box.h
    abi.mpcd_set_stream(h, stream.cuda_stream)
    n = box.n
    mixed = p.precision == abi.MPCD_MIXED

    box.step(args.warmup)
    box.sync()
    props = torch.cuda.get_device_properties(local)
    bus = getattr(props, "pci_bus_id", None)
    sampler = ClockSampler(bus if isinstance(bus, str) else None)
    value, ms, launches, ktimes, clocks = timed_steps(abi, torch, dist, box, stream, args.steps, world, sampler)

    # --- end to end through the host-buffer API: upload, one step, download ---
    r_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    v_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    r_np, v_np = r_h.numpy(), v_h.numpy()
    abi.mpcd_get_state(h, r_np, v_np)
    abi.mpcd_set_state(h, r_np, v_np, abi.mpcd_steps_done(h))  # one untimed cycle (first-touch costs)
    abi.mpcd_step(h, 1)
    abi.mpcd_get_state(h, r_np, v_np)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        abi.mpcd_set_state(h, r_np, v_np, abi.mpcd_steps_done(h))
        abi.mpcd_step(h, 1)
        abi.mpcd_get_state(h, r_np, v_np)
    e2e_s = time.perf_counter() - t0
    from paper_2212_11878_gb300 import replicas
    e2e_value, _, _ = replicas.job_throughput(n * args.e2e_steps, e2e_s * 1e3, dist if world > 1 else None, device="cuda")
    C = box.ncell
    kernels = kernel_table(p, mixed, n, C, ktimes, args.steps)
    # the basis of the forms' speed-ups: this box again, timed over the forms' step count
    basis = None
    if not mixed and not args.no_forms:
        box.set_state(r_np, v_np, abi.mpcd_steps_done(h))
        box.step(args.warmup)
        box.sync()
        bval, bms, _, _, _ = timed_steps(abi, torch, dist, box, stream, args.form_steps, world)
        basis = {"workload": w.name, "value": bval, "steps": args.form_steps, "warmup": args.warmup,
                 "ms_per_step": bms / args.form_steps}
    box.close()
    del r_h, v_h

    # --- the mixed-precision and ensemble forms, timed the same way, against this FP64 run ---
    forms = {}
    if not mixed and not args.no_forms:
        for name in FORMS:
            fw, fp, fbox, fens = open_box(abi, inputs, name, rank)
            abi.mpcd_set_stream(fbox.h, stream.cuda_stream)
            tuned = None
            if fens:  # the ensemble's tile shape, block size and launch form: the autotuner's choice
                best, best_ms = abi.mpcd_autotune(fbox.h, trial_steps=5)
                tuned = dict(best.as_dict(), ms_per_step_in_trial=best_ms,
                             candidates="group_target {128..176} x warps {2,4} x fuse {1,0} (one launch per step or eight)")
            fbox.step(args.warmup)
            fbox.sync()
            fval, fms, fl, fkt, _ = timed_steps(abi, torch, dist, fbox, stream, args.form_steps, world)
            fn = fbox.n
            fmixed = fens or fw.precision == "mixed"
            fk = kernel_table(fp, fmixed, fn, fbox.ncell, fkt, args.form_steps)
            captured = not (getattr(fw, "walls_z", 0) or getattr(fw, "thermostat", 0) or any(getattr(fw, "g", (0.0,)))
                            or getattr(fw, "angular", 0))
            if fmixed:
                froof = roofline_of(fk, True, hbm_peak, peak_src, fn, captured=captured)
            else:  # the per-cell collide of these FP64 variants has no instruction model
                froof = None
            forms[name] = {"value": fval, "unit": UNIT, "steps": args.form_steps, "ms_per_step": fms / args.form_steps,
                           "particles": fn, "cells": fbox.ncell, "boxes": fw.rec.nbox if fens else 1,
                           "speedup_vs_fp64": fval / basis["value"], "accuracy": FORM_ACCURACY.get(name),
                           "gpu_launches": fl,
                           "hbm_roofline_frac_step": fval / world * (ALGO_STEP_BYTES_MIXED if fmixed else
                                                                     ALGO_STEP_BYTES_FP64) / 1e9 / hbm_peak,
                           "roofline": froof, "autotuned": tuned,
                           "kernels": {k: {"ms_per_step": v["ms_per_step"], "share": v["share"], "gbs": v["gbs"]}
                                       for k, v in fk.items()}}
            fbox.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not ensemble:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        cpu = cpu_oracle_run(w, args.cpu_steps, "cpu_baseline", all_cores=True)
        cpu["single_core"] = cpu_oracle_run(w, args.cpu_steps, "cpu_baseline")

    if rank == 0:
        ms_step = ms / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if mixed else "f64", "data": "synthetic",
            "config": {"workload": w.name, "L": list(w.L) if not ensemble else None,
                       "boxes": w.rec.nbox if ensemble else 1, "particles": n, "cells": C, "ppc": w.ppc,
                       "precision": w.precision, "resort_k": w.resort_k, "alpha_deg": w.alpha_deg, "dt": w.dt,
                       "l2": "no flush: state %.2f GB > 129 MB L2" % (n * (64 if mixed else 104) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "hbm_roofline_frac_step": value / world * (ALGO_STEP_BYTES_MIXED if mixed else ALGO_STEP_BYTES_FP64) / 1e9
            / hbm_peak,
            "roofline": roofline_of(kernels, mixed, hbm_peak, peak_src, n, fp64_probe=fp64_probe),
            "kernels": kernels,
            "forms": forms or None,
            "forms_basis": basis,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 48, "d2h_bytes_per_step": n * 48,
                    "steps": args.e2e_steps},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
