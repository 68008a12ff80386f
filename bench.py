#!/usr/bin/env python
"""Benchmark: ns per spin update of the heat-bath + over-relaxation + parallel
tempering step on one GB300 (and N GPUs as independent replicas).

A step is the whole hot path once: 1 heat-bath sweep, 5 over-relaxation
sweeps, FP64 energies and one parallel-tempering pass (hsg_step), with the
overlap measurement (hsg_measure) every 10th step.  t_update follows the
paper's definition, t_run / [(n_OR + n_HB) * steps * systems * N] (Sec. 4).

Default workload: L = 128, 2 replicas x 24 temperatures in [0.08, 0.3], FP16
spins and couplings, H_r = 0.1 (100.7M spins, 604 MB of spin state, larger
than L2, so no flush is needed between steps).  The line also carries the
plain-FP32 form of the same lattice and the plain-FP32 L = 32 production
shape (25 MB, L2 flushed between timed steps) for the compressed-vs-plain
comparison, the paper's Table 1 configuration, and the multi-hit tile
schedule (per-update time and the time to an uncorrelated sample).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ns per spin update"
UNIT = "ns/spin-update"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="L128_fp16")
    ap.add_argument("--measure-every", type=int, default=10)
    ap.add_argument("--no-extras", action="store_true", help="skip the plain-FP32 comparison lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--schedule", default="auto", choices=["auto", "two_pass", "persistent"],
                    help="step schedule: tuned at the first step (default) or fixed")
    ap.add_argument("--sweep-kernel", default="auto", choices=["auto", "half", "fused", "wave", "staged"],
                    help="over-relaxation sweep kernel: tuned (default), one launch per half-sweep, "
                         "the fused one-pass sweep, the wave sweep, or half-sweeps with staged rows")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_samples(wl, rank):
    """Rank r > 0 runs its own disorder sample (independent problems, no
    collective on the data path): fresh couplings from a rank-keyed generator."""
    if rank:
        import numpy as np
        from paper_1204_6192_gb300 import inputs
        rng = np.random.default_rng(1000 + rank)
        for s in wl.samples:
            s.J = inputs.gaussian_couplings(s.L, rng)
    return wl


def max_over_ranks(x, torch, device):
    """The slowest rank's value (every rank gets it)."""
    if not torch.distributed.is_available() or not torch.distributed.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ms, updates_per_rank, world):
    """ns per spin update of the whole job: every rank's updates over the slowest rank's time."""
    return ms * 1e6 / (updates_per_rank * world)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                self.samples.append([x.strip() for x in row])
            except Exception:
                pass

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.samples if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.samples if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.samples:
            for k, n in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
SPIN_BYTES = {"fp32": 12, "fp16": 6, "bf16": 6, "angle16": 4, "oct16": 4, "yx4": 8}


def bytes_per_update(wl, W, fused=True):
    """Bytes one spin update must move.  Fused (one pass per sweep): the spin is
    read once and written once (2 S) and every site's 3 bonds and 3 field
    components are read once for the W systems that share them.  Two-pass (one
    launch per half-sweep): each updated spin's own read and write plus one read
    of the opposite-parity spin it sees (3 S), and the 6 bonds + 3 field
    components of every updated site's record."""
    S = SPIN_BYTES[wl.precision]
    jb = 2 if wl.j_fp16 else 4
    return 2 * S + 6 * jb / W if fused else 3 * S + 9 * jb / W


def algorithmic_half_sweep_bytes(ctx, wl, fused=True):
    """Algorithmic bytes of one half-sweep launch (N/2 sites x W systems updated)."""
    sites = sum(s.L ** 3 for s in wl.samples) // 2
    return int(round(sites * ctx.W * bytes_per_update(wl, ctx.W, fused)))


def run_ours(args, wl, torch, dev, rank, world, measure_every, do_roofline=True):
    from paper_1204_6192_gb300 import hsg
    stream = torch.cuda.Stream(device=dev)
    variant = {"auto": hsg.VARIANT_AUTO, "two_pass": hsg.VARIANT_TWO_PASS,
               "persistent": hsg.VARIANT_PERSISTENT}[getattr(args, "schedule", "auto")]
    kernel = {"auto": hsg.SWEEP_AUTO, "half": hsg.SWEEP_HALF, "fused": hsg.SWEEP_FUSED,
              "wave": hsg.SWEEP_WAVE, "staged": hsg.SWEEP_STAGED}[getattr(args, "sweep_kernel", "auto")]
    ctx = hsg.Context(wl.samples, wl.n_replicas, wl.seed + rank, precision=wl.precision,
                      j_fp16=wl.j_fp16, n_hb=wl.n_hb, n_or=wl.n_or, device=dev.index,
                      stream=stream.cuda_stream, variant=variant, sweep_kernel=kernel)
    info = ctx.info()
    spins = info.total_spins
    sweeps = wl.n_hb + wl.n_or
    n_meas = 0
    for k in range(args.warmup):
        ctx.step(1)
        if measure_every and (k + 1) % measure_every == 0:
            ctx.measure()
    ctx.measure()
    ctx.sync()
    res = {"ctx": ctx, "stream": stream}
    return res, spins, sweeps


def timed_steps(ctx, stream, torch, steps, measure_every, flush=None):
    """Time `steps` steps with CUDA events on the context's stream.  With
    `flush`, L2 is flushed before every step and only the steps are timed."""
    n_meas = 0
    if flush is None:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(steps):
            ctx.step(1)
            if measure_every and (k + 1) % measure_every == 0:
                ctx.measure()
                n_meas += 1
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1), n_meas
    total = 0.0
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        ctx.step(1)
        if measure_every and (k + 1) % measure_every == 0:
            ctx.measure()
            n_meas += 1
        t1.record(stream)
        t1.synchronize()
        total += t0.elapsed_time(t1)
    return total, n_meas


SWEEP_NAMES = {1: "half", 2: "fused", 3: "wave", 4: "staged"}


def one_launch_per_sweep(info):
    """The fused and the wave sweep do both half-sweeps in one launch."""
    return info.sweep_kernel in (2, 3)


def roofline(ctx, stream, torch, wl, reps=20, half=True):
    """Average kernel durations with CUDA events on the context's stream:
    the over-relaxation sweep as the step runs it (fused or wave: `reps`
    launches of one sweep each; otherwise 2 * `reps` half-sweep launches), the
    over-relaxation half-sweep kernel on its own (sweep_or(1) runs it beside the
    fused sweep; with the wave sweep a context with the half-sweep kernel is
    timed) and the heat-bath half-sweep.  Returns (ms per OR launch, sweep kind,
    ms per OR half-sweep launch, ms per HB half-sweep launch)."""
    info = ctx.info()
    kind = SWEEP_NAMES[info.sweep_kernel]

    def timed(fn):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        fn()
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1)

    ctx.sweep_or(2)
    ms_or = timed(lambda: ctx.sweep_or(reps)) / (reps if one_launch_per_sweep(info) else 2 * reps)
    ms_half = ms_or
    if kind == "fused":
        ms_half = timed(lambda: [ctx.sweep_or(1) for _ in range(reps // 2)]) / (2 * (reps // 2))
    elif kind == "wave" and half:
        from paper_1204_6192_gb300 import hsg
        h = hsg.Context(wl.samples, wl.n_replicas, wl.seed, precision=wl.precision,
                        j_fp16=wl.j_fp16, device=torch.cuda.current_device(), stream=stream.cuda_stream,
                        variant=hsg.VARIANT_TWO_PASS, sweep_kernel=hsg.SWEEP_HALF,
                        chunks_per_thread=info.chunks_per_thread)
        h.sweep_or(2)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        h.sweep_or(reps)
        t1.record(stream)
        t1.synchronize()
        ms_half = t0.elapsed_time(t1) / (2 * reps)
        h.close()
    k = reps // 4 or 1
    ms_hb = timed(lambda: ctx.sweep_hb(k)) / (2 * k)
    return ms_or, kind, ms_half, ms_hb


def multihit_extras(torch, dev, inputs, lattice_ns):
    """The multi-hit tile schedule (hsg_step_multihit; Sec. 3.2, Table 1's last
    rows): ns per spin update on the bench lattice (one round and ten rounds
    per tile) and on Table 1's configuration; tau_int of the replica overlap
    per schedule on a small lattice at one temperature (Sokal window); and the
    time to an uncorrelated sample relative to the lattice schedule, taking
    each schedule's per-update time on the bench lattice (`lattice_ns`: the
    bench's own value) and its tau in sweeps."""
    import numpy as np
    from paper_1204_6192_gb300 import analysis, hsg
    out = {}
    mh1 = dict(tile=8, n_rounds=1, n_or=10, n_hb=1)
    mh10 = dict(tile=8, n_rounds=10, n_or=10, n_hb=1)

    def timed(stream, fn, k):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        fn(k)
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / k

    per_update = {}
    for name, label, mh, k, paper_ns in (
            ("L128_fp16", "10 OR + 1 HB per 8^3 tile", mh1, 10, None),
            ("L128_fp16", "10 x (1 HB + 10 OR) per 8^3 tile", mh10, 3, None),
            ("table1_hb10or", "10 x (1 HB + 10 OR) per 8^3 tile", mh10, 3, 0.36)):
        w = inputs.workload(name)
        stream = torch.cuda.Stream(device=dev)
        ctx = hsg.Context(w.samples, w.n_replicas, w.seed, precision=w.precision,
                          j_fp16=w.j_fp16, device=dev.index, stream=stream.cuda_stream)
        ctx.step_multihit(1, **mh)
        ms = timed(stream, lambda n: ctx.step_multihit(n, **mh), k)
        ns = ms * 1e6 / (ctx.info().total_spins * mh["n_rounds"] * (mh["n_or"] + mh["n_hb"]))
        entry = {"step": label + ", then energies + PT", "value": round(ns, 6), "unit": UNIT,
                 "ms_per_step": round(ms, 4)}
        if paper_ns:
            entry.update({"paper_gtx480_ns": paper_ns, "ratio_paper_over_ours": round(paper_ns / ns, 1)})
        out[f"{name}: {label}"] = entry
        if name == "L128_fp16":
            per_update[label] = ns
        ctx.close()

    # tau_int of the squared overlaps q_ab^2 = D_ab(0)^2 of the six pairs of 4
    # replicas, L = 16, one temperature (T = 0.2: no PT move mixes
    # configurations), H_r = 0.05 (the energy is a fast observable:
    # over-relaxation conserves it)
    smp = inputs.make_sample(16, np.array([0.2]), 0.05, disorder_seed=7)
    chains = (("lattice: 1 HB + 5 OR", None, 6000, lattice_ns),
              ("tiles: 10 OR + 1 HB", mh1, 8000, per_update["10 OR + 1 HB per 8^3 tile"]),
              ("tiles: 10 x (1 HB + 10 OR)", mh10, 8000,
               per_update["10 x (1 HB + 10 OR) per 8^3 tile"]))
    tau = {}
    base = None
    for label, mh, n, ns_l128 in chains:
        stream = torch.cuda.Stream(device=dev)
        ctx = hsg.Context([smp], 4, 3, device=dev.index, stream=stream.cuda_stream,
                          variant=hsg.VARIANT_TWO_PASS)
        step = (lambda k: ctx.step(k)) if mh is None else (lambda k: ctx.step_multihit(k, **mh))
        sweeps = 6 if mh is None else mh["n_rounds"] * (mh["n_or"] + mh["n_hb"])
        step(max(100, 6000 // sweeps))                 # equilibration: >= 6000 sweeps
        q2 = np.empty((n, 6))
        for i in range(n):
            step(1)
            q2[i] = ctx.measure_overlaps(chiral=False)["D"][0, 0, :, 0, 0] ** 2
        ti, _ = analysis.integrated_autocorrelation_time(q2)
        t_steps = float(np.mean(ti))
        t_sweeps = t_steps * sweeps
        cost = t_sweeps * ns_l128                      # per spin, in ns: sweeps x time per update
        base = cost if base is None else base
        tau[label] = {"sweeps_per_step": sweeps, "tau_int_steps": round(t_steps, 2),
                      "tau_int_sweeps": round(t_sweeps, 1), "steps": n,
                      "reliable": bool(n >= 50 * t_steps),
                      "ns_per_update_L128": round(ns_l128, 6),
                      "time_per_uncorrelated_sample_vs_lattice": round(cost / base, 2)}
        ctx.close()
    out["tau"] = {"observable": "q_ab^2 of the 6 pairs of 4 replicas, L = 16, T = 0.2, H_r = 0.05",
                  "chains": tau}
    return out


def time_observables(ctx, reps=3):
    """Host wall time of one call of each measurement entry point (outside the
    timed steps): hsg_measure (energies, q, q(k)) and hsg_measure_overlaps (spin
    and chiral pair overlaps)."""
    out = {}
    for name, fn in (("hsg_measure", lambda: ctx.measure()),
                     ("hsg_measure_overlaps", lambda: ctx.measure_overlaps())):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        out[name] = round((time.perf_counter() - t0) * 1e3 / reps, 3)
    return out


def traffic_summary(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it is current."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(kernel_key)
        if not e:
            return None
        from paper_1204_6192_gb300 import build as b
        if e.get("source_hash") != b.source_hash():
            return None
        return e.get("dram_bytes_per_launch")
    except Exception:
        return None


def e2e_run(ctx, wl, torch, steps, via="checkpoint"):
    """Through the public API with host buffers; host wall clock around it.
    Every step uploads the chain's state from pinned host memory, runs
    hsg_step and reads the observables back (hsg_measure).  via="checkpoint":
    the state as the library's own blob (hsg_checkpoint_load: spins in their
    storage format plus the chain's permutations, temperatures, energies and
    counters); via="xyz": the spins as binary32 (x, y, z) (hsg_set_spins).
    Returns (seconds, host-to-device bytes per step, device-to-host bytes per step)."""
    obs_bytes = (ctx.n_samples * ctx.n_replicas * ctx.n_temps * (8 + 4) +
                 ctx.n_samples * ctx.n_temps * (9 + 54) * 8)
    if via == "checkpoint":
        n = ctx.checkpoint_size()
        pinned = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        host = pinned.numpy()
        ctx.checkpoint(out=host)
        upload, h2d = (lambda: ctx.restore(host)), n
    else:
        total = ctx.info().total_spins * 3
        pinned = torch.empty(total, dtype=torch.float32, pin_memory=True)
        host = pinned.numpy()
        ctx.get_spins(out=host)
        upload, h2d = (lambda: ctx.set_spins(host)), total * 4
    upload()
    ctx.step(1)
    ctx.measure()
    ctx.sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        upload()
        ctx.step(1)
        ctx.measure()
    ctx.sync()
    dt = time.perf_counter() - t0
    return dt, h2d, obs_bytes


class OracleSample:
    """The FP64 oracle as it stands, on this host's cores, on a bounded sample of
    the workload: the same lattice, couplings and storage codec, 16 of the
    systems (2 replicas x the 8 lowest temperatures).  One call of step() is one
    sweep; heat-bath and over-relaxation sweeps alternate in the 1:5 ratio of
    the step, with energies and a PT pass after every sixth sweep."""

    def __init__(self, wl, n_temps=8):
        import oracle
        from paper_1204_6192_gb300 import inputs
        oracle.build()
        self.threads = int(oracle.lib().orc_num_threads())
        smp = wl.samples[0]
        n_t = min(n_temps, len(smp.temps))
        sub = inputs.Sample(L=smp.L,
                            J=inputs.round_fp16(smp.J) if wl.j_fp16 else smp.J,
                            H=inputs.round_fp16(smp.H) if wl.j_fp16 else smp.H,
                            temps=smp.temps[:n_t])
        self.codec = "none" if wl.precision == "fp32" else wl.precision
        self.sim = oracle.OracleSim([sub], 2, wl.seed, codec=self.codec)
        self.W = 2 * n_t
        self.L = smp.L
        self.sweeps = 0

    def step(self):
        if self.sweeps % 6 == 0:
            self.sim.sweep_hb(1)
        else:
            self.sim.sweep_or(1)
        self.sweeps += 1
        if self.sweeps % 6 == 0:
            self.sim.pt_exchange()
        return self.W * self.L ** 3

    def describe(self, sweeps, updates, dt):
        return (f"L={self.L}, {self.codec} storage emulated, {self.W} systems, {sweeps} sweeps "
                f"(HB:OR 1:5, PT every 6), {updates} spin updates in {dt:.1f} s")


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: implementer
    and part numbers), with the core count."""
    import platform
    name = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
        for key in ("model name", "CPU part"):
            vals = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith(key)]
            if vals:
                name = vals[0] if key == "model name" else f"Arm CPU part {vals[0]}"
                break
    except OSError:
        pass
    return f"{name or platform.processor() or 'unknown'} ({platform.machine()}, {os.cpu_count()} cores)"


def cpu_baseline(wl, max_seconds=20.0):
    ob = OracleSample(wl)
    updates = 0
    t0 = time.perf_counter()
    n = 0
    while n < 6 or time.perf_counter() - t0 < max_seconds:
        updates += ob.step()
        n += 1
        if time.perf_counter() - t0 > 3 * max_seconds:
            break
    dt = time.perf_counter() - t0
    out = {"value": round(dt * 1e9 / updates, 4), "unit": UNIT,
           "cores": min(ob.threads, ob.W), "kind": "oracle",
           "sample": ob.describe(n, updates, dt), "cpu": cpu_model()}
    # the same oracle on one core (the setting of the paper's serial CPU figures),
    # one step's sweeps (1 HB + 5 OR + PT) of 2 of the systems
    import oracle
    one = OracleSample(wl, n_temps=1)
    oracle.lib().orc_set_num_threads(1)
    try:
        updates1 = 0
        t1 = time.perf_counter()
        for _ in range(6):
            updates1 += one.step()
        dt1 = time.perf_counter() - t1
    finally:
        oracle.lib().orc_set_num_threads(ob.threads)
    out["single_core"] = {"value": round(dt1 * 1e9 / updates1, 4), "unit": UNIT,
                          "sample": one.describe(6, updates1, dt1)}
    return out


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_1204_6192_gb300 import build as cuda_build, inputs

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cuda_build.build()

    wl = shard_samples(inputs.workload(args.workload), rank)
    res, spins, sweeps = run_ours(args, wl, torch, dev, rank, world, args.measure_every)
    ctx, stream = res["ctx"], res["stream"]

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd and cvd.split(",")[local].strip().isdigit():
        gpu_index = int(cvd.split(",")[local])
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms, n_meas = timed_steps(ctx, stream, torch, args.steps, args.measure_every)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    rl_times = roofline(ctx, stream, torch, wl)
    clocks.stop()
    observables_ms = time_observables(ctx)
    ms = max_over_ranks(ms, torch, dev)

    info = ctx.info()
    updates_rank = sweeps * spins * args.steps
    updates = updates_rank * world
    value = whole_job_value(ms, updates_rank, world)
    peak, peak_kind = measured_peak()
    rl = roofline_entry(ctx, wl, rl_times, value, peak, peak_kind)

    line = {
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "L": wl.samples[0].L, "n_samples": len(wl.samples),
                   "replicas": wl.n_replicas, "temps": wl.n_temps, "spins": spins,
                   "storage": wl.precision, "couplings": "fp16" if wl.j_fp16 else "fp32",
                   "step": f"{wl.n_hb} HB + {wl.n_or} OR + energies + PT, measure every "
                           f"{args.measure_every}",
                   "l2": "state larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                   "schedule": schedule_of(info)},
        "spin_updates_per_s": round(updates / (ms * 1e-3), 1),
        "gpu_launches": args.steps * launches_per_step(info, wl) + n_meas * 2,
        "roofline": rl,
        "clocks": clocks.summary(),
        "observables_ms": observables_ms,
    }

    if not args.no_e2e:
        k = min(args.steps, 20)
        dt, h2d, d2h = e2e_run(ctx, wl, torch, k)
        dx, hx, _ = e2e_run(ctx, wl, torch, min(k, 10), via="xyz")
        line["e2e"] = {"value": round(dt * 1e9 / (sweeps * spins * k), 6), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": k,
                       "api": "hsg_checkpoint_load(pinned host blob: the chain state, spins in their "
                              "storage format) + hsg_step + hsg_measure(host)",
                       "xyz_upload": {"value": round(dx * 1e9 / (sweeps * spins * min(k, 10)), 6),
                                      "h2d_bytes_per_step": hx,
                                      "api": "hsg_set_spins(pinned host binary32 xyz) + hsg_step + "
                                             "hsg_measure(host)"}}
    ctx.close()

    configs = {}
    if not args.no_extras and world == 1:
        # the paper's own benchmark (Table 1: 256 systems of L = 32 at T = 100, FP32), with its
        # GTX 480 figures beside ours for context
        paper = {"table1_hb100or": 0.29, "table1_hb10or": 0.45, "table1_hb": 2.23, "table1_or": 1.30}
        t1 = {}
        for name, ref_ns in paper.items():
            w2 = inputs.workload(name)
            r2, sp2, sw2 = run_ours(args, w2, torch, dev, rank, world, 0)
            k2 = 10 if w2.n_or >= 100 else 30
            ms2, _ = timed_steps(r2["ctx"], r2["stream"], torch, k2, 0)
            v = ms2 * 1e6 / (sw2 * sp2 * k2)
            t1[name] = {"step": f"{w2.n_hb} HB + {w2.n_or} OR", "value": round(v, 6), "unit": UNIT,
                        "paper_gtx480_ns": ref_ns, "ratio_paper_over_ours": round(ref_ns / v, 1)}
            r2["ctx"].close()
        line["paper_table1_config"] = t1
        line["multihit"] = multihit_extras(torch, dev, inputs, value)
        # every production shape of the method, one compact entry each (L2-resident
        # states are timed with L2 flushed before every step)
        for name in ("L8_plain", "L32_fp32", "L64_fp16", "L64_angle16", "batch512_mixedL",
                     "L128_fp32", "L128_bf16", "L128_oct16", "L128_yx4"):
            configs[name] = config_line(args, name, torch, dev, peak)

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl)
    if configs:
        configs[args.workload] = {"ns": line["value"], "ms_step": line["ms_per_step"],
                                  "or_frac": rl["frac"], "schedule": schedule_of(info, short=True),
                                  "l2": "> L2"}
        line["configs"] = configs
        if "L128_fp32" in configs and args.workload == "L128_fp16":
            line["vs_plain_fp32"] = {
                "L128": round(configs["L128_fp32"]["ns"] / line["value"], 3),
                "note": "plain FP32 ns / compressed ns per update on the same lattice, same GPU"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def schedule_of(info, short=False):
    persistent = info.variant == 2
    kind = SWEEP_NAMES.get(info.sweep_kernel, "half")
    if short:
        return (("persistent" if persistent else "graph") + f"/gpt{info.chunks_per_thread}"
                + f"/p{info.n_passes}" + ("" if kind == "half" else f"/{kind}"))
    or_sweep = {"half": "one launch per half-sweep",
                "staged": "one launch per half-sweep, neighbour rows staged in shared memory",
                "fused": "fused (one launch per sweep, through shared memory)",
                "wave": "wave (one launch per sweep, odd blocks trailing even blocks in L2)"}[kind]
    out = {"variant": "persistent" if persistent else "two_pass (CUDA graph)",
           "chunks_per_thread": info.chunks_per_thread, "passes": info.n_passes,
           "or_sweep": or_sweep}
    if kind == "fused":
        out.update({"fused_band_rows": info.fused_band_rows, "fused_items": info.fused_items})
    if kind == "wave":
        out.update({"wave_lag_blocks": info.wave_lag})
    return out


def launches_per_step(info, wl):
    """Kernel launches of one step: the sweeps (two per sweep and pass, one per
    fused sweep), the energy sums' first level and the PT pass with the sums'
    last level (one launch for up to 4096 systems in all, else two)."""
    if info.variant == 2:
        return 1
    tail = 2 if info.n_samples * info.Wp <= 4096 else 3
    if info.sweep_kernel == 2 and info.n_passes == 1:
        pairs = (wl.n_or - 1) // 2
        return 2 * wl.n_hb + 2 * pairs + 2 * (wl.n_or - 2 * pairs) + tail
    if info.sweep_kernel == 3:
        return info.n_passes * (2 * wl.n_hb + wl.n_or) + tail
    return info.n_passes * 2 * (wl.n_hb + wl.n_or) + tail


def roofline_entry(ctx, wl, rl, value_ns, peak, peak_kind):
    """Roofline of the dominant kernel, the over-relaxation sweep, on the bytes
    the method must move (the fused one-pass count: each spin read and written
    once per sweep).  With the fused kernel one launch is a whole sweep; the
    half-sweep kernel is reported beside it, also against the two-pass byte
    count.  step_frac compares the whole step with the time the fused bytes of
    every update would take at the peak."""
    ms_or, kind, ms_half, ms_hb = rl
    A_half = algorithmic_half_sweep_bytes(ctx, wl, fused=True)
    A2 = algorithmic_half_sweep_bytes(ctx, wl, fused=False)
    A = A_half if kind in ("half", "staged") else 2 * A_half
    achieved = A / (ms_or * 1e-3) / 1e9
    key = {"half": "or_half_sweep", "fused": "fused_sweep", "wave": "wave_sweep",
           "staged": "staged_half_sweep"}[kind]
    traffic = traffic_summary(f"{key}_{wl.precision}")
    floor_ns = bytes_per_update(wl, ctx.W, fused=True) / peak      # ns per update at the peak
    name = {"half": "k_half_sweep OR", "fused": "k_fused_or (one sweep)",
            "wave": "k_wave_sweep OR (one sweep)", "staged": "k_staged_half OR"}[kind]
    return {"bound": "hbm",
            "kernel": f"{name} {wl.precision}",
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": traffic,
            "algorithmic_bytes_per_launch": A,
            "traffic_over_algorithmic": round(traffic / A, 3) if traffic else None,
            "ms_per_launch": round(ms_or, 5),
            "step_frac": round(floor_ns / value_ns, 4),
            "half_sweep": {"ms_per_launch": round(ms_half, 5),
                           "frac": round(A_half / (ms_half * 1e-3) / 1e9 / peak, 4),
                           "frac_two_pass": round(A2 / (ms_half * 1e-3) / 1e9 / peak, 4)},
            "hb_ms_per_launch": round(ms_hb, 5)}


def config_line(args, name, torch, dev, peak):
    """One production shape: ns per spin update of its step (with the overlap
    measurement every 10th step), its schedule and the OR kernel's fraction of
    the HBM peak on the fused bytes."""
    from paper_1204_6192_gb300 import inputs
    w2 = inputs.workload(name)
    state = sum(s.L ** 3 for s in w2.samples) * w2.n_replicas * w2.n_temps * SPIN_BYTES[w2.precision]
    flush = state < 256 * 1024 * 1024
    r2, sp2, sw2 = run_ours(args, w2, torch, dev, 0, 1, args.measure_every)
    buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev) if flush else None
    k2 = 30 if flush else 20
    ms2, _ = timed_steps(r2["ctx"], r2["stream"], torch, k2, args.measure_every, flush=buf)
    ms_or, kind, _, _ = roofline(r2["ctx"], r2["stream"], torch, w2, half=False)
    A = algorithmic_half_sweep_bytes(r2["ctx"], w2, fused=True) * (1 if kind in ("half", "staged") else 2)
    out = {"ns": round(ms2 * 1e6 / (sw2 * sp2 * k2), 6), "ms_step": round(ms2 / k2, 4),
           "or_frac": round(A / (ms_or * 1e-3) / 1e9 / peak, 3),
           "schedule": schedule_of(r2["ctx"].info(), short=True),
           "l2": "flushed" if flush else "> L2"}
    r2["ctx"].close()
    del buf
    return out


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    """Each step is one sweep of the oracle on the bounded sample above; host
    wall clock per step; mean over the timed steps."""
    if rank != 0:
        return
    from paper_1204_6192_gb300 import inputs
    wl = inputs.workload(args.workload)
    ob = OracleSample(wl)
    for _ in range(args.warmup):
        ob.step()
    updates = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        updates += ob.step()
    dt = time.perf_counter() - t0
    value = dt * 1e9 / updates
    sample = ob.describe(args.steps, updates, dt)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "L": wl.samples[0].L, "storage": wl.precision,
                       "step": "one oracle sweep of a 16-system sample (HB:OR 1:5, PT every 6)"},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT,
                             "cores": min(ob.threads, ob.W), "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
