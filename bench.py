"""Throughput of the facet-to-IQ echo path on B300.

One step = one harm_echo_accumulate call over the whole workload: every facet of
the 4 km x 2 km wave scene (2000 x 1000 facets of 2 m), every pulse of the burst
(2048 at 1700 Hz) and every receive channel (Harmony A and B x 3 phase centres),
i.e. 2.4576e10 facet-pulse-channel contributions, spread by the 8-tap
Kaiser-sinc into 6 x 2048 x 4096 complex64 IQ samples.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import harm_scenes as hs  # noqa: E402

METRIC = "facet·pulse·channel contributions/s at stated IQ error vs FP64 oracle; adjoint/fwd ratio"
UNIT = "contributions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--pulses", type=int, default=2048, help="burst length of the scene")
    ap.add_argument("--window", type=int, default=0,
                    help="pulses per step (0 = the whole burst); for the slow FP64 form")
    ap.add_argument("--cpu-pulses", type=int, default=16,
                    help="pulses in the oracle sample, spread over the burst (16 pulses: ~45 s on 16 host cores)")
    ap.add_argument("--ref-pulses", type=int, default=2,
                    help="pulses per step of the reference arm (2 pulses: ~5 s on 16 host cores)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-scene batched measurement")
    ap.add_argument("--no-generator", action="store_true", help="skip the standalone facet-generator timing")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the timing of the surface and scattering variants")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain FP64 and FP32 legs (windows of the headline scene)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the arithmetic-pipe microbenchmarks")
    ap.add_argument("--error-report", action="store_true",
                    help="instead of timing: the mixed path's errors on the 20 x 5 km scene over the 1000-pulse "
                         "subset (every 4th pulse), against the plain FP64 GPU path, which is itself checked "
                         "against the oracle on two of those pulses")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# Algorithmic FP32 work per contribution, frozen from the formulation before any
# tuning: the accumulator's per-(facet, pulse, channel) arithmetic (geometry,
# patterns, NRCS, phase, 8 taps, bin add: 150 flops) plus the surface generator's
# direct synthesis of (eta, eta_x, eta_y) from 256 components (1536 FMA = 3072
# flops per facet and pulse), shared by the channels.
ALGO_FLOPS_ACCUMULATOR = 150.0
ALGO_FLOPS_GENERATOR_PER_FACET_PULSE = 3072.0
# What the kernel executes per contribution, from the instruction-mix counters on
# the 512-pulse capture of the headline scene (FFMA2 = 4 flops, FFMA / FMUL2 /
# FADD2 = 2, FMUL / FADD = 1; per contribution 40.33 FFMA2 + 0.50 FFMA + 13.88 FMUL2
# + 2.43 FMUL + 8.55 FADD2 + 1.48 FADD): the time-Taylor generator replaces the
# direct synthesis, so this is far below the algorithmic count.
EXECUTED_FLOPS_PER_CONTRIBUTION = 211.1
# All instructions issued per contribution (thread level, same capture).
INSTR_PER_CONTRIBUTION = 175.7
# DRAM bytes (read + write) of one headline launch (2048 pulses), from one ncu
# capture of dram__bytes_read.sum + dram__bytes_write.sum, and the SHA-256 of the
# kernel sources' code (comments and blank lines dropped) it was taken on: the
# figure is reported only while they match.
TRAFFIC_BYTES = 80954624 + 26728704
TRAFFIC_PULSES = 2048
TRAFFIC_SOURCES = ("echo_mixed.cuh", "harm_kernels.cuh", "harm_internal.cuh")
TRAFFIC_SHA256 = "5b2b069a24698c209b8dcd9a83b6c320bd15dc510339c1fae6af99a20396cd26"


def _code_lines(raw):
    """Source text without // comments and blank lines: what the compiler sees of
    the kernel sources (a comment edit does not invalidate the capture)."""
    out = []
    for line in raw.decode().splitlines():
        i = line.find("//")
        if i >= 0:
            line = line[:i]
        line = line.rstrip()
        if line:
            out.append(line)
    return ("\n".join(out) + "\n").encode()


def captured_traffic(np_step):
    """DRAM bytes per launch from the stored capture, or None when the launch
    differs from the captured one or the kernel code changed since."""
    import hashlib
    if np_step != TRAFFIC_PULSES:
        return None
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2405_09938_b300", "csrc")
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(_code_lines(fh.read()))
    return float(TRAFFIC_BYTES) if h.hexdigest() == TRAFFIC_SHA256 else None


def max_over_ranks(total_ms, dist=None, device="cpu"):
    """Slowest rank's timed total (ms): the replicas' common clock."""
    if dist is None:
        return float(total_ms)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, units_per_rank, steps, total_ms):
    """Whole-job throughput of `world` independent replicas: all ranks' units over
    the slowest rank's time."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return None


def run_oracle_sample(desc, n_pulses_sample):
    import oracle
    pulses = sample_pulses(desc["n_pulses"], n_pulses_sample)
    t0 = time.perf_counter()
    iq = oracle.echo(desc, pulses)
    dt = time.perf_counter() - t0
    units = hs.n_facets(desc) * len(pulses) * len(desc["rx"])
    return {"pulses": pulses, "iq": iq, "seconds": dt, "units": units, "cores": oracle.num_threads()}


def run_oracle_single_core():
    """The oracle on one host core: the headline scene's geometry, waves and 6
    channels on a 400 x 200 facet patch (same work per contribution), 2 pulses."""
    import oracle
    d = hs.ati_scene(nx=400, ny=200)
    pulses = [0, d["n_pulses"] // 2]
    prev = oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.echo(d, pulses)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(prev)
    units = hs.n_facets(d) * len(pulses) * len(d["rx"])
    return {"value": units / dt, "unit": UNIT, "cores": 1,
            "sample": "2 pulses x 400 x 200 facets x %d channels of the headline scene's setup (%.1f s)" % (
                len(d["rx"]), dt)}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    desc = hs.ati_scene(n_pulses=args.pulses)
    samples = []
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not repeated
    for _ in range(args.steps):
        samples.append(run_oracle_sample(desc, args.ref_pulses))
    secs = sum(s["seconds"] for s in samples)
    units = sum(s["units"] for s in samples)
    value = units / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "ati_4x2km_2048p_6ch", "facets": hs.n_facets(desc),
                   "pulses": desc["n_pulses"], "channels": len(desc["rx"]), "range_samples": desc["n_range"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": samples[0]["cores"], "kind": "oracle",
                         "sample": "%d pulse(s) x all %d facets x %d channels per step" % (
                             args.ref_pulses, hs.n_facets(desc), len(desc["rx"]))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.error_report:
        error_report(args)
        return

    import torch
    from paper_2405_09938_b300 import harm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prec = {"mixed": harm.HARM_PREC_MIXED, "fp64": harm.HARM_PREC_FP64, "fp32": harm.HARM_PREC_FP32}[args.precision]
    cdt = torch.complex128 if prec == harm.HARM_PREC_FP64 else torch.complex64
    desc = hs.ati_scene(n_pulses=args.pulses)
    nc, nr = len(desc["rx"]), desc["n_range"]
    np_step = desc["n_pulses"] if args.window <= 0 else min(args.window, desc["n_pulses"])
    n0_step = (desc["n_pulses"] - np_step) // 2
    units = hs.n_facets(desc) * np_step * nc

    stream = torch.cuda.current_stream()
    scene = harm.harm_scene_create(desc, prec, stream)
    iq = torch.empty((nc, np_step, nr), dtype=cdt, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step(zero=True):
        harm.harm_echo_accumulate(scene, n0_step, np_step, iq, zero_first=zero)

    for _ in range(args.warmup):
        step()
    harm.harm_scene_sync(scene)

    # -- timed region: K steps, device time by CUDA events, L2 flushed between steps
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    harm.harm_scene_sync(scene)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = replica_value(world, units, args.steps, total_ms)

    # -- roofline of the accumulator kernel alone (no memset), same stream
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(1, args.steps))]
    for a, b in kev:
        flush.zero_()
        a.record(stream)
        step(zero=False)
        b.record(stream)
    torch.cuda.synchronize()
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)

    # -- end to end through the public API with host buffers: scene creation
    # (host precompute + table upload) and the echo written to pinned host memory
    # by harm_echo_accumulate_host (pulse blocks copied out while the next block
    # is computed)
    host_iq = torch.empty((nc, np_step, nr), dtype=cdt, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = 0
    create_s = 0.0
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        sc = harm.harm_scene_create(desc, prec, stream)
        if not h2d:
            h2d = _scene_table_bytes(desc, prec, harm.harm_scene_query(sc)["pulse_batch"])
        create_s += time.perf_counter() - ta
        harm.harm_echo_accumulate_host(sc, n0_step, np_step, host_iq)
        harm.harm_scene_sync(sc)
        sc.close()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    create_s /= e2e_steps
    d2h = host_iq.numel() * host_iq.element_size()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    algo_per_unit = ALGO_FLOPS_ACCUMULATOR + ALGO_FLOPS_GENERATOR_PER_FACET_PULSE / nc
    flops = algo_per_unit * units
    peaks = measured_peaks()
    sm_max = (peaks or {}).get("sm_max_mhz", 2032.0)
    fp32_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, unit counts x max SM clock
    achieved = flops / (kern_ms * 1e-3) / 1e12
    executed = EXECUTED_FLOPS_PER_CONTRIBUTION * units / (kern_ms * 1e-3) / 1e12
    issue_peak = 148 * 4 * 32 * sm_max * 1e6  # thread instructions / s
    issue_frac = INSTR_PER_CONTRIBUTION * units / (kern_ms * 1e-3) / issue_peak

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {harm.HARM_PREC_MIXED: "f32+f64", harm.HARM_PREC_FP64: "f64"}.get(prec, "f32"),
        "data": "synthetic",
        "config": {"workload": "ati_4x2km_2048p_6ch", "facets": hs.n_facets(desc), "pulses": np_step,
                   "channels": nc, "range_samples": nr, "precision": args.precision,
                   "output": "complex64" if cdt == torch.complex64 else "complex128",
                   "l2": "flushed between steps (256 MiB write); IQ output %.0f MB" % (d2h / 1e6),
                   "replicas": world},
        "roofline": {"bound": "alu", "achieved": achieved if prec == harm.HARM_PREC_MIXED else None,
                     "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak if prec == harm.HARM_PREC_MIXED else None,
                     "traffic": captured_traffic(np_step) if prec == harm.HARM_PREC_MIXED else None,
                     "kernel": "accumulate_mixed_kernel" if prec == harm.HARM_PREC_MIXED else "accumulate_plain_kernel",
                     "kernel_ms": kern_ms, "flops_per_contribution": algo_per_unit,
                     "flops_basis": "algorithmic: %.0f accumulator (Rx pattern and NRCS counted per channel; "
                                    "the kernel evaluates them once per receive antenna and shares them between "
                                    "its phase centres, hence frac slightly above 1) + %.0f / %d channels "
                                    "generator (direct 256-component synthesis) per contribution" % (
                                        ALGO_FLOPS_ACCUMULATOR, ALGO_FLOPS_GENERATOR_PER_FACET_PULSE, nc),
                     "peak_basis": "148 SM x 128 FP32 lanes x 2 x %.0f MHz (max SM clock)" % sm_max,
                     "executed_flops_per_contribution": EXECUTED_FLOPS_PER_CONTRIBUTION,
                     "executed_tflops": executed if prec == harm.HARM_PREC_MIXED else None,
                     "executed_frac": executed / fp32_peak if prec == harm.HARM_PREC_MIXED else None,
                     "issue_frac": issue_frac,
                     "issue_basis": "%.1f thread instructions per contribution vs 148 SM x 4 x 32 per clock"
                                    % INSTR_PER_CONTRIBUTION},
        "clocks": clk,
        "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": "harm_scene_create + harm_echo_accumulate_host (IQ streamed to pinned host memory "
                        "in pulse blocks) + harm_scene_sync",
                "ms_per_step": e2e_s * 1e3, "scene_create_ms": create_s * 1e3},
        "gpu_launches": args.steps * _launches_per_step(desc, prec, np_step),
    }
    cpu_pulses = sample_pulses(desc["n_pulses"], args.cpu_pulses)
    if prec == harm.HARM_PREC_MIXED and not args.no_peaks:
        pk = measure_peaks()
        line["peaks_measured"] = pk
        ffma = pk["ffma_tflops"]
        line["roofline"]["peak_measured"] = ffma
        line["roofline"]["peak_measured_basis"] = "FP32 FMA chains (libharm_peaks), %s" % pk["basis"]
        line["roofline"]["frac_of_measured"] = achieved / ffma
        line["roofline"]["executed_frac_of_measured"] = executed / ffma
    if prec == harm.HARM_PREC_MIXED and not args.no_plain:
        # windows of the same scene that start at an oracle sample pulse near the
        # middle of the burst, so that their IQ error is measured on it
        mid = min(cpu_pulses, key=lambda p: abs(p - desc["n_pulses"] // 2))
        line["fp64"] = measure_plain(args, stream, flush, harm.HARM_PREC_FP64, desc, mid, 64)
        line["fp32"] = measure_plain(args, stream, flush, harm.HARM_PREC_FP32, desc, mid, 256)
        mixed_rate = units / (kern_ms * 1e-3)
        line["vs_fp64"] = mixed_rate / line["fp64"]["value"]
        line["vs_fp64_basis"] = ("mixed-path kernel rate on the full burst over the plain FP64 kernel rate on a "
                                 "64-pulse window of the same scene (contributions/s, CUDA events)")
    if prec == harm.HARM_PREC_MIXED and not args.no_adjoint:
        line["adjoint"] = measure_adjoint(args, stream, flush)
    if prec == harm.HARM_PREC_MIXED and not args.no_batched:
        line["batched"] = measure_batched(args, stream)
    if prec == harm.HARM_PREC_MIXED and not args.no_variants:
        line["variants"] = measure_variants(args, stream, flush)
    if prec == harm.HARM_PREC_MIXED and not args.no_generator:
        line["generator"] = measure_generator(args, stream, flush)
    if not args.no_cpu:
        cpu = run_oracle_sample(desc, args.cpu_pulses)
        # IQ error of the GPU path on the sampled pulses
        sel = [p - n0_step for p in cpu["pulses"] if n0_step <= p < n0_step + np_step]
        if sel:
            got = host_iq.numpy()[:, sel, :]  # the end-to-end leg's IQ: one zeroed run
            want = cpu["iq"][:, [i for i, p in enumerate(cpu["pulses"]) if n0_step <= p < n0_step + np_step], :]
            err, pe = iq_errors(got, want)
            line["iq_rel_rms"] = err
            line["iq_peak_err"] = pe
            line["iq_error_sample"] = "%d pulses %s spread over the burst, all channels and range samples" % (
                len(sel), sel)
        for leg in ("fp64", "fp32"):
            if leg in line and line[leg].get("_iq") is not None:
                g = line[leg].pop("_iq")
                i = cpu["pulses"].index(line[leg]["window"][0])
                err, pe = iq_errors(g, cpu["iq"][:, [i], :])
                line[leg]["iq_rel_rms"] = err
                line[leg]["iq_peak_err"] = pe
                line[leg]["iq_error_sample"] = "pulse %d, all channels and range samples" % cpu["pulses"][i]
        line["cpu_baseline"] = {"value": cpu["units"] / cpu["seconds"], "unit": UNIT, "cores": cpu["cores"],
                                "kind": "oracle",
                                "sample": "%d pulse(s) of the workload x %d facets x %d channels (%.1f s)" % (
                                    len(cpu["pulses"]), hs.n_facets(desc), nc, cpu["seconds"]),
                                "single_core": run_oracle_single_core()}
    for leg in ("fp64", "fp32"):
        if leg in line:
            line[leg].pop("_iq", None)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def error_report(args):
    """Errors of the mixed path on the 20 km x 5 km scene (10000 x 2500 facets,
    4096 pulses, Harmony A x 3 phase centres): one launch over the whole burst,
    compared on the 1000 pulses 0, 4, ..., 3996 with the plain FP64 GPU path (one
    launch per pulse), whose own error against the FP64 oracle is measured on two
    of those pulses. Reports the IQ relative RMS over the subset and its worst
    pulse, the largest per-element error relative to the row peak, and the ATI
    interferometric phase bias of the three phase-centre pairs."""
    import torch
    from paper_2405_09938_b300 import harm
    import oracle
    d = hs.mixed_scene()
    nc, npul, nr = len(d["rx"]), d["n_pulses"], d["n_range"]
    pulses = list(range(0, 4000, 4))
    assert max(pulses) < npul
    t0 = time.perf_counter()
    sm = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    iq = torch.zeros((nc, npul, nr), dtype=torch.complex64, device="cuda")
    harm.harm_echo_accumulate(sm, 0, npul, iq)
    harm.harm_scene_sync(sm)
    sm.close()
    mixed = iq.cpu().numpy()[:, pulses, :].astype(np.complex128)
    del iq
    torch.cuda.empty_cache()
    t_mixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    s64 = harm.harm_scene_create(d, harm.HARM_PREC_FP64)
    buf = torch.zeros((nc, 1, nr), dtype=torch.complex128, device="cuda")
    ref = np.zeros((nc, len(pulses), nr), dtype=np.complex128)
    for i, p in enumerate(pulses):
        harm.harm_echo_accumulate(s64, p, 1, buf)
        ref[:, i, :] = buf[:, 0, :].cpu().numpy()
    harm.harm_scene_sync(s64)
    s64.close()
    t_fp64 = time.perf_counter() - t0
    t0 = time.perf_counter()
    chk = [pulses[250], pulses[750]]
    want = oracle.echo(d, chk)
    t_oracle = time.perf_counter() - t0
    fp64_err, fp64_pe = iq_errors(ref[:, [250, 750], :], want)
    mix_vs_oracle, _ = iq_errors(mixed[:, [250, 750], :], want)
    err, pe = iq_errors(mixed, ref)
    per_pulse = np.sqrt(np.sum(np.abs(mixed - ref) ** 2, axis=(0, 2)) / np.sum(np.abs(ref) ** 2, axis=(0, 2)))

    def bias(a, b):
        g = np.angle(np.sum(mixed[a] * np.conj(mixed[b])))
        w = np.angle(np.sum(ref[a] * np.conj(ref[b])))
        return float((g - w + np.pi) % (2 * np.pi) - np.pi)

    out = {"report": "mixed-path errors, 20 x 5 km scene, 1000-pulse subset",
           "workload": "mixed_20x5km_4096p_3ch", "facets": hs.n_facets(d), "pulses": npul, "channels": nc,
           "subset": "pulses 0, 4, ..., 3996 (1000), all channels and %d range samples" % nr,
           "reference": "plain FP64 GPU path (HARM_PREC_FP64), one launch per pulse",
           "iq_rel_rms": err, "iq_peak_err": pe,
           "iq_rel_rms_worst_pulse": float(per_pulse.max()), "iq_rel_rms_median_pulse": float(np.median(per_pulse)),
           "ati_phase_bias_rad": {"(0,1)": bias(0, 1), "(1,2)": bias(1, 2), "(0,2)": bias(0, 2)},
           "fp64_vs_oracle": {"pulses": chk, "iq_rel_rms": fp64_err, "iq_peak_err": fp64_pe},
           "mixed_vs_oracle_same_pulses": mix_vs_oracle,
           "seconds": {"mixed_burst": t_mixed, "fp64_subset": t_fp64, "oracle_2_pulses": t_oracle}}
    print(json.dumps(out), flush=True)


def sample_pulses(n_pulses, count):
    """Oracle sample: `count` pulses spread evenly over the burst."""
    return sorted(set(int(round(v)) for v in np.linspace(0, n_pulses - 1, count)))


def iq_errors(got, want):
    """IQ relative RMS and the largest per-element error relative to each (channel,
    pulse) row's peak."""
    err = float(np.sqrt(np.sum(np.abs(got - want) ** 2) / np.sum(np.abs(want) ** 2)))
    g = got.reshape(-1, got.shape[-1])
    w = want.reshape(-1, want.shape[-1])
    peak = np.abs(w).max(axis=1)
    rows = peak > 0
    pe = float((np.abs(g - w).max(axis=1)[rows] / peak[rows]).max()) if rows.any() else None
    return err, pe


def measure_peaks():
    """FP32 FMA, packed FP32x2 FMA, FP64 FMA and __sinf rates of this GPU
    (libharm_peaks: independent chains, 8 CTAs of 256 threads per SM, best of 5
    CUDA-event-timed launches), with the SM clock sampled while they ran."""
    from paper_2405_09938_b300 import peaks
    clocks = ClockSampler(0)
    clocks.start()
    out = {}
    for kind in ("ffma", "ffma2", "dfma", "sinf"):
        rate, ms, sms = peaks.measure(kind)
        out[kind] = {"rate": rate, "best_ms": ms}
    clk = clocks.stop()
    mhz = clk.get("sm_mhz") or 2032.0
    return {"ffma_tflops": out["ffma"]["rate"] / 1e12, "ffma2_tflops": out["ffma2"]["rate"] / 1e12,
            "dfma_tflops": out["dfma"]["rate"] / 1e12,
            "sinf_per_clk_per_sm": out["sinf"]["rate"] / (sms * mhz * 1e6),
            "sinf_per_s": out["sinf"]["rate"], "sms": sms, "clocks": clk,
            "basis": "independent chains, 8 CTAs x 256 threads per SM, best of 5 launches, SM clock median %s MHz"
                     % (clk.get("sm_mhz"),)}


def measure_plain(args, stream, flush, prec, desc, n0, npw):
    """The plain path of precision `prec` (every per-facet step in FP64 or in FP32)
    on a window of `npw` pulses of the headline scene starting at pulse n0: mean
    device time of harm_echo_accumulate over --steps runs after one warm-up, L2
    flushed before each; keeps the IQ of pulse n0 for the error against the
    oracle sample."""
    import torch
    from paper_2405_09938_b300 import harm
    cdt = torch.complex128 if prec == harm.HARM_PREC_FP64 else torch.complex64
    nc, nr = len(desc["rx"]), desc["n_range"]
    npw = min(npw, desc["n_pulses"] - n0)
    scene = harm.harm_scene_create(desc, prec, stream)
    iq = torch.empty((nc, npw, nr), dtype=cdt, device="cuda")
    times = []
    for i in range(1 + max(1, min(args.steps, 3))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        harm.harm_echo_accumulate(scene, n0, npw, iq)
        b.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            times.append(a.elapsed_time(b))
    harm.harm_scene_sync(scene)
    scene.close()
    ms = statistics.mean(times)
    units = hs.n_facets(desc) * npw * nc
    first = iq[:, 0:1, :].cpu().numpy().astype(np.complex128)
    del iq
    torch.cuda.empty_cache()
    return {"precision": "fp64" if prec == harm.HARM_PREC_FP64 else "fp32", "window": [n0, n0 + npw],
            "contributions": units, "ms": ms, "value": units / (ms * 1e-3),
            "output": "complex128" if cdt == torch.complex128 else "complex64", "_iq": first}


def measure_adjoint(args, stream, flush):
    """Forward and adjoint on the differentiable scene (2 km x 1 km, 1024 pulses,
    6 channels, 100 m cells): misfit to the IQ of a Gaussian-correlated current
    perturbation (0.1 m/s, 500 m); device time of harm_echo_accumulate and of
    harm_echo_adjoint, same stream, L2 flushed between calls."""
    import torch
    from paper_2405_09938_b300 import harm
    d = hs.adjoint_scene()
    c = d["cells"]
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED, stream)
    s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda")
    uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda")
    uvp = uv + torch.tensor(hs.current_perturbation(c["ncx"], c["ncy"], c["cell_m"]), device="cuda")
    nc, npul, nr = len(d["rx"]), d["n_pulses"], d["n_range"]
    tgt = torch.empty((nc, npul, nr), dtype=torch.complex64, device="cuda")
    harm.harm_scene_set_cells(scene, c["ncx"], c["ncy"], c["cell_m"], s0, uvp)
    harm.harm_echo_accumulate(scene, 0, npul, tgt)
    harm.harm_scene_set_cells(scene, c["ncx"], c["ncy"], c["cell_m"], s0, uv)
    iq = torch.empty_like(tgt)
    gs, guv = torch.zeros_like(s0), torch.zeros_like(uv)
    fwd, adj = [], []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        harm.harm_echo_accumulate(scene, 0, npul, iq)
        b.record(stream)
        r = iq - tgt
        gs.zero_()
        guv.zero_()
        flush.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        harm.harm_echo_adjoint(scene, 0, npul, r, gs, guv)
        c1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            fwd.append(a.elapsed_time(b))
            adj.append(c0.elapsed_time(c1))
    harm.harm_scene_sync(scene)
    units = hs.n_facets(d) * npul * nc
    f_ms, a_ms = statistics.mean(fwd), statistics.mean(adj)
    scene.close()
    return {"workload": "adj_2x1km_1024p_6ch_100m_cells", "contributions": units, "fwd_ms": f_ms,
            "adj_ms": a_ms, "adj_over_fwd": a_ms / f_ms, "fwd_value": units / (f_ms * 1e-3),
            "adj_value": units / (a_ms * 1e-3), "loss": float(torch.sum(torch.abs(r) ** 2).item()),
            "grad_uv_norm": float(torch.linalg.norm(guv).item())}


def measure_batched(args, stream):
    """48 uneven scenes (0.5 x 0.5 km .. 8 x 4 km, 256 .. 2048 pulses, 1024 .. 8192
    range samples, 6 channels each) as one persistent launch replayed from a CUDA
    graph, after the autotuner picked the launch shape (tile rows and time-Taylor
    window per size class, CTAs per SM). One untimed warm-up run, then the median
    of five timed replays (device time by CUDA events); then the same with the
    fixed default shape (16-row tiles, full windows, 2 CTAs per SM) for the
    tuner's gain."""
    import torch
    from paper_2405_09938_b300 import harm
    descs = hs.batch_scenes()
    t0 = time.perf_counter()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED, stream) for d in descs]
    create_s = time.perf_counter() - t0
    iqs = [torch.empty((len(d["rx"]), d["n_pulses"], d["n_range"]), dtype=torch.complex64, device="cuda")
           for d in descs]
    b = harm.harm_batch_create(scenes)
    t0 = time.perf_counter()
    harm.harm_batch_tune(b, iqs)
    tune_s = time.perf_counter() - t0
    cfg = harm.harm_batch_config(b)
    rows = cfg["rows"]

    def replays(k):
        harm.harm_batch_run(b, iqs)
        torch.cuda.synchronize()
        out = []
        for _ in range(k):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            harm.harm_batch_run(b, iqs)
            e.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(e))
        return out

    reps = replays(5)
    ms = statistics.median(reps)
    pb = harm.harm_scene_query(scenes[0])["pulse_batch"]
    harm.harm_batch_set_config(b, [16] * len(descs), [pb] * len(descs), 2)
    default_ms = statistics.median(replays(3))
    units = sum(hs.n_contributions(d) for d in descs)
    b.close()
    for sc in scenes:
        sc.close()
    del iqs
    torch.cuda.empty_cache()
    return {"workload": "batch_48_uneven_scenes_6ch", "scenes": len(descs), "contributions": units,
            "ms": ms, "ms_replays": reps, "value": units / (ms * 1e-3), "launches": 1, "graph": True,
            "tile_rows": {"8": rows.count(8), "16": rows.count(16)},
            "windows": {str(w): cfg["windows"].count(w) for w in sorted(set(cfg["windows"]))},
            "ctas_per_sm": cfg["ctas_per_sm"], "default_shape_ms": default_ms, "tuner_gain": default_ms / ms,
            "scene_create_s": create_s, "tune_s": tune_s}


def measure_generator(args, stream, flush):
    """The facet generator on its own (harm_facets_generate): states (eta, eta_x,
    eta_y) of every facet of the headline scene for the first 256 pulses (one
    time-Taylor window), written to HBM as float32 [256][3][n_facets] (6.14 GB);
    one warm-up, then the mean of three timed runs, L2 flushed before each. Bound
    by the HBM write stream."""
    import torch
    from paper_2405_09938_b300 import harm
    d = hs.ati_scene()
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED, stream)
    npw = harm.harm_scene_query(scene)["pulse_batch"]
    st = torch.empty((npw, 3, d["ny"], d["nx"]), dtype=torch.float32, device="cuda")
    times = []
    for i in range(4):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        harm.harm_facets_generate(scene, 0, npw, st)
        b.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            times.append(a.elapsed_time(b))
    harm.harm_scene_sync(scene)
    scene.close()
    ms = statistics.mean(times)
    nbytes = st.numel() * st.element_size()
    del st
    torch.cuda.empty_cache()
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs")
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": "ati_4x2km_states_%dp" % npw, "facet_pulses": hs.n_facets(d) * npw, "ms": ms,
            "value": hs.n_facets(d) * npw / (ms * 1e-3), "unit": "facet-pulse states/s",
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm if hbm else None,
                         "bytes": nbytes, "bytes_basis": "states written (float32, 3 fields); wave tables are "
                                                         "L2-resident"}}


def measure_variants(args, stream, flush):
    """The surface and scattering variants of Sec. III on one mid-size scene
    (2 km x 1 km, 512 pulses, 6 channels, 4096 range samples; 1.536e9
    contributions): device time of harm_echo_accumulate per variant (one warm-up,
    then the mean of two timed runs, L2 flushed before each), and the ratio to
    the plain scene."""
    import torch
    from paper_2405_09938_b300 import harm
    base = hs.ati_scene(n_pulses=512, nx=1000, ny=500, n_range=4096)
    variants = {
        "plain": base,
        "ar1_doppler": hs.ar1_speckle(base, tau_s=0.03, doppler_hz=12.0, epoch_pulses=8),
        "uv_grids": hs.uv_patterns(base),
        "hetero_512m": hs.hetero_sea(base, tile_m=512.0),
        "cwm": hs.choppy(base),
        "all": hs.uv_patterns(hs.choppy(hs.hetero_sea(
            hs.ar1_speckle(base, tau_s=0.03, doppler_hz=12.0, epoch_pulses=8), tile_m=512.0))),
    }
    nc, npul, nr = len(base["rx"]), base["n_pulses"], base["n_range"]
    iq = torch.empty((nc, npul, nr), dtype=torch.complex64, device="cuda")
    units = hs.n_contributions(base)
    out = {"workload": "ati_2x1km_512p_6ch", "contributions": units}
    for name, d in variants.items():
        scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED, stream)
        times = []
        for i in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            harm.harm_echo_accumulate(scene, 0, npul, iq)
            b.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                times.append(a.elapsed_time(b))
        harm.harm_scene_sync(scene)
        scene.close()
        ms = statistics.mean(times)
        out[name] = {"ms": ms, "value": units / (ms * 1e-3)}
    for name in variants:
        out[name]["vs_plain"] = out["plain"]["ms"] / out[name]["ms"]
    del iq
    torch.cuda.empty_cache()
    return out


def _launches_per_step(desc, prec, np_step):
    from paper_2405_09938_b300 import harm
    if prec == harm.HARM_PREC_MIXED:
        batches = math.ceil(np_step / 128) + 1
        return max(1, math.ceil(batches / 65535))
    return max(1, math.ceil(np_step / 65535))


def _scene_table_bytes(desc, prec, pulse_batch):
    """Bytes harm_scene_create uploads: pulse states (t, t_s and a 10-double
    antenna state) and per-channel receive states (antenna state, reduced phase,
    bin offset); the wave numbers and frequencies (kx, ky, omega, |k|) and the
    wave list of the phasor-table kernel (5 doubles; the tables themselves are
    computed on the device) per wave set; u-v grid descriptors and the flag
    words; for mixed scenes the time-Taylor tables: e^{-i omega t_c} per window
    of ``pulse_batch`` pulses (complex64), the real factors (float32, fields x 6
    orders) and the pulse offsets tau (float32)."""
    from paper_2405_09938_b300 import harm
    nw = desc["n_omega"] * desc["n_theta"]
    het = desc.get("hetero")
    nsw = nw * (int(np.asarray(het["u10"]).size) if het else 1)
    npul, nc = desc["n_pulses"], len(desc["rx"])
    pulse = npul * (8 * 2 + 8 * 10) + npul * nc * (8 * 10 + 16)
    waves = nsw * 4 * 8 + nsw * 5 * 8
    if prec == harm.HARM_PREC_MIXED:
        nf = 8 if desc.get("cwm") else 3
        waves += math.ceil(npul / pulse_batch) * nsw * 8 + nsw * nf * 6 * 4 + npul * 4
    return pulse + waves + (1 + nc) * 56 + 4 * 4


if __name__ == "__main__":
    main()
