"""Benchmark: one step = the whole hot path (bin -> criterion + 4D labelling -> per-feature
statistics) over the combustion-shaped workload: 256^3 fp32 field x 24 timesteps, 8M particles
with four attributes (temperature, mixture fraction, speed, age), criterion field > 0.5 AND mean
temperature above its 60th percentile AND mean mixture fraction in its [q20, q80] band, all edge
classes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--config 3]

Prints one JSON line. ``value`` is voxel-timesteps per second (Gvt/s) of the whole step with the
dataset resident in HBM (K steps timed with CUDA events, no per-kernel instrumentation);
``segment_only`` is the same metric for the segment query alone (msf_segment, criterion +
labelling), with its own roofline at the algorithmic bytes per voxel-timestep. ``e2e`` is the
step through the C ABI with host buffers (the host->device copy of the field and particles and
the device->host copy of the labels and the feature table inside every step). Per-kernel
figures come from a second pass of K steps with CUDA events around every launch. Under
torchrun each rank runs its own replica (the path has no exchange step for independent
workloads): weak scaling, value = all ranks' voxel-timesteps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gvoxel-timesteps/s per segment query (% HBM roofline); batched queries/s, p99"
UNIT = "Gvoxel-timesteps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from an ncu capture of
# the same kernel code on the same workload (profiles/kernels_mid_step.md): {(config, kernel):
# bytes}. An entry is removed whenever its kernel changes.
TRAFFIC = {
    # ncu DRAM bytes (read + write) of one launch, from a single-kernel capture of the unchanged
    # kernel (profiles/); combustion: the 4-timestep capture (--timesteps 4) scaled by 6 to the
    # 24-step launch (a launch's records and voxels grow in proportion to its field steps)
    (3, "k_feat_points"): (600_658_176 + 10_216_960) * 6,
}


def d2d_copy_gbs(dev, nbytes=1 << 31, reps=5):
    """A device-to-device copy of `nbytes` (torch copy_, CUDA events, median of `reps`): bytes
    read plus bytes written per second, beside the roofline's measured peak."""
    import torch
    n = nbytes // 4
    src = torch.empty(n, dtype=torch.float32, device=dev).fill_(1.0)
    dst = torch.empty_like(src)
    stream = torch.cuda.current_stream(dev)
    dst.copy_(src)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dst.copy_(src)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = sorted(ts)[len(ts) // 2]
    del src, dst
    torch.cuda.empty_cache()
    return round(2 * n * 4 / (ms * 1e-3) / 1e9, 1)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the context is open (the
    warm-up, the timed steps and the profiled pass); summary() reports the samples taken
    between two marks (the timed region) beside those of the whole session."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []
        self.marks = {}

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, name):
        self.marks[name] = time.perf_counter()

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    @staticmethod
    def _digest(lines):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return sm, mx, reasons

    def summary(self, start=None, end=None):
        t0 = self.marks.get(start, float("-inf"))
        t1 = self.marks.get(end, float("inf"))
        sm, mx, reasons = self._digest([ln for t, ln in self.lines if t0 <= t <= t1])
        ssm, smx, sreasons = self._digest([ln for _, ln in self.lines])
        if not ssm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm) if sm else statistics.median(ssm),
                "sm_max_mhz": max(mx) if mx else max(smx), "reasons": sorted(reasons | sreasons),
                "samples": len(sm),
                "session": {"samples": len(ssm), "sm_mhz_median": statistics.median(ssm),
                            "sm_mhz_min": min(ssm), "reasons": sorted(sreasons)}}


# per-kernel algorithmic bytes: the bytes each kernel must move through HBM per launch by the
# definition of its step (inputs it alone reads, outputs it alone writes); traffic of
# intermediate state (sorted records, segment masks, union-find tables) is not counted
def algorithmic_bytes(wl, n_pred_arrays, keep_sumq=False, fused_criterion=False):
    T, nz, ny, nx = wl.field.shape
    V = nx * ny * nz
    tw = wl.t1 - wl.t0
    P = wl.pos.shape[2]
    A = wl.attr.shape[1]
    crit = V * tw * 4 * n_pred_arrays                        # field + predicate arrays in
    return {
        "k_bin_keys": P * T * (12 + 4),                      # positions in, voxel keys out
        "k_bin_place": P * T * 4 * A,                        # attributes in
        "k_bin_reduce": V * T * (4 + 4 * A + (8 * A if keep_sumq else 0)),  # count + means out
        # the criterion's reads belong to its streaming pass, or to the tile pass that
        # evaluates it when the schedule fuses them
        ("k_tile" if fused_criterion else "k_mask"): crit,
        "k_links": P * tw * 4,                               # keys of the window in
        "k_final": V * tw * 4,                               # labels out
        "k_feat_vox": V * tw * 8,                            # labels + field in
        "k_feat_points": P * tw * (4 + 4 * A),               # keys + attributes of the window in
    }


def segment_bytes_per_vt(wl, n_pred_arrays):
    """Algorithmic bytes of one segment query per voxel-timestep: every distinct predicate
    array read once (field, count or one attribute's means), the labels written once, and the
    window's trajectory keys read once (4 P / V per step)."""
    T, nz, ny, nx = wl.field.shape
    V = nx * ny * nz
    P = wl.pos.shape[2]
    traj = 4.0 * P / V if (wl.edges & 4) and P else 0.0
    return 4.0 * n_pred_arrays + 4.0 + traj


def host_cpu():
    """Model name and logical core count of the host (lscpu, else os.cpu_count)."""
    model, cores = None, os.cpu_count()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() == "Model name" and model is None:
                model = v.strip()
            elif k.strip() == "CPU(s)":
                cores = int(v.strip())
    except Exception:
        pass
    return {"model": model, "logical_cores": cores}


def input_sha256(*arrays):
    """SHA-256 over the raw bytes of the generated inputs (host copies, in order)."""
    import hashlib
    h = hashlib.sha256()
    for a in arrays:
        h.update(memoryview(a.numpy()).cast("B"))
    return h.hexdigest()


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1903_12294_gb300 import build as libbuild
    from paper_1903_12294_gb300 import msf, replicas, synth

    world, rank, local = replicas.layout()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        libbuild.build()
    barrier = replicas.barrier
    barrier()

    wl = synth.make(args.config, device=dev, **({"T": args.timesteps} if args.timesteps else {}))
    T, nz, ny, nx = wl.field.shape
    V = nx * ny * nz
    tw = wl.t1 - wl.t0
    vt = V * tw
    stream = torch.cuda.current_stream(dev)
    ctx = msf.Context(local, stream)
    crit = msf.make_criteria(wl.t0, wl.t1, wl.preds, wl.edges)
    labels = torch.empty((tw, nz, ny, nx), dtype=torch.int32, device=dev)
    fcap = 1 << 20
    feats = torch.empty((fcap * msf.FEATURE_DTYPE.itemsize,), dtype=torch.uint8, device=dev)
    lib = msf.load_library()
    nf_out = msf.ctypes.c_int64(0)

    ctx.load(wl.field, wl.pos, wl.attr)
    tuning = None
    if args.schedule:
        # a fixed tile shape and schedule (to profile the configuration a tuning run chose)
        by, bz, bt, sched = (int(x) for x in args.schedule.split(","))
        ctx.set_tile(by, bz, bt)
        ctx.set_schedule(sched)
        tuning = {"fixed": [by, bz, bt, sched]}
    elif not args.no_tune:
        # tile shape and schedule of the query's segment pass picked by the library's
        # autotuner (untimed, before the warm-up; every choice gives the same labels)
        msf.msf_bin_particles(ctx.h, 0)
        tuning = msf.msf_autotune(ctx.h, crit, 3)
        tuning = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in tuning.items()}

    def step():
        msf.msf_bin_particles(ctx.h, 0)
        n = msf.msf_segment(ctx.h, crit, labels)
        st = lib.msf_extract_features(ctx.h, msf.ctypes.byref(crit), labels.data_ptr(),
                                      msf.MSF_DEVICE, feats.data_ptr(), msf.MSF_DEVICE, fcap,
                                      msf.ctypes.byref(nf_out))
        if st != 0:
            raise msf.MsfError(st, "msf_extract_features")
        return n

    def timed(fn, k):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1) / k, r

    with Clocks(local) as clk:
        for _ in range(args.warmup):
            n_features = step()
        torch.cuda.synchronize()
        # the headline: K steps, nothing instrumented
        clk.mark("timed_start")
        ms, n_features = timed(step, args.steps)
        clk.mark("timed_end")
        # the segment query alone (criterion + labelling, msf_segment with device labels)
        for _ in range(args.warmup):
            msf.msf_segment(ctx.h, crit, labels)
        seg_ms, _ = timed(lambda: msf.msf_segment(ctx.h, crit, labels), args.steps)
        seg_ms_long, _ = timed(lambda: msf.msf_segment(ctx.h, crit, labels),
                               max(args.steps, 200))
        # per-kernel split: K more steps with CUDA events around every launch (each on the
        # stream the kernel runs on)
        ctx.kernel_times(reset=True)
        ctx.profiling(True)
        ms_prof, _ = timed(step, args.steps)
        ktimes = ctx.kernel_times(reset=True)
        ctx.profiling(False)
    ms = replicas.max_over_ranks(ms, dev)
    value = replicas.weak_throughput(vt, ms, world) / 1e9
    launches_per_step = sum(n for _, n in ktimes.values()) // max(args.steps, 1)

    # dominant kernel and its roofline (per-launch CUDA-event durations from the profiled pass)
    npa = len({(s, a if s == 2 else 0) for s, a, *_ in wl.preds})
    fused = bool(msf.msf_get_tuning(ctx.h, crit)[3] & msf.MSF_SCHED_FUSED_CRITERION)
    abytes = algorithmic_bytes(wl, npa, fused_criterion=fused)
    peak, peak_kind = peaks()
    copy_gbs = d2d_copy_gbs(dev) if rank == 0 else None
    per_kernel = {}
    for k, (tot, nl) in ktimes.items():
        e = {"ms_per_step": round(tot / args.steps, 4), "launches_per_step": nl // max(args.steps, 1)}
        if abytes.get(k) and nl:
            # the kernel's algorithmic bytes of one step over its time in one step (a kernel may
            # launch more than once per step, e.g. a tile pass split in halves)
            gbs = abytes[k] / (tot / args.steps * 1e-3) / 1e9
            e.update({"algorithmic_bytes": abytes[k], "gb_per_s": round(gbs, 1),
                      "frac": round(gbs / peak, 4)})
        per_kernel[k] = e
    name, (tot_ms, nl) = max(ktimes.items(), key=lambda kv: kv[1][0])
    per_launch_ms = tot_ms / nl
    ab = abytes.get(name)
    roof = None
    if ab:
        ab = ab * args.steps / nl  # per launch: the step's bytes over its launches
        ach = ab / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": TRAFFIC.get((args.config, name)), "algorithmic_bytes_per_launch": ab,
                "avg_launch_ms": round(per_launch_ms, 5)}
    step_bytes = sum(abytes.values())
    step_roof = {"algorithmic_bytes": step_bytes,
                 "achieved_gb_per_s": round(step_bytes / (ms * 1e-3) / 1e9, 1),
                 "frac": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4)}
    bpv = segment_bytes_per_vt(wl, npa)
    seg_roof = {"bound": "hbm", "bytes_per_vt": round(bpv, 3),
                "achieved": round(bpv * vt / (seg_ms_long * 1e-3) / 1e9, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(bpv * vt / (seg_ms_long * 1e-3) / 1e9 / peak, 4)}

    # end to end through the C ABI with host buffers
    e2e = None
    hashes = None
    if not args.no_e2e:
        hf = wl.field.cpu().pin_memory()
        hp = wl.pos.cpu().pin_memory()
        ha = wl.attr.cpu().pin_memory()
        hl = torch.empty((tw, nz, ny, nx), dtype=torch.int32).pin_memory()
        # the feature table lands in pinned host memory too (pageable memory would copy at a
        # fraction of the link's rate)
        hfeat_t = torch.zeros((fcap * msf.FEATURE_DTYPE.itemsize,), dtype=torch.uint8).pin_memory()
        hfeat = hfeat_t.numpy().view(msf.FEATURE_DTYPE)
        if rank == 0:
            hashes = {"field": input_sha256(hf), "pos": input_sha256(hp), "attr": input_sha256(ha)}

        nseg_out = msf.ctypes.c_int64(0)

        def e2e_step():
            # load (host data streamed in chunks, binned as it arrives), bin, then labels and
            # features in one call whose host labels go down the link beside the feature passes
            ctx.load(hf, hp, ha)
            msf.msf_bin_particles(ctx.h, 0)
            st = lib.msf_segment_features(ctx.h, msf.ctypes.byref(crit), hl.data_ptr(),
                                          msf.MSF_HOST, msf.ctypes.byref(nseg_out),
                                          hfeat.ctypes.data, msf.MSF_HOST, fcap,
                                          msf.ctypes.byref(nf_out))
            if st != 0:
                raise msf.MsfError(st, "msf_segment_features")
            return int(nf_out.value)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nfe = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / args.steps * 1e3
        ms_e2e = max(e0.elapsed_time(e1) / args.steps, wall)
        ms_e2e = replicas.max_over_ranks(ms_e2e, dev)
        h2d = hf.numel() * 4 + hp.numel() * 4 + ha.numel() * 4
        d2h = hl.numel() * 4 + nfe * msf.FEATURE_DTYPE.itemsize
        e2e = {"value": round(replicas.weak_throughput(vt, ms_e2e, world) / 1e9, 3), "unit": UNIT,
               "ms_per_step": round(ms_e2e, 3), "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        del hf, hp, ha, hl, hfeat, hfeat_t

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)
    ctx.close()
    del labels, feats
    wl_name, wl_shape = wl.name, (nx, ny, nz, T, wl.pos.shape[2], wl.attr.shape[1])
    wl_desc = (wl.t0, wl.t1, wl.preds)
    del wl
    torch.cuda.empty_cache()
    clustering = None
    if rank == 0 and not args.no_cluster:
        # the paper's clustering on the mid workload (128^3 x 32, 1M points)
        mwl = synth.mid(device=dev)
        mctx = msf.Context(local, stream)
        mctx.load(mwl.field, mwl.pos, mwl.attr)
        mctx.bin()
        clustering, last = run_clustering(mctx, mwl, dev)
        clustering["post"] = run_post(mctx, mwl, dev, *last)
        del last
        mctx.close()
        del mwl
        torch.cuda.empty_cache()
    # the batched and served forms are reported from rank 0 (each replica would measure the same)
    batched = None
    if rank == 0 and not args.no_batched:
        batched = run_batched(dev)
    serving = None
    if rank == 0 and not args.no_serving:
        serving = run_serving(dev, seconds=args.serve_seconds)

    if rank == 0:
        cs = clk.summary("timed_start", "timed_end")
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{wl_name}: {wl_shape[0]}x{wl_shape[1]}x{wl_shape[2]} fp32 "
                                   f"field x {wl_shape[3]} timesteps, {wl_shape[4]} particles x "
                                   f"{wl_shape[5]} attributes, window [{wl_desc[0]},{wl_desc[1]}), "
                                   f"preds {wl_desc[2]}",
                       "step": "bin + criterion/label + features", "vt_per_step": vt,
                       "n_features": int(n_features),
                       "l2": "inputs larger than L2 (field alone 4*V*T bytes)",
                       "parallelism": f"replicas x{world}", "tuning": tuning,
                       "input_sha256": hashes},
            "segment_only": {"ms": round(seg_ms, 4), "ms_200": round(seg_ms_long, 4),
                             "value": round(vt / (seg_ms * 1e-3) / 1e9, 3) if seg_ms else None,
                             "value_200": round(vt / (seg_ms_long * 1e-3) / 1e9, 3),
                             "unit": UNIT, "roofline": seg_roof},
            "roofline": roof, "step_roofline": step_roof, "d2d_copy_gb_per_s": copy_gbs,
            "clocks": cs, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "gpu_launches_per_step": int(launches_per_step),
            "ms_per_step_profiled": round(ms_prof, 4),
            "kernels": per_kernel, "cpu_baseline": cpu,
            "batched": batched, "serving": serving, "clustering": clustering,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_batched(dev, reps=3):
    """Batched form: 64 queries with their own thresholds, attributes and windows (T_w uniform in
    2..32) on a 192^3 x 32 field with 4M 3-attribute points, as one msf_segment_batch call,
    against a loop of msf_segment calls on the same context. Both produce identical labels."""
    import torch

    from paper_1903_12294_gb300 import msf, synth
    wl = synth.batched(device=dev)
    T, nz, ny, nx = wl.field.shape
    V = nx * ny * nz
    stream = torch.cuda.current_stream(dev)
    ctx = msf.Context(dev.index, stream)
    ctx.load(wl.field, wl.pos, wl.attr)
    ctx.bin()
    crits = [msf.make_criteria(t0, t1, pr, e) for (t0, t1, pr, e) in wl.queries]
    labels = [torch.empty((t1 - t0, nz, ny, nx), dtype=torch.int32, device=dev)
              for (t0, t1, _, _) in wl.queries]
    vt = sum((t1 - t0) * V for (t0, t1, _, _) in wl.queries)

    def plain():
        return [msf.msf_segment(ctx.h, c, l) for c, l in zip(crits, labels)]

    def batch():
        return msf.msf_segment_batch(ctx.h, crits, labels)

    # the batched form's tile shape picked by the library's batch autotuner (untimed)
    tuning = msf.msf_autotune_batch(ctx.h, crits, labels, 2)
    tuning = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in tuning.items()}
    out = {}
    ctx.kernel_times(reset=True)
    tuned_sched = tuning.get("sched")

    def with_sched(sched):  # the same batch (tuned tiles) with another schedule
        def run():
            ctx.set_batch_schedule(sched)
            try:
                return batch()
            finally:
                ctx.set_batch_schedule(tuned_sched)
        return run
    # the phase launches (their per-phase split) and the persistent launch, beside the tuned
    # choice; the last arm is the tuned batch with graphs on: its warm-up runs plainly, then
    # captures, and the timed calls replay the graph
    for name, fn in (("plain", plain), ("batched", batch), ("batched_phases", with_sched(1)),
                     ("batched_persistent", with_sched(msf.MSF_SCHED_PERSISTENT | 1)),
                     ("batched_graph", batch)):
        if name == "batched_graph":
            ctx.set_batch_graphs(True)
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(reps):
            nf = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3) / reps
        out[name] = {"ms_per_batch": round(ms, 3), "queries_per_s": round(len(crits) / (ms * 1e-3), 1),
                     "gvt_per_s": round(vt / (ms * 1e-3) / 1e9, 2), "n_features_total": int(sum(nf))}
        ctx.profiling(True)                       # one more pass for the per-kernel split
        fn()
        ctx.profiling(False)
        out[name]["kernels_ms"] = {k: round(v[0], 3) for k, v in ctx.kernel_times(reset=True).items()}
    replays = ctx.batch_graph_replays()
    ctx.set_batch_graphs(False)
    # same labels both ways
    ref = [l.clone() for l in labels]
    batch()
    same = all(torch.equal(a, b) for a, b in zip(ref, labels))
    ctx.close()
    del labels, ref
    torch.cuda.empty_cache()
    return {"workload": f"{nx}x{ny}x{nz} x {T}, {wl.pos.shape[2]} points x {wl.attr.shape[1]} "
                        f"attrs, {len(crits)} queries, T_w in 2..32, {vt} query-voxel-timesteps",
            "plain": out["plain"], "batched": out["batched"],
            "batched_phases": out["batched_phases"],
            "batched_persistent": out["batched_persistent"],
            "batched_graph": dict(out["batched_graph"], graph_replays=replays),
            "batch_tuning": tuning,
            "speedup": round(out["plain"]["ms_per_batch"] / out["batched"]["ms_per_batch"], 2),
            "speedup_graph": round(out["plain"]["ms_per_batch"] /
                                   out["batched_graph"]["ms_per_batch"], 2),
            "labels_identical": bool(same)}


def run_serving(dev, seconds=10.0, rate=200.0, saturate=256):
    """Serving form: the 2D+time traffic-shaped dataset (1024^2 x 96 density field, 208,334
    walkers x 96 steps) resident on the device; queries with windows of 4..64 steps and random
    criteria arrive as a Poisson process at `rate`/s and go through the query server
    (continuous batching, memory admission). Reports latency from submission to the batch's
    completion on the device (p50/p99), queries/s at that offered load, and the server's
    capacity on a burst of `saturate` queries against a loop of plain msf_segment calls."""
    import torch

    from paper_1903_12294_gb300 import msf, synth
    wl = synth.serving(device=dev)
    T, nz, ny, nx = wl.field.shape
    V = nx * ny * nz
    stream = torch.cuda.current_stream(dev)
    ctx = msf.Context(dev.index, stream)
    ctx.load(wl.field, wl.pos, wl.attr)
    ctx.bin()
    arrivals = synth.poisson_arrivals(rate, seconds, synth.SEED_BASE + 500)
    nq = max(len(arrivals), saturate)
    queries = synth.random_queries(wl, nq, synth.SEED_BASE + 501, (4, 64), field_q=(0.90, 0.99))
    pool = 8 << 30

    def serve(times, check=()):
        """Submit queries[i] at times[i] (seconds from start); returns per-query records."""
        srv = msf.Server(ctx, pool_bytes=pool, max_batch=64, slots=2)
        n = len(times)
        rec, kept = {}, {}

        stop = threading.Event()
        deadline = time.perf_counter() + max(times, default=0.0) + 120.0

        def consume():
            while len(rec) < n and not stop.is_set() and time.perf_counter() < deadline:
                for r in srv.poll(cap=128, timeout_ms=100):
                    rec[r.tag] = (r.status, r.n_features, r.batch_size, r.t_submit_ns,
                                  r.t_admit_ns, r.t_done_ns)
                    if r.tag in check:
                        kept[r.tag] = srv.take_labels(r)
                    elif r.labels:
                        srv.release(r.tag)
        th = threading.Thread(target=consume)
        th.start()
        try:
            t_start = time.perf_counter()
            for i, t in enumerate(times):
                d = t_start + t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                t0, t1, pr, e = queries[i]
                srv.submit(i, t0, t1, pr, e)
        except BaseException:
            stop.set()
            raise
        finally:
            th.join()
            st = srv.stats()
            srv.close()
        if len(rec) < n:
            raise RuntimeError(f"serving: {len(rec)} of {n} results before the deadline")
        return rec, kept, st

    def summary(rec, st):
        lat = sorted((v[5] - v[3]) * 1e-6 for v in rec.values())
        span = (max(v[5] for v in rec.values()) - min(v[3] for v in rec.values())) * 1e-9

        def q(p):
            return lat[min(len(lat) - 1, int(p * len(lat)))]
        return {"queries": len(rec), "failed": sum(v[0] != 0 for v in rec.values()),
                "queries_per_s": round(len(rec) / span, 1),
                "latency_ms": {"p50": round(q(0.50), 3), "p99": round(q(0.99), 3),
                               "mean": round(sum(lat) / len(lat), 3), "max": round(lat[-1], 3)},
                "batches": st.batches, "mean_batch": round(len(rec) / max(st.batches, 1), 2),
                "max_batch": st.max_batch_seen, "max_slots_busy": st.max_slots_busy,
                "pool_peak_gb": round(st.pool_peak / 1e9, 3)}

    serve([0.0] * 8)                                         # warm-up
    rec, _, st = serve(arrivals)
    offered = summary(rec, st)
    check = set(range(0, saturate, max(1, saturate // 16)))
    rec_b, kept, st_b = serve([0.0] * saturate, check)
    burst = summary(rec_b, st_b)
    # plain per-query loop on the same burst, and the identity of the server's results
    crits = [msf.make_criteria(t0, t1, pr, e) for (t0, t1, pr, e) in queries[:saturate]]
    lab = torch.empty((64, nz, ny, nx), dtype=torch.int32, device=dev)
    for c in crits[:4]:
        msf.msf_segment(ctx.h, c, lab)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in crits:
        msf.msf_segment(ctx.h, c, lab)
    torch.cuda.synchronize()
    plain_qps = saturate / (time.perf_counter() - t0)
    same = True
    for i in sorted(check):
        a, b, pr, e = queries[i]
        n = msf.msf_segment(ctx.h, crits[i], lab[:b - a])
        same &= (n == rec_b[i][1]) and torch.equal(lab[:b - a], kept[i])
    ctx.close()
    del lab
    torch.cuda.empty_cache()
    vt_mean = sum((t1 - t0) * V for (t0, t1, _, _) in queries[:saturate]) / saturate
    return {"workload": f"{nx}x{ny}x{nz} x {T}, {wl.pos.shape[2]} walkers x {T} steps, "
                        f"T_w in 4..64 (mean {vt_mean / V:.1f} steps), random criteria",
            "offered": {"rate_per_s": rate, "seconds": seconds, **offered},
            "burst": {"queries": saturate, **burst, "plain_loop_queries_per_s": round(plain_qps, 1),
                      "speedup_vs_plain": round(burst["queries_per_s"] / plain_qps, 2)},
            "labels_identical_alone_and_in_mix": bool(same), "checked": len(check),
            "pool_gb": pool / 2**30}


def run_clustering(ctx, wl, dev, reps=3):
    """The paper's clustering (§3.2) on the resident workload: k = 16 x 16 x 16 x 4 centres
    (8 x 8 x 8 voxels x 8 steps each), the speed attribute as point variable, up to 10 updates;
    sample-updates per second (field + point samples of the window times the updates made).
    Beside it, the oracle and the GPU on the tiny workload (K = 128), the same run both ways."""
    import numpy as np
    import torch

    from paper_1903_12294_gb300 import msf, synth
    T, nz, ny, nx = wl.field.shape
    args = dict(w_p=1.0, w_f=1.0, w_d=0.05, c_f=1.0, eps_c=1e-3, max_iter=10)
    k = (16, 16, 16, 4)
    stream = torch.cuda.current_stream(dev)
    ctx.cluster(0, T, 0, k, **args)                                   # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fl, pl, c, n, it = ctx.cluster(0, T, 0, k, **args)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    samples = int(n.sum())
    ctx.kernel_times(reset=True)
    ctx.profiling(True)                     # one more run for the per-kernel split
    ctx.cluster(0, T, 0, k, **args)
    ctx.profiling(False)
    kms = {kk: round(vv[0], 3) for kk, vv in ctx.kernel_times(reset=True).items()}
    # like for like on the tiny workload
    import oracle
    tw = synth.tiny(device=dev)
    tctx = msf.Context(dev.index, stream)
    tctx.load(tw.field, tw.pos, tw.attr)
    tctx.bin()
    tctx.cluster(0, 8, 0, (4, 4, 4, 2), **args)
    torch.cuda.synchronize()
    g0 = time.perf_counter()
    _, _, _, tn, tit = tctx.cluster(0, 8, 0, (4, 4, 4, 2), **args)
    torch.cuda.synchronize()
    g_ms = (time.perf_counter() - g0) * 1e3
    key = tctx.bins("cpu")[0].numpy()
    tctx.close()
    f, p, a = tw.numpy()
    oracle.build()
    c0 = time.perf_counter()
    ores = oracle.slic(f, p, a, key, 0, 8, 0, (4, 4, 4, 2), **args)
    c_ms = (time.perf_counter() - c0) * 1e3
    return {"workload": f"{nx}x{ny}x{nz} x {T} field + {wl.pos.shape[2]} points, k = {k} "
                        f"({int(np.prod(k))} centres), attribute 0, {args}",
            "ms_per_run": round(ms, 3), "updates": it, "samples": samples,
            "g_sample_updates_per_s": round(samples * it / (ms * 1e-3) / 1e9, 3),
            "kernels_ms": kms,
            "tiny_like_for_like": {"gpu_ms": round(g_ms, 3), "oracle_ms": round(c_ms, 1),
                                   "oracle_cores": 1, "updates": tit,
                                   "identical_updates": ores[4] == tit}}, (fl, pl, c)


def run_post(ctx, wl, dev, fl, pl, c, reps=5):
    """The steps after a clustering, on its result (§3.3, §3.4): merging its centres (eps_m =
    0.05, both value terms), relabelling its field labels, its per-cluster summaries, a range
    query, and the trajectory pieces of its point labels and of the step's feature labels. Each
    is timed through its C-ABI call (which synchronises), host clock, median of `reps`."""
    import numpy as np
    import torch

    from paper_1903_12294_gb300 import msf
    T = wl.field.shape[0]
    P = wl.pos.shape[2]
    K = len(c)
    cd = torch.as_tensor(c).to(dev)
    seg, _ = ctx.segment(wl.t0, wl.t1, wl.preds, wl.edges)
    lo = np.full(6, -np.inf, np.float32)
    hi = np.full(6, np.inf, np.float32)
    lo[5] = 0.5                                   # centres of high field value
    mapd = torch.empty(K, dtype=torch.int32, device=dev)
    out = {}

    def timed(name, fn, units=None, unit=None):
        fn()                                      # warm-up
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            r = fn()
            ts.append((time.perf_counter() - t0) * 1e3)
        ms = float(np.median(ts))
        out[name] = {"ms": round(ms, 3)}
        if units is not None:
            out[name][unit] = round(units / (ms * 1e-3) / 1e9, 3)
        return r

    _, groups = timed("merge", lambda: ctx.merge_clusters(cd, 0.05, out=mapd),
                      K * (K - 1) / 2, "g_pairs_per_s")
    out["merge"].update({"centres": K, "groups": groups})
    fl2 = fl.clone()
    timed("relabel", lambda: ctx.relabel(fl2, mapd), fl.numel(), "g_labels_per_s")
    st = timed("cluster_stats", lambda: ctx.cluster_stats(0, T, 0, fl, pl, K),
               fl.numel() + pl.numel(), "g_samples_per_s")
    out["cluster_stats"]["non_empty"] = int(((st["n_field"] + st["n_point"]) > 0).sum())
    sel = timed("select", lambda: ctx.select_clusters(cd, lo, hi))
    out["select"]["selected"] = int(len(sel))
    # pieces into a device buffer of the right size (one count, scan and write pass per call)
    for name, t0, t1, lab, space in [("pieces_points", 0, T, pl, msf.MSF_SPACE_POINTS),
                                     ("pieces_voxels", wl.t0, wl.t1, seg, msf.MSF_SPACE_VOXELS)]:
        n = len(ctx.split_trajectories(t0, t1, lab, space))
        buf = torch.empty((max(n, 1), 4), dtype=torch.int32, device=dev)
        timed(name, lambda: ctx.split_trajectories(t0, t1, lab, space, out=buf),
              P * (t1 - t0), "g_point_samples_per_s")
        out[name]["pieces"] = n
        del buf
    del seg, fl2
    return out


def _oracle_sample(wl, t_lo, t_hi):
    """The oracle on timesteps [t_lo, t_hi) of the workload (bin + segment + features)."""
    import oracle
    f = wl.field[t_lo:t_hi].cpu().numpy()
    p = wl.pos[t_lo:t_hi].cpu().numpy()
    a = wl.attr[t_lo:t_hi].cpu().numpy()
    oracle.build()
    t0 = time.perf_counter()
    oracle.run_all(f, p, a, 0, t_hi - t_lo, wl.preds, wl.edges)
    return time.perf_counter() - t0


def cpu_baseline(wl, steps_in_sample=8):
    T, nz, ny, nx = wl.field.shape
    n = min(steps_in_sample, wl.t1 - wl.t0)
    secs = _oracle_sample(wl, wl.t0, wl.t0 + n)
    vt = nx * ny * nz * n
    return {"value": round(vt / secs / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"timesteps [{wl.t0},{wl.t0 + n}) of the workload ({vt} voxel-timesteps, "
                      f"{wl.pos.shape[2]} particles): bin + segment + features, single thread",
            "seconds": round(secs, 3), "host": host_cpu()}


def run_reference(args):
    """The reference arm: the CPU oracle, timed on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch

    from paper_1903_12294_gb300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    wl = synth.make(args.config, device=dev, **({"T": args.timesteps} if args.timesteps else {}))
    T, nz, ny, nx = wl.field.shape
    n = 2   # timesteps per step sample
    for _ in range(args.warmup):
        _oracle_sample(wl, wl.t0, wl.t0 + n)
    secs = [_oracle_sample(wl, wl.t0, wl.t0 + n) for _ in range(args.steps)]
    ms = statistics.mean(secs) * 1e3
    vt = nx * ny * nz * n
    value = vt / (ms * 1e-3) / 1e9
    sample = (f"timesteps [{wl.t0},{wl.t0 + n}) of the workload per step ({vt} voxel-timesteps): "
              "bin + segment + features, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name, "sample": sample},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="segment with the fixed tile rule and schedule instead of the autotuner's")
    ap.add_argument("--schedule", default="",
                    help="by,bz,bt,sched: segment with this tile shape and schedule, no tuning")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cluster", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--timesteps", type=int, default=0,
                    help="the workload with this many timesteps (same grid and points per step): "
                         "a smaller case of the same kernels for profiler captures; 0 = as named")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
