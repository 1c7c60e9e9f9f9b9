#!/usr/bin/env python
"""Benchmark of the FlashSplat hot path on GB300.

One step = one whole scene solve (Sec. 3.2-3.3, Sec. 4.2): every mask pixel
of every view is alpha-composited through the scene, alpha*T is accumulated
per (Gaussian, label), and the biased closed-form assignment runs -- the
binary segmentation workload at real-scene scale: 1,000,000 Gaussians from 20
anisotropic clusters, 100 forward-facing views of 1008x756, noisy binary
masks, gamma = 0.5 (seeded synthetic data).

Metric: Gpix/s = mask pixels solved per second (76.2 M pixels per scene), and
seconds per scene solve.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Default arm: the CUDA library (device-resident inputs, L2 flushed before each
timed step, CUDA-event timing on the launching stream), plus the end-to-end
number through the C ABI with host masks and host outputs.  Under torchrun
every rank solves its own replica of the scene (independent problems, no
collective on the data path).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per scene solve & Gpix/s of α·T accumulation; batched BF16 vs plain FP32"
UNIT = "Gpix/s"
FLOPS_PER_PAIR = 19   # FP32 flops of one (pixel, Gaussian) compositing step, FMA = 2
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of blend_kernel per work unit (census pair), from
# one ncu capture of the current kernel: the six launches of an 8-view solve
# of the binary workload read 240.4 MB and wrote 0.62 MB for 435.7 M census
# pairs (profiles/blend_kernel_binary_1M_8views.txt); scaled by the units of
# the launches timed here.
BLEND_DRAM_BYTES_PER_PAIR = 241.0e6 / 435.7e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="flashsplat", choices=["flashsplat", "reference"])
    ap.add_argument("--views-per-batch", type=int, default=0)
    ap.add_argument("--depth-chunks", type=int, default=0)
    ap.add_argument("--workload", default="binary", choices=["binary", "multi"],
                    help="binary: 1M Gaussians, 100 forward-facing views 1008x756, uint8 "
                         "masks (default); multi: 3M Gaussians in 32 instances, 200 orbit "
                         "views 1256x828, int32 id masks, 33 labels")
    ap.add_argument("--views", type=int, default=0, help="0: the workload's own count")
    ap.add_argument("--n", type=int, default=0, help="0: the workload's own count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip timing the other precision form of the workload")
    ap.add_argument("--no-multi", action="store_true",
                    help="skip the multi-instance workload's extra measurement")
    ap.add_argument("--multi-steps", type=int, default=5)
    ap.add_argument("--no-graph", action="store_true",
                    help="skip timing the solve captured into a CUDA graph")
    ap.add_argument("--cpu-sample-views", type=int, default=12)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"],
                    help="fp16: the reduced-precision form (BF16 quat/scale, FP16 opacity, "
                         "per-view records with an FP16 whitening matrix and FP32 mean)")
    ap.add_argument("--serve", action="store_true",
                    help="request-server benchmark: 16 resident scenes of uneven size, a "
                         "Poisson request trace, p50/p99 latency vs sequential solves")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--serve-scale", type=float, default=1.0)
    ap.add_argument("--recheck-margin", type=float, default=0.0,
                    help="FP64 re-check of decisions with a margin below this (0: library "
                         "default 1e-4; negative: off)")
    return ap.parse_args()


def synth_mod():
    from paper_2409_08270_gb300 import synth
    return synth


def workload(args):
    if args.workload == "multi":
        return synth_mod().multi_scene(n=args.n or 3_000_000, views=args.views or 200)
    return synth_mod().binary_scene(n=args.n or 1_000_000, views=args.views or 100)


def config_of(w, args, extra=None):
    if w.name == "multi":
        what = (f"multi-instance segmentation, {w.n} Gaussians / {w.E - 1} instances, "
                f"{len(w.cams)} orbit views {w.cams[0]['width']}x{w.cams[0]['height']}, int32 "
                f"id masks, {w.E} labels, gamma {w.gamma}")
    else:
        what = (f"binary segmentation, {w.n} Gaussians / 20 clusters, {len(w.cams)} views "
                f"{w.cams[0]['width']}x{w.cams[0]['height']}, uint8 masks, gamma {w.gamma}")
    c = {"workload": what,
         "gaussians": w.n, "views": len(w.cams), "width": w.cams[0]["width"],
         "height": w.cams[0]["height"], "labels": w.E, "gamma": w.gamma,
         "pixels_per_scene": w.pixels, "table": "fp32 [N x E] (FP64 cross-view sum)",
         "form": ("reduced precision: BF16 quat/scale, FP16 opacity, FP16 whitening + FP32 "
                  "mean per view" if args.precision == "fp16" else "plain FP32"),
         "mask_noise_fraction": round(w.info.get("noise_fraction", 0.0), 4)}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """SM clock, power and clock-event reasons sampled during the timed region.

    Reads NVML (the driver's libnvidia-ml) from a thread every 20 ms; falls
    back to `nvidia-smi -lms 100` when NVML cannot be loaded.  Read-only: no
    setting of the GPU is touched.
    """
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid=None):
        self.rows, self.p, self.nvml = [], None, None
        try:
            self._start_nvml(uuid)
        except Exception:
            self.nvml = None
            self._start_smi(uuid)

    def _start_nvml(self, uuid):
        import ctypes
        import threading
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        if uuid:
            rc = lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h))
        else:
            rc = lib.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h))
        if rc != 0:
            raise RuntimeError("no NVML handle")
        mx = ctypes.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))      # 1 = SM clock
        self.max_mhz = float(mx.value)
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.nvml, self.stop_ev = lib, threading.Event()

        def loop():
            clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            while not self.stop_ev.is_set():
                if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                    lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw))
                    get_reasons(h, ctypes.byref(rs))
                    self.rows.append((float(clk.value), pw.value / 1000.0, int(rs.value)))
                self.stop_ev.wait(0.02)

        self.th = threading.Thread(target=loop, daemon=True)
        self.th.start()

    def _start_smi(self, uuid):
        self.path = tempfile.mktemp(prefix="fs_clocks_", suffix=".csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.nvml is not None:
            self.stop_ev.set()
            self.th.join()
            self.nvml.nvmlShutdown()
            if not self.rows:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"]}
            reasons = sorted({name for _, _, r in self.rows for bit, name in self.REASONS.items()
                              if r & bit})
            return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                    "sm_max_mhz": self.max_mhz, "reasons": reasons,
                    "samples": len(self.rows), "source": "NVML every 20 ms",
                    "power_w_max": max(r[1] for r in self.rows)}
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "source": "nvidia-smi every 100 ms",
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---------------------------------------------------------------------------
# multi-rank reduction (one process per GPU; replicas, no data-path collective)
# ---------------------------------------------------------------------------

def max_over_ranks(x, world, device):
    """The largest per-rank value over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_gpix(world, pixels_per_rank, steps, total_ms):
    """Whole-job throughput: every rank's pixels over the slowest rank's time."""
    return world * pixels_per_rank * steps / (total_ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# the CUDA arm
# ---------------------------------------------------------------------------

def make_solver(fsb, w, args, local_rank, precision, census=False, time_stages=True):
    """A solver over the workload's scene in one of the two forms: plain FP32
    inputs with float-pair records, or the reduced-precision form (BF16 quat
    and scale, FP16 opacity, FP16 whitening matrix + FP32 mean per view)."""
    import torch
    gaussians = w.gaussians
    if precision == "fp16":
        r = synth_mod().rounded_gaussians(w.gaussians)
        gaussians = {"mean": torch.from_numpy(r["mean"]),
                     "quat": torch.from_numpy(r["quat"]).to(torch.bfloat16),
                     "scale": torch.from_numpy(r["scale"]).to(torch.bfloat16),
                     "opacity": torch.from_numpy(r["opacity"]).to(torch.float16)}
    return fsb.Solver(gaussians, device=local_rank, views_per_batch=args.views_per_batch,
                      depth_chunks=args.depth_chunks, time_stages=time_stages and not census,
                      recheck_margin=args.recheck_margin,
                      record_precision=fsb.FS_F16 if precision == "fp16" else 0, census=census)


def timed_solves(fsb, solver, w, dmasks, steps, warmup, flush, stream, dev):
    """`warmup` untimed solves, then `steps` timed ones, each after an L2
    flush, timed with CUDA events on the launching stream.  Returns the
    per-step ms, the summed per-solve statistics and the last output."""
    import torch
    out = None
    for _ in range(warmup):
        out = solver.solve(w.cams, dmasks, w.E, w.gamma, sync=False)
    fsb.fs_synchronize(solver.ctx, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    ms, sums = [], {"blend_ms": 0.0, "blend_launches": 0, "list_entries": 0,
                    "staged_entries": 0, "rechecked": 0, "recheck_pairs": 0,
                    "kernel_launches": 0, "stage_ms": [0.0] * len(fsb.STAGES)}
    for _ in range(steps):
        flush.fill_(1)                       # evict the previous step's data from L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = solver.solve(w.cams, dmasks, w.E, w.gamma, sync=False)
        e1.record(stream)
        st = fsb.fs_synchronize(solver.ctx, stream.cuda_stream)
        ms.append(e0.elapsed_time(e1))
        for k in sums:
            if k == "stage_ms":
                for i in range(len(sums[k])):
                    sums[k][i] += st.stage_ms[i]
            else:
                sums[k] += getattr(st, k)
    torch.cuda.synchronize(dev)
    return ms, sums, out


def stages_of(fsb, sums, steps):
    """Device time per stage and step (CUDA events on the stream each stage
    runs on; the next view batch's projection overlaps the current batch on a
    side stream, so the stages can add up to more than the step)."""
    out = {name: round(sums["stage_ms"][i] / max(1, steps), 4)
           for i, name in enumerate(fsb.STAGES)}
    out["note"] = "per-stage device time; overlapping stages make the sum exceed the step"
    return out


def census_pairs_of(fsb, w, args, local_rank, precision, dmasks, stream):
    """Work units of the blend, counted by one census solve (a counting
    variant of the same kernels, untimed)."""
    cs = make_solver(fsb, w, args, local_rank, precision, census=True)
    try:
        cs.solve(w.cams, dmasks, w.E, w.gamma, sync=False)
        st = fsb.fs_synchronize(cs.ctx, stream.cuda_stream)
        return st
    finally:
        cs.close()


def form_accuracy(w, outs, rows=96, seed=7):
    """Each form's table rows and labels against the FP64 oracle on the
    ORIGINAL (unrounded) inputs, on a seeded sample of seen Gaussians: max /
    mean relative error of the entries the oracle's near-threshold bound does
    not cover, and the fraction of sampled labels that agree."""
    import numpy as np
    import oracle
    from oracle.assign import assign, labels_from_membership
    any_out = next(iter(outs.values()))
    seen = np.flatnonzero(any_out["table"].sum(1) > 0)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(seen, min(rows, seen.size), replace=False))
    t0 = time.perf_counter()
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E, sel=sel)
    dt = time.perf_counter() - t0
    lab_o = labels_from_membership(assign(acc.table, w.gamma))
    ref = acc.table
    res = {}
    for name, o in outs.items():
        g = o["table"][sel].astype(np.float64)
        ok = (ref >= 1e-6 * ref.max()) & (acc.risk <= 1e-6 * ref)
        rel = np.abs(g - ref)[ok] / ref[ok]
        lab = o["label"][sel]
        res[name] = {"rows": int(sel.size), "entries_free_of_bound": int(ok.sum()),
                     "max_rel_err": float(rel.max()) if rel.size else None,
                     "mean_rel_err": float(rel.mean()) if rel.size else None,
                     "label_agreement": float((lab == lab_o).mean())}
    return res, dt


def run_flashsplat(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2409_08270_gb300 import build as lib_build
    from paper_2409_08270_gb300 import flashsplat as fsb

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib_build.build()
    fsb.load()
    w = workload(args)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    solver = make_solver(fsb, w, args, local_rank, args.precision)
    dmasks = solver.upload_masks(w.masks)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    uuid = None
    try:
        uuid = "GPU-" + str(props.uuid)
    except Exception:
        pass
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(uuid)
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    ms_steps, sums, out = timed_solves(fsb, solver, w, dmasks, args.steps, args.warmup, flush,
                                       stream, dev)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    blend_ms, blend_launches = sums["blend_ms"], sums["blend_launches"]
    entries, staged = sums["list_entries"], sums["staged_entries"]
    rechecked, recheck_pairs = sums["rechecked"], sums["recheck_pairs"]
    launches = sums["kernel_launches"]
    total_ms = max_over_ranks(sum(ms_steps), world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    gpix = whole_job_gpix(world, w.pixels, args.steps, total_ms)

    # ---- work units of the blend: one census solve (untimed) ----------------
    # The roofline's unit is a (pixel, Gaussian) pair with alpha >= 1/255 that
    # the pixel's front-to-back walk reaches, its stop included -- the pairs
    # the compositing rule of Eq. 1 must evaluate, whatever the culling.  The
    # workload is fixed, so one census solve (a counting variant of the same
    # kernels) gives the units of every timed step.
    cst = census_pairs_of(fsb, w, args, local_rank, args.precision, dmasks, stream)
    census_pairs, census_evaluated = int(cst.census_pairs), int(cst.pairs)
    census_shape = {"rounds": int(cst.census_rounds), "steps": int(cst.census_steps),
                    "rounds_mixed_labels": int(cst.census_rounds_mixed),
                    "staged": int(cst.staged_entries), "list_entries": int(cst.list_entries)}
    pairs = census_pairs * args.steps

    # ---- argmax-only re-solve for a new gamma on the resident table ----------
    # (Sec. 4.2: the assignment alone is re-run when only the bias changes)
    tab = out["table"]
    n_g, E_g = tab.shape
    r_bits = torch.empty(n_g, dtype=torch.int64, device=dev)
    r_label = torch.empty(n_g, dtype=torch.int32, device=dev)
    r_margin = torch.empty(n_g, dtype=torch.float32, device=dev)

    def resolve(g):
        fsb.fs_assign(solver.ctx, tab.data_ptr(), fsb.FS_F32, n_g, E_g, g, r_bits.data_ptr(),
                      r_label.data_ptr(), r_margin.data_ptr(), stream.cuda_stream)

    for _ in range(3):
        resolve(0.3)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        resolve(0.3)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    gamma_resolve = {"ms": e0.elapsed_time(e1) / 20, "gamma": 0.3, "launches": 1,
                     "table": f"fp32 [{n_g} x {E_g}] resident on the device",
                     "paper_context": "0.4 ms per object on an RTX A6000 (Table 2), another "
                                      "scene and GPU"}

    # ---- end to end through the C ABI: host masks in, host outputs out --------
    e2e = None
    if not args.no_e2e:
        host_masks = [torch.from_numpy(m).pin_memory() for m in w.masks]
        n = w.n
        h_bits = torch.empty(n, dtype=torch.int64).pin_memory()
        h_label = torch.empty(n, dtype=torch.int32).pin_memory()
        h_margin = torch.empty(n, dtype=torch.float32).pin_memory()
        res = fsb.fs_result()
        res.memory, res.table_dtype = fsb.FS_MEM_HOST, fsb.FS_F32
        res.table = None
        res.member_bits, res.label, res.margin = (h_bits.data_ptr(), h_label.data_ptr(),
                                                  h_margin.data_ptr())
        cams = fsb.make_cameras(w.cams)
        mptr = [m.data_ptr() for m in host_masks]
        mask_dt = fsb.FS_I32 if w.masks[0].dtype == np.int32 else fsb.FS_U8

        def e2e_step():
            fsb.fs_solve(solver.ctx, solver.scene, cams, mptr, mask_dt, fsb.FS_MEM_HOST, w.E,
                         float(w.gamma), res, stream.cuda_stream)
            fsb.fs_synchronize(solver.ctx, stream.cuda_stream)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        h2d = sum(m.numel() * m.element_size() for m in host_masks)
        d2h = n * (8 + 4 + 4)
        # the result is on the host: check it once (labels in range, some members)
        lab = h_label.numpy()
        assert lab.min() >= -1 and lab.max() < w.E
        e2e = {"value": whole_job_gpix(world, w.pixels, args.steps, e2e_ms), "unit": UNIT,
               "ms_per_step": e2e_ms / args.steps, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "api": "fs_solve (host masks, host outputs)"}

    # ---- roofline of the dominant kernel (blend/accumulate) -------------------
    sm_clk = clk.get("sm_max_mhz") or 2070.0
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_clk * 1e6 / 1e12
    achieved = (FLOPS_PER_PAIR * pairs) / (blend_ms * 1e-3) / 1e12 if blend_ms > 0 else None
    roofline = {"kernel": "blend_kernel (alpha*T accumulation)", "bound": "alu",
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": (achieved / peak_tflops) if achieved else None,
                "traffic": (BLEND_DRAM_BYTES_PER_PAIR * pairs / max(1, blend_launches)
                            if BLEND_DRAM_BYTES_PER_PAIR and blend_launches else None),
                "traffic_unit": "DRAM bytes per launch (ncu capture scaled by work units)",
                "peak_source": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_clk:.0f} MHz",
                "unit_of_work": "pair with alpha >= 1/255 reached before the pixel's stop "
                                "(stop included), counted by a census solve",
                "pairs_per_step": census_pairs,
                "evaluated_pairs_per_step": census_evaluated,
                "census": census_shape,
                "list_entries_per_step": entries // max(1, args.steps),
                "staged_entries_per_step": staged // max(1, args.steps),
                "flops_per_pair": FLOPS_PER_PAIR,
                "blend_ms_per_step": blend_ms / args.steps,
                "blend_share_of_step": blend_ms / max(total_ms, 1e-9),
                "blend_launches_per_step": blend_launches // max(1, args.steps)}

    line = {
        "metric": METRIC, "value": gpix, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "s_per_scene": ms_per_step / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded clustered 3D-GS scene and noisy masks; stands in for the "
                "paper's LLFF/MIP-360/T&T scenes with SAM masks)",
        "config": config_of(w, args, {"l2": "flushed (512 MB write) before each timed step",
                                      "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                                      "wall_s_timed": t_wall}),
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "clocks": clk,
        "stages_ms_per_step": stages_of(fsb, sums, args.steps),
        "gamma_resolve": gamma_resolve,
        "near_tie_recheck": {"margin_below": (args.recheck_margin if args.recheck_margin > 0 else
                                              1e-4 if args.recheck_margin == 0 else None),
                             "gaussians_per_step": rechecked // max(1, args.steps),
                             "fp64_pairs_per_step": recheck_pairs // max(1, args.steps)},
    }
    # ---- the same solve captured into a CUDA graph and replayed ----------------
    if not args.no_graph:
        line["graph"] = measure_graph(fsb, solver, w, dmasks, args, flush, stream, dev, out, world)
    # ---- the same workload in the other form: plain FP32 vs reduced precision --
    if world == 1 and not args.no_forms:
        line["forms"] = measure_forms(fsb, args, w, local_rank, dev, stream, flush, solver,
                                      dmasks, ms_steps, out)
    solver.close()
    del dmasks
    # ---- the multi-instance workload (3M Gaussians, 200 views, 33 labels) -----
    if world == 1 and not args.no_multi and args.workload == "binary":
        line["workloads"] = {"multi": measure_multi(fsb, args, local_rank, dev, stream, flush,
                                                    n_sm, sm_clk)}
    return line, w


def measure_graph(fsb, solver, w, dmasks, args, flush, stream, dev, out_main, world):
    """The solve captured once (fs_graph_create) and replayed `steps` times,
    timed like the main loop (L2 flushed before each replay, CUDA events on
    the stream); the near-tie re-check and the FP32 rounding run after each
    replay, outside the graph, as in fs_graph_launch."""
    import numpy as np
    import torch
    t0 = time.perf_counter()
    g = solver.capture(w.cams, dmasks, w.E, w.gamma)
    t_capture = time.perf_counter() - t0
    try:
        for _ in range(args.warmup):
            g.launch(stream)
        g.synchronize(stream)
        if world > 1:
            torch.distributed.barrier()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.launch(stream)
            e1.record(stream)
            st = g.synchronize(stream)
            ms.append(e0.elapsed_time(e1))
        total = max_over_ranks(sum(ms), world, dev)
        same = bool(np.array_equal(g.outputs["label"].cpu().numpy(),
                                   out_main["label"].cpu().numpy()))
    finally:
        g.close()
    return {"ms_per_step": total / args.steps,
            "value": whole_job_gpix(world, w.pixels, args.steps, total), "unit": UNIT,
            "capture_s": round(t_capture, 2), "labels_equal_uncaptured": same,
            "graph_launches_per_step": 1, "rechecked_per_step": int(st.rechecked),
            "what": "fs_graph_launch: one CUDA graph (projection, depth sort, binning, blend, "
                    "FP64 sum, assignment) + the near-tie re-check and FP32 rounding after it"}


def _form_entry(w, ms_steps, sums, steps):
    total = sum(ms_steps)
    return {"ms_per_step": total / steps, "value": w.pixels * steps / (total * 1e-3) / 1e9,
            "unit": UNIT, "blend_ms_per_step": sums["blend_ms"] / steps if sums else None}


def measure_forms(fsb, args, w, local_rank, dev, stream, flush, solver, dmasks, ms_main,
                  out_main):
    """The other precision form timed like the main one (same steps, L2 flush,
    events), and both forms' accuracy against the FP64 oracle on the original
    inputs for a sample of rows, plus how many labels differ between them."""
    other = "fp16" if args.precision == "fp32" else "fp32"
    name = {"fp32": "plain_fp32", "fp16": "bf16"}
    s2 = make_solver(fsb, w, args, local_rank, other)
    try:
        ms2, sums2, out2 = timed_solves(fsb, s2, w, dmasks, args.steps, args.warmup, flush,
                                        stream, dev)
    finally:
        s2.close()
    host = {name[args.precision]: {"table": out_main["table"].float().cpu().numpy(),
                                   "label": out_main["label"].cpu().numpy()},
            name[other]: {"table": out2["table"].float().cpu().numpy(),
                          "label": out2["label"].cpu().numpy()}}
    acc, dt = form_accuracy(w, host)
    forms = {name[args.precision]: _form_entry(w, ms_main, None, args.steps),
             name[other]: _form_entry(w, ms2, sums2, args.steps)}
    for k in forms:
        forms[k].update(acc[k])
    a, b = host["plain_fp32"]["label"], host["bf16"]["label"]
    forms["labels_differing_between_forms"] = int((a != b).sum())
    forms["gaussians"] = int(a.size)
    forms["bf16_form"] = ("BF16 quaternion and scale, FP16 opacity (scene storage); per view an "
                          "FP16 whitening matrix and FP32 mean (32 B record); blending FP32, "
                          "table FP64 across views")
    forms["oracle"] = (f"FP64 oracle on the original FP32 inputs, {acc[name[other]]['rows']} "
                       f"seeded seen Gaussians over all views, {dt:.1f} s")
    return forms


def measure_multi(fsb, args, local_rank, dev, stream, flush, n_sm, sm_clk):
    """The multi-instance workload in the default run: a few timed solves and
    the blend's roofline from a census solve."""
    import torch
    t0 = time.perf_counter()
    wm = synth_mod().multi_scene()
    t_gen = time.perf_counter() - t0
    sm = make_solver(fsb, wm, args, local_rank, "fp32")
    try:
        dm = sm.upload_masks(wm.masks)
        ms, sums, _ = timed_solves(fsb, sm, wm, dm, args.multi_steps, 2, flush, stream, dev)
        cst = census_pairs_of(fsb, wm, args, local_rank, "fp32", dm, stream)
    finally:
        sm.close()
    steps = args.multi_steps
    total = sum(ms)
    peak = n_sm * FP32_LANES_PER_SM * 2 * sm_clk * 1e6 / 1e12
    blend_ms = sums["blend_ms"] / steps
    achieved = FLOPS_PER_PAIR * int(cst.census_pairs) / (blend_ms * 1e-3) / 1e12
    plain = argparse.Namespace(**{**vars(args), "precision": "fp32"})
    del dm
    torch.cuda.synchronize(dev)
    return {"config": config_of(wm, plain, {"generation_s": round(t_gen, 1)}),
            "steps": steps, "warmup": 2, "ms_per_step": total / steps, "s_per_scene": total / steps / 1e3,
            "value": wm.pixels * steps / (total * 1e-3) / 1e9, "unit": UNIT,
            "roofline": {"kernel": "blend_kernel (alpha*T accumulation)", "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "pairs_per_step": int(cst.census_pairs),
                         "evaluated_pairs_per_step": int(cst.pairs),
                         "blend_ms_per_step": blend_ms,
                         "blend_share_of_step": sums["blend_ms"] / max(total, 1e-9)},
            "stages_ms_per_step": stages_of(fsb, sums, steps),
            "list_entries_per_step": sums["list_entries"] // steps,
            "near_tie_recheck_gaussians_per_step": sums["rechecked"] // steps}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, views):
    import oracle
    cams = w.cams[:views]
    masks = w.masks[:views]
    t0 = time.perf_counter()
    acc = oracle.accumulate(w.gaussians, cams, masks, w.E)
    oracle.assign(acc.table, w.gamma)
    dt = time.perf_counter() - t0
    pix = sum(m.size for m in masks)
    return pix, dt


def cpu_cores():
    return len(os.sched_getaffinity(0))


def run_reference(args, rank, world):
    import oracle
    oracle.build()
    w = workload(args)
    px1 = int(w.masks[0].size)
    cfg = config_of(w, args, {"sample": f"1 view per step ({px1:,} pixels), all Gaussians"})
    for _ in range(args.warmup):
        oracle_sample(w, 1)
    pix, tsum = 0, 0.0
    for _ in range(args.steps):
        p, dt = oracle_sample(w, 1)
        pix += p
        tsum += dt
    val = pix / tsum / 1e9
    ms = tsum / args.steps * 1e3
    sample = (f"1 of {len(w.cams)} views per step ({px1:,} pixels); FP64 oracle over all "
              f"{w.n:,} Gaussians")
    return {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded clustered 3D-GS scene and noisy masks)", "config": cfg,
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------------------------
# request server: latency under a Poisson trace, throughput vs sequential
# ---------------------------------------------------------------------------

def run_serve(args):
    import threading
    import numpy as np
    from paper_2409_08270_gb300 import build as lib_build, flashsplat as fsb
    synth = synth_mod()
    lib_build.build()
    fsb.load()
    t_gen = time.perf_counter()
    scenes = synth.serving_scenes(scale=args.serve_scale)
    # two seeded noise draws per scene, prepared before the timed region
    variants = [[synth.request_masks(w, 7919 * k + j) for j in range(2)]
                for k, w in enumerate(scenes)]
    t_gen = time.perf_counter() - t_gen
    rng = np.random.default_rng(synth.SEED_BASE + 55)
    R = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, R))
    picks = rng.integers(0, len(scenes), R)

    def run_trace(srv, ids, paced, window=2 * args.slots):
        tickets = [None] * R
        fetched = [0]

        def submitter():
            t0 = time.perf_counter()
            for i in range(R):
                if paced:
                    dt = t0 + arrivals[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                else:   # back to back, with at most `window` requests outstanding
                    while i - fetched[0] >= window:
                        time.sleep(0.0005)
                k = int(picks[i])
                tickets[i] = srv.submit(ids[k], scenes[k].cams, variants[k][i % 2], scenes[k].E,
                                        scenes[k].gamma)

        th = threading.Thread(target=submitter)
        t_start = time.perf_counter()
        th.start()
        infos = []
        for i in range(R):
            while tickets[i] is None:
                time.sleep(0.0005)
            infos.append(srv.fetch(tickets[i])["info"])
            fetched[0] = i + 1
        th.join()
        wall = time.perf_counter() - t_start
        lat = np.array([x.done_s - x.submit_s for x in infos])
        svc = np.array([x.done_s - x.start_s for x in infos])
        return wall, lat, svc, infos

    def make(slots, graphs=0):
        srv = fsb.Server(slots=slots, autotune=True, graphs=graphs)
        ids = [srv.add_scene(w.gaussians) for w in scenes]
        for k, w in enumerate(scenes):      # warm-up: tuning, untimed
            srv.fetch(srv.submit(ids[k], w.cams, variants[k][0], w.E, w.gamma))
        # every slot sizes its workspace once for the largest scenes (a slot
        # that grows later frees memory, which waits for the whole device)
        big = {int(np.argmax([w.n for w in scenes])), int(np.argmax([w.pixels for w in scenes]))}
        for k in big:
            ts = [srv.submit(ids[k], scenes[k].cams, variants[k][0], scenes[k].E, scenes[k].gamma)
                  for _ in range(slots)]
            for t in ts:
                srv.fetch(t)
        return srv, ids

    srv, ids = make(args.slots)
    wall, lat, svc, infos = run_trace(srv, ids, paced=True)
    wall_b, lat_b, _, _ = run_trace(srv, ids, paced=False)
    srv.close()
    seq, seq_ids = make(1)
    wall_s, lat_s, svc_s, _ = run_trace(seq, seq_ids, paced=False, window=1)
    seq.close()
    # every request a replay of its scene's captured solve (fs_graph_*)
    gsrv, gids = make(args.slots, graphs=len(scenes))
    wall_g, lat_g, svc_g, _ = run_trace(gsrv, gids, paced=True)
    wall_gb, lat_gb, _, _ = run_trace(gsrv, gids, paced=False)
    gsrv.close()
    pix = sum(scenes[int(k)].pixels for k in picks)
    q = lambda a, p: float(np.quantile(a, p))
    return {
        "metric": "request server: p50/p99 latency under a Poisson trace; requests/s",
        "value": q(lat, 0.5), "unit": "s (p50 latency)", "n_gpus": 1, "higher_is_better": False,
        "p99_latency_s": q(lat, 0.99), "p50_latency_s": q(lat, 0.5),
        "requests_per_s": R / wall, "offered_rate": args.rate, "requests": R,
        "burst": {"requests_per_s": R / wall_b, "gpix_per_s": pix / wall_b / 1e9,
                  "p50_latency_s": q(lat_b, 0.5), "p99_latency_s": q(lat_b, 0.99)},
        "sequential": {"requests_per_s": R / wall_s, "gpix_per_s": pix / wall_s / 1e9,
                       "p50_service_s": q(svc_s, 0.5), "p99_service_s": q(svc_s, 0.99)},
        "service_s": {"p50": q(svc, 0.5), "p99": q(svc, 0.99)},
        "captured": {"what": "each request replays its scene's captured solve (CUDA graph) "
                             "after its masks are copied into the captured buffers",
                     "p50_latency_s": q(lat_g, 0.5), "p99_latency_s": q(lat_g, 0.99),
                     "requests_per_s": R / wall_g,
                     "service_s": {"p50": q(svc_g, 0.5), "p99": q(svc_g, 0.99)},
                     "burst": {"requests_per_s": R / wall_gb, "gpix_per_s": pix / wall_gb / 1e9,
                               "p50_latency_s": q(lat_gb, 0.5),
                               "p99_latency_s": q(lat_gb, 0.99)}},
        "dtype": "f32", "data": "synthetic (16 seeded clustered scenes, orbit cameras, "
                                "noisy label masks; two noise draws per scene)",
        "config": {"workload": "16 resident scenes: N log-uniform 2e5..2e6, 20..150 views, "
                               "512^2..1600x1200, 1..16 labels, gamma 0.5",
                   "scale": args.serve_scale, "slots": args.slots, "autotune": True,
                   "scene_gaussians": [w.n for w in scenes],
                   "scene_views": [len(w.cams) for w in scenes],
                   "generation_s": round(t_gen, 1)},
        "tuned": sorted({(x.views_per_batch, x.depth_chunks) for x in infos}),
    }


def main():
    args = parse()
    if args.serve:
        print(json.dumps(run_serve(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line, w = run_flashsplat(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pix, dt = oracle_sample(w, args.cpu_sample_views)
        line["cpu_baseline"] = {
            "value": pix / dt / 1e9, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"first {args.cpu_sample_views} of {len(w.cams)} views "
                      f"({pix:,} pixels), all {w.n:,} Gaussians, FP64, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
