#!/usr/bin/env python
"""Benchmark of the inpainting hot path on GB300.

A step is one whole inpainting of a synthetic layered-motion clip through the
C ABI (vi_upload + vi_run + vi_fetch_result): pyramid and features, shift-map
initialisation, onion-peel initialisation, per level the PatchMatch search
and reconstruction until the stopping rule, level transitions and the final
best-patch step. Default workload: 320x240 px x 60 frames RGB, 3 sprites,
8% occlusion tube, 4 levels, colour + 2 texture channels, FP32 storage.

Output: one JSON line (rank 0). `value` is patch-distance evaluations per
second over the whole job (all ranks), inputs resident in device memory when
the timed region starts. `e2e` is the same metric through the same calls with
host buffers (host->device upload and device->host fetch inside the timed
region). `roofline` is the PatchMatch step kernel's gathered source bytes
(20 B per source voxel read; a full evaluation is 125 voxels = 2,500 B, and
exact pruning skips or shortens most of them) over its CUDA-event time,
against the measured HBM copy bandwidth. `cpu_baseline` times the CPU oracle
(sequential PatchMatch, one thread) on a bounded sample of the same workload.
--workload layered_1280x720x100 selects the HD clip (5 levels).

Multi-GPU (torchrun): replicas only -- each rank inpaints its own clip; no
collective on the data path; barrier + max-over-ranks timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "patch-distance evals/s (and inpainted voxels/s) vs HBM roofline"
UNIT = "evals/s"
WORKLOAD = "layered_320x240x60"
BYTES_PER_VOXEL_FP32_C5 = 5 * 4           # one source voxel: 5 FP32 channels
BYTES_PER_EVAL_FP32_C5 = 125 * BYTES_PER_VOXEL_FP32_C5   # a whole source patch
BYTES_PER_VOXEL_FP16 = 4 * 2             # channels c0..c3 of a voxel from the FP16 copy

# DRAM bytes (read + write) per launch of the PatchMatch step kernels,
# averaged over the step launches of one inpainting of the default workload
# in its default configuration (FP32 storage, Eq. 3 random search, one sweep
# per iteration, autotuned lanes, no realignment), and the source voxels
# those launches gathered per launch, from one ncu capture
# (profiles/k_ann_step_layered_320x240x60.md). Applies to that configuration
# only; None while the kernels have changed since the capture.
NCU_STEP_TRAFFIC = {"workload": "layered_320x240x60", "storage": "fp32", "rs_mode": "eq3", "sub_sweeps": 1,
                    "bytes": (3634.43e6 + 38.00e6) / 330, "gathered_voxels": 68953343.0 / 20}


def combine_ranks(values, dist=None, device="cpu"):
    """(max over ranks, sum over ranks) of a list of floats. With one rank
    (dist None or not initialised) both are the values themselves."""
    import torch
    if dist is None or not dist.is_initialized():
        return list(values), list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id=None):
        self.proc = None
        self.device_id = device_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return summarise_clocks(out)


def summarise_clocks(text):
    """The clocks object of the JSON line from nvidia-smi's CSV samples (the
    FIELDS of ClockSampler, no header, no units): median SM clock under load,
    the maximum, and every throttle reason seen active in any sample."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def _tune_load(args, vi):
    """Imports a lanes-per-target table (--tune-load), e.g. the one an
    unprofiled run saved, so that a profiled run launches the same kernels."""
    if getattr(args, "tune_load", None):
        with open(args.tune_load) as f:
            vi.tune_import(f.read())


def _tune_save(args, vi):
    if getattr(args, "tune_save", None):
        with open(args.tune_save, "w") as f:
            f.write(vi.tune_export())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


WORKLOADS = {
    # name: (W, H, T, sprites, sprite px, hole fraction, levels, seed offset, dynamic texture)
    "layered_320x240x60": (320, 240, 60, 3, (20, 50), 0.08, 4, 2, False),
    "layered_1280x720x100": (1280, 720, 100, 6, (40, 160), 0.05, 5, 3, True),
}


def make_clip(rank, workload=WORKLOAD):
    from paper_1503_05528_gb300 import synth
    W, H, T, ns, sp, frac, L, off, dyn = WORKLOADS[workload]
    # weak scaling: every rank inpaints its own clip of the same size
    return synth.layered_clip(W, H, T, ns, sp, frac, L, synth.BASE_SEED + off + rank,
                              dynamic_texture=dyn, name=workload)


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline field and the --impl reference arm)
# ---------------------------------------------------------------------------
class OracleSample:
    """Level-0 state of the workload for timing the oracle's PatchMatch:
    the oracle's own pyramid level, occluded voxels set to mid-grey, a random
    shift map from the oracle's initialisation."""

    def __init__(self, clip):
        import numpy as np
        from oracle import oracle as O
        self.O = O
        lv = O.build_pyramid(clip.rgb, clip.mask, clip.levels, True)[0]
        lv.x[lv.hole == 1] = 0.5
        lv.phi = O.init_nnf(lv.htilde, lv.dtilde, (1503, 0), O.tag(O.PURPOSE_INIT, 0))
        lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
        self.lv = lv
        self.T = lv.hole.shape[0]
        self.next_t = 2

    def slab(self, frames):
        """One ANN search (rescore + 10 sequential PatchMatch iterations,
        Algorithm 1 as printed) over the targets of `frames` consecutive frames.
        Returns (evals, seconds)."""
        import numpy as np
        lv = self.lv
        t0 = self.next_t
        self.next_t = 2 + (self.next_t - 2 + frames) % max(self.T - 4 - frames, 1)
        tgt = np.zeros_like(lv.htilde)
        tgt[t0:t0 + frames] = lv.htilde[t0:t0 + frames]
        phi = lv.phi.copy()
        d2 = lv.d2.copy()
        s = time.perf_counter()
        ev = self.O.ann(lv.x, tgt, lv.dtilde, phi, d2, n_pm=10, schedule="SEQ", key=(1503, 0),
                        tag_base=self.O.tag(self.O.PURPOSE_SEARCH, 0, 0))
        return ev, time.perf_counter() - s


def cpu_baseline(clip, seconds):
    smp = OracleSample(clip)
    evals, el, frames = 0, 0.0, 0
    while el < seconds:
        ev, dt = smp.slab(2)
        evals += ev
        el += dt
        frames += 2
    return {"value": evals / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"sequential ANN search (rescore + 10 PatchMatch iterations) over the "
                      f"level-0 targets of {frames} frames of {clip.name}: {evals} evaluations "
                      f"in {el:.1f} s, one thread"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    workload = args.workload if args.workload in WORKLOADS else WORKLOAD
    clip = make_clip(0, workload)
    smp = OracleSample(clip)
    frames = 2
    for _ in range(args.warmup):
        smp.slab(frames)
    evals, el = 0, 0.0
    for _ in range(args.steps):
        ev, dt = smp.slab(frames)
        evals += ev
        el += dt
    value = evals / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "sample": f"{frames} frames per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: sequential ANN search over the level-0 "
                                       f"targets of {frames} frames of {workload}, one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    from paper_1503_05528_gb300 import vi

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vi.load(build_if_missing=True)
    _tune_load(args, vi)
    clip = make_clip(rank, args.workload)
    rgb_d = torch.from_numpy(clip.rgb).cuda()
    mask_d = torch.from_numpy(clip.mask).cuda()
    out_d = torch.empty_like(rgb_d)
    stream = torch.cuda.current_stream()
    storage = 1 if args.storage == "fp16" else 0
    ctx = vi.Context(levels=clip.levels, use_texture=1, seed=1503 + rank, clip=rank,
                     stream=stream.cuda_stream, lanes_per_target=args.lanes, storage=storage,
                     rs_mode=1 if args.rs_mode == "multi" else 0, sub_sweeps=args.sub_sweeps)
    n_hole = int(clip.mask.sum())

    T = clip.mask.shape[0]
    if args.realign:
        al_d, am_d = torch.empty_like(rgb_d), torch.empty_like(mask_d)
        res_d = torch.empty_like(rgb_d)

    def realign_in():
        to_ref = vi.affine_to_reference(vi.affine_estimate(rgb_d, mask_d, stream=stream.cuda_stream), T)
        vi.affine_align(rgb_d, mask_d, to_ref, al_d, am_d, stream=stream.cuda_stream)
        return to_ref

    def step():
        if args.realign:
            # Algorithm 4 with AlignVideo first and UnwarpVideo last
            to_ref = realign_in()
            ctx.upload(al_d, am_d)
            ctx.run()
            ctx.fetch_result(res_d)
            vi.affine_unwarp(rgb_d, mask_d, res_d, to_ref, out_d, stream=stream.cuda_stream)
            return
        ctx.upload(rgb_d, mask_d)
        ctx.run()
        ctx.fetch_result(out_d)

    for _ in range(args.warmup):
        step()
    _tune_save(args, vi)
    ctx.profile(True)
    s0 = ctx.stats()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    s1 = ctx.stats()
    ctx.profile(False)
    energy = ctx.energy(0)          # Eq. 1 over H and over H~ at the finest level, after the run
    ms = e0.elapsed_time(e1)
    evals = s1["evals"] - s0["evals"]
    step_evals = s1["step_evals"] - s0["step_evals"]
    step_gathered = s1["step_gathered"] - s0["step_gathered"]
    step_gathered_h = s1["step_gathered_h"] - s0["step_gathered_h"]
    screened = s1["screened"] - s0["screened"]
    passed = s1["screen_passed"] - s0["screen_passed"]
    step_ms = s1["step_ms"] - s0["step_ms"]
    step_launches = s1["step_timed"] - s0["step_timed"]
    launches = s1["launches"] - s0["launches"]
    outer = s1["outer"]

    realign_ms = None
    if args.realign:
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            to_ref = realign_in()
            vi.affine_unwarp(rgb_d, mask_d, res_d, to_ref, out_d, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        realign_ms = 1e3 * (time.perf_counter() - t) / args.steps

    # end to end through host buffers: upload from pinned memory, fetch to host
    rgb_h = torch.from_numpy(clip.rgb).pin_memory()
    mask_h = torch.from_numpy(clip.mask).pin_memory()
    out_h = torch.empty_like(rgb_h).pin_memory()
    ctx.upload(rgb_h.numpy(), mask_h.numpy())
    ctx.run()
    ctx.fetch_result(out_h.numpy())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    se = ctx.stats()
    t = time.perf_counter()
    for _ in range(args.steps):
        ctx.upload(rgb_h.numpy(), mask_h.numpy())
        ctx.run()
        ctx.fetch_result(out_h.numpy())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t
    e2e_evals = ctx.stats()["evals"] - se["evals"]

    mx, sm = combine_ranks([ms, float(evals), float(n_hole), e2e_s, float(e2e_evals)], dist, "cuda")
    ms_max, evals_tot, hole_tot = mx[0], sm[1], sm[2]
    e2e_max, e2e_evals_tot = mx[3], sm[4]
    ctx.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = _peaks()
    # algorithmic bytes of the step kernel: the source voxels it has to gather
    # (20 B each: 5 FP32 channels; 8 B from the FP16 copy when screening). A
    # candidate equal to a shift already compared needs no gather, and a gather
    # stops once the partial sum shows the candidate cannot win; both leave
    # every decision unchanged.
    gathered_bytes = step_gathered * BYTES_PER_VOXEL_FP32_C5 + step_gathered_h * BYTES_PER_VOXEL_FP16
    achieved = gathered_bytes / (step_ms / 1e3) / 1e9 if step_ms > 0 else None
    traffic = None
    if (NCU_STEP_TRAFFIC and step_launches and NCU_STEP_TRAFFIC["workload"] == args.workload
            and NCU_STEP_TRAFFIC["storage"] == args.storage and NCU_STEP_TRAFFIC["rs_mode"] == args.rs_mode
            and NCU_STEP_TRAFFIC["sub_sweeps"] == args.sub_sweeps and not args.lanes and not args.realign):
        per_voxel = NCU_STEP_TRAFFIC["bytes"] / NCU_STEP_TRAFFIC["gathered_voxels"]
        traffic = per_voxel * step_gathered / step_launches
    line = {
        "metric": METRIC, "value": evals_tot / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "levels": clip.levels, "channels": 5, "storage": args.storage,
                   "random_search": args.rs_mode, "sub_sweeps": args.sub_sweeps,
                   "realign": bool(args.realign),
                   "hole_voxels": n_hole, "parallelism": f"replicas x{world}",
                   "lanes_per_target": args.lanes or "auto",
                   "l2": "inputs larger than L2: level-0 state about 0.3 GB per clip, rebuilt every step"},
        "inpainted_voxels_per_s": hole_tot * args.steps / (ms_max / 1e3),
        "evals_per_step": evals / args.steps,
        "outer_iterations_per_level": outer[:clip.levels],
        "energy_level0": {"E_H": energy[0], "E_Htilde": energy[1]},
        "realign_ms_per_step": realign_ms,
        "screening": ({"screened": screened, "passed": passed,
                       "pass_rate": passed / screened if screened else None,
                       "fp16_voxels": step_gathered_h, "fp32_voxels": step_gathered}
                      if storage else None),
        "roofline": {"bound": "hbm", "kernel": "k_ann_step + k_ann_step_warp (PatchMatch propagation + random search, every level)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                     "traffic": traffic,
                     "unit_of_work": "gathered source voxel, 20 B (5 FP32 channels) or 8 B (FP16 copy of c0..c3)",
                     "gathered_bytes_per_launch": gathered_bytes / step_launches if step_launches else None,
                     "launches_timed": step_launches,
                     "evals_per_launch": step_evals / step_launches if step_launches else None,
                     "evals_per_s_in_kernel": step_evals / (step_ms / 1e3) if step_ms > 0 else None,
                     "full_eval_bytes": BYTES_PER_EVAL_FP32_C5,
                     "gathered_bytes_per_eval": gathered_bytes / step_evals if step_evals else None,
                     "kernel_ms_share": step_ms / ms if ms > 0 else None},
        "e2e": {"value": e2e_evals_tot / e2e_max, "unit": UNIT,
                "h2d_bytes_per_step": int(clip.rgb.nbytes + clip.mask.nbytes),
                "d2h_bytes_per_step": int(clip.rgb.nbytes)},
        "gpu_launches": launches,
        "lanes_tuned": vi.tune_export().splitlines(),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(clip, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


BATCH_WORKLOAD = "batch48"


def make_batch_clips(rank, n=48):
    """48 layered clips of uneven sizes (W ~ logU[160, 640], H ~ logU[120, 480],
    frames ~ logU[20, 80], hole 3-12%); levels by the rule of Sec. 3.6."""
    from paper_1503_05528_gb300 import synth
    clips = []
    for i, (W, H, T, frac) in enumerate(synth.batch_sizes(n)):
        clips.append(synth.layered_clip(W, H, T, 3, (16, 48), frac, 0,
                                        synth.BASE_SEED + 200 + 1000 * rank + i, name=f"batch_{i}"))
    return clips


def run_batch(args):
    """A step inpaints 48 uneven clips as one batch (vi_batch_*): add and
    prepare every clip, rounds until all are done, fetch every result. The
    same clips run one after another through vi_run give the single-clip
    comparison (bit-identical results, hence the same energies)."""
    import torch

    from paper_1503_05528_gb300 import vi

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vi.load(build_if_missing=True)
    _tune_load(args, vi)
    clips = make_batch_clips(rank)
    dev = [(torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()) for c in clips]
    outs = [torch.empty_like(r) for r, _ in dev]
    n_hole = sum(int(c.mask.sum()) for c in clips)
    n_vox = sum(int(c.mask.size) for c in clips)
    stream = torch.cuda.current_stream()
    storage = 1 if args.storage == "fp16" else 0
    b = vi.Batch(stream=stream.cuda_stream, levels=0, lanes_per_target=args.lanes, storage=storage,
                 sub_sweeps=args.sub_sweeps)

    def step():
        ids = [b.add(r, m, levels=0, seed=1503 + i, clip=i) for i, (r, m) in enumerate(dev)]
        b.run()
        for cid, o in zip(ids, outs):
            b.fetch(cid, o)
        for cid in ids:
            b.remove(cid)

    for _ in range(args.warmup):
        step()
    _tune_save(args, vi)
    b.profile(True)
    s0 = b.stats()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    s1 = b.stats()
    b.profile(False)
    ms = e0.elapsed_time(e1)
    evals = s1["evals"] - s0["evals"]
    step_ms = s1["step_ms"] - s0["step_ms"]
    gathered = s1["gathered"] - s0["gathered"]
    gathered_h = s1["gathered_h"] - s0["gathered_h"]
    screened = s1["screened"] - s0["screened"]
    passed = s1["screen_passed"] - s0["screen_passed"]
    rounds = (s1["rounds"] - s0["rounds"]) / args.steps

    # the same clips one after another through the single-clip path
    torch.cuda.synchronize()
    t = time.perf_counter()
    single_evals = 0
    for i, (r, m) in enumerate(dev):
        with vi.Context(levels=0, seed=1503 + i, clip=i, stream=stream.cuda_stream,
                        lanes_per_target=args.lanes, storage=storage, sub_sweeps=args.sub_sweeps) as ctx:
            ctx.upload(r, m)
            ctx.run()
            ctx.fetch_result(outs[i])
            single_evals += ctx.stats()["evals"]
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t
    b.close()

    mx, sm = combine_ranks([ms, float(evals), float(n_hole), single_s, float(single_evals)], dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    gbytes = gathered * BYTES_PER_VOXEL_FP32_C5 + gathered_h * BYTES_PER_VOXEL_FP16
    achieved = gbytes / (step_ms / 1e3) / 1e9 if step_ms > 0 else None
    line = {
        "metric": METRIC, "value": sm[1] / (mx[0] / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mx[0] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "clips": len(clips), "voxels": n_vox, "hole_voxels": n_hole,
                   "levels": "rule of Sec. 3.6 per clip", "channels": 5, "storage": args.storage,
                   "parallelism": f"replicas x{world}", "lanes_per_target": args.lanes or "auto",
                   "rounds_per_step": rounds,
                   "l2": "inputs larger than L2: about 10 GB of clip state rebuilt every step"},
        "inpainted_voxels_per_s": sm[2] * args.steps / (mx[0] / 1e3),
        "evals_per_step": evals / args.steps,
        "screening": ({"screened": screened, "passed": passed,
                       "pass_rate": passed / screened if screened else None} if storage else None),
        "single_clip_path": {"value": sm[4] / mx[3], "unit": UNIT,
                             "inpainted_voxels_per_s": sm[2] / mx[3], "seconds": mx[3],
                             "note": "the same 48 clips one after another through vi_run; "
                                     "bit-identical results"},
        "roofline": {"bound": "hbm", "kernel": "k_ann_step_batch + k_ann_step_batch_warp (PatchMatch step, all clips)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                     "traffic": None,
                     "unit_of_work": "gathered source voxel, 20 B (5 FP32 channels) or 8 B (FP16 copy of c0..c3)",
                     "kernel_ms_share": step_ms / ms if ms > 0 else None},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


SERVE_WORKLOAD = "serve_poisson4"


def make_serve_pool(rank, n_pool):
    """Distinct clips for the serving workload: layered-motion clips (integer
    camera drift, textured sprites, moving elliptical occlusion tube) with
    sizes W ~ logU[320, 1280], H ~ logU[240, 720], frames ~ logU[30, 120] and
    3-10% occlusion; levels by the rule of Sec. 3.6."""
    from paper_1503_05528_gb300 import synth
    return [synth.fast_layered_clip(W, H, T, frac, synth.BASE_SEED + 5000 + 1000 * rank + i,
                                    name=f"serve_{i}")
            for i, (W, H, T, frac) in enumerate(synth.serve_sizes(n_pool))]


def run_serve(args):
    """A Poisson stream of inpainting requests (mean 4 per second, seeded)
    through the continuous-batching server: admission by an HBM budget,
    clips joining and leaving the running batch between rounds, host buffers
    in and out. Latency = completion - arrival (queueing, upload, preparation,
    iterations, fetch). The plain path serves the same arrivals one request
    at a time through vi_run (FCFS single server; its latencies follow from
    each request's measured service time by the Lindley recursion)."""
    import numpy as np
    import torch

    from paper_1503_05528_gb300 import vi
    from paper_1503_05528_gb300.serve import (CudaBackend, NativeServer, Server, StreamBackend,
                                              poisson_arrivals, run_load)

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vi.load(build_if_missing=True)
    _tune_load(args, vi)
    pool = make_serve_pool(rank, args.serve_pool)
    n = args.requests
    reqs = [(pool[i % len(pool)].rgb, pool[i % len(pool)].mask, {"seed": 7000 + i, "clip": i})
            for i in range(n)]
    arrivals = poisson_arrivals(n, args.rate, seed=1503 + rank)
    hole = [int(pool[i % len(pool)].mask.sum()) for i in range(n)]
    vox = [int(pool[i % len(pool)].mask.size) for i in range(n)]
    stream = torch.cuda.current_stream()
    budget = int(args.hbm_budget_gb * (1 << 30))
    storage = 1 if args.storage == "fp16" else 0
    native = args.serve_backend == "native"
    if args.serve_backend == "batch":
        backend = CudaBackend(stream=stream.cuda_stream, levels=0, use_texture=1, storage=storage)
    elif native:
        backend = NativeServer(budget, args.slots, levels=0, use_texture=1, storage=storage)
    else:
        backend = StreamBackend(max_workers=args.slots, device=local, levels=0, use_texture=1,
                                storage=storage)

    # warm-up: every distinct clip once, alone (also settles the lane autotuner)
    warm = backend if native else Server(backend, budget, max_slots=args.slots)
    for i, c in enumerate(pool[:max(args.warmup, len(pool))]):
        warm.submit(c.rgb, c.mask, seed=1, clip=i)
        while warm.step():
            pass

    _tune_save(args, vi)
    batch = getattr(backend, "batch", None)
    if batch is not None:
        batch.profile(True)
    s0 = batch.stats() if batch is not None else None
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if native:
        backend.done.clear()
        backend.next_ticket, backend.max_concurrent, backend.rounds = 0, 0, 0
        srv = backend
    else:
        srv = Server(backend, budget, max_slots=args.slots)
    wall, srv = run_load(srv, reqs, arrivals)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    lat = np.array([srv.done[t].latency for t in range(n)])
    failed = sum(1 for r in srv.done.values() if r.info.get("failed"))
    if batch is not None:
        s1 = batch.stats()
        batch.profile(False)
        evals = s1["evals"] - s0["evals"]
        step_ms = s1["step_ms"] - s0["step_ms"]
        gathered = s1["gathered"] - s0["gathered"]
        gathered_h = s1["gathered_h"] - s0["gathered_h"]
        rounds = s1["rounds"] - s0["rounds"]
    else:
        evals = None                 # counted below from the plain path (the same evaluations)
        step_ms = gathered = gathered_h = 0
        rounds = srv.rounds
    served = {t: srv.done[t].result for t in range(min(n, len(pool)))}
    backend.close()

    # plain path: each request alone through vi_run, back to back
    service, single_evals = [], 0
    torch.cuda.synchronize()
    for i, (rgb, mask, job) in enumerate(reqs):
        t = time.perf_counter()
        with vi.Context(levels=0, use_texture=1, stream=stream.cuda_stream, **job) as ctx:
            ctx.upload(rgb, mask)
            ctx.run()
            out = ctx.fetch_result()
            single_evals += ctx.stats()["evals"]
        service.append(time.perf_counter() - t)
        if i in served:
            assert (out.view(np.uint32) == served[i].view(np.uint32)).all(), \
                f"request {i}: served result differs from vi_run alone"
    free, lat1 = 0.0, []
    for a, s in zip(arrivals, service):
        free = max(free, a) + s
        lat1.append(free - a)
    lat1 = np.array(lat1)
    plain_wall = free

    if evals is None:
        evals = single_evals         # every request makes the evaluations it makes alone
    mx, sm = combine_ranks([wall, float(evals), float(sum(hole)), plain_wall, float(single_evals)],
                           dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    gbytes = gathered * BYTES_PER_VOXEL_FP32_C5 + gathered_h * BYTES_PER_VOXEL_FP16
    achieved = gbytes / (step_ms / 1e3) / 1e9 if step_ms > 0 else None
    pct = lambda x, q: float(np.percentile(x, q, method="inverted_cdf"))  # noqa: E731
    line = {
        "metric": METRIC, "value": sm[1] / mx[0], "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * mx[0],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "requests": n, "rate_per_s": args.rate,
                   "distinct_clips": len(pool), "voxels_mean": float(np.mean(vox)),
                   "hole_voxels": int(sum(hole)), "hbm_budget_gb": args.hbm_budget_gb,
                   "max_slots": args.slots, "backend": args.serve_backend,
                   "levels": "rule of Sec. 3.6 per clip", "channels": 5,
                   "storage": args.storage, "parallelism": f"replicas x{world}",
                   "step": "the whole arrival stream, host buffers in and out",
                   "l2": "inputs larger than L2: every request uploads and rebuilds its state"},
        "latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": float(lat.max()),
                      "mean": float(lat.mean())},
        "inpainted_voxels_per_s": sm[2] / mx[0],
        "requests_per_s": n * world / mx[0],
        "failed": failed, "max_concurrent": srv.max_concurrent, "rounds": rounds,
        "plain_fp32_path": {"value": sm[4] / mx[3], "unit": UNIT,
                            "latency_s": {"p50": pct(lat1, 50), "p99": pct(lat1, 99),
                                          "max": float(lat1.max())},
                            "inpainted_voxels_per_s": sm[2] / mx[3],
                            "busy_s": float(sum(service)),
                            "note": "same arrivals, one request at a time through vi_run"},
        "roofline": ({"bound": "hbm", "kernel": "k_ann_step_batch + k_ann_step_batch_warp (PatchMatch step, all clips)",
                      "achieved": achieved, "peak": peak, "unit": "GB/s",
                      "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                      "traffic": None,
                      "unit_of_work": "gathered source voxel, 20 B (5 FP32 channels) or 8 B (FP16 copy of c0..c3)",
                      "kernel_ms_share": step_ms / (1e3 * wall) if wall > 0 else None}
                     if args.serve_backend == "batch" else None),
        "e2e": {"value": sm[1] / mx[0], "unit": UNIT,
                "h2d_bytes_per_step": int(sum(v * 13 for v in vox)),
                "d2h_bytes_per_step": int(sum(v * 12 for v in vox))},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_slabs(args):
    """One clip's whole inpainting split by frames over --slabs contexts on
    this GPU (vi_run_slabs): the decomposition a multi-GPU run of one clip
    would use, with its boundary copies made on one device. Reports the
    evaluation rate, the bytes exchanged per step and the same clip's time
    through vi_run, measured in the same process; the results are identical
    (checked here, bit for bit)."""
    import numpy as np
    import torch

    from paper_1503_05528_gb300 import vi

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    vi.load(build_if_missing=True)
    _tune_load(args, vi)
    clip = make_clip(rank, args.workload)
    rgb_d = torch.from_numpy(clip.rgb).cuda()
    mask_d = torch.from_numpy(clip.mask).cuda()
    out_d, ref_d = torch.empty_like(rgb_d), torch.empty_like(rgb_d)
    stream = torch.cuda.current_stream()
    cfg = dict(levels=clip.levels, use_texture=1, seed=1503 + rank, clip=rank, lanes_per_target=args.lanes,
               rs_mode=1 if args.rs_mode == "multi" else 0, sub_sweeps=args.sub_sweeps)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = [fn() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, out[-1]

    ms, (_, st, nbytes) = timed(lambda: vi.run_slabs(rgb_d, mask_d, args.slabs, out=out_d,
                                                     stream=stream.cuda_stream, **cfg))
    evals = st["evals"]

    def alone():
        with vi.Context(stream=stream.cuda_stream, **cfg) as ctx:
            ctx.upload(rgb_d, mask_d)
            ctx.run()
            ctx.fetch_result(ref_d)
            return ctx.stats()["evals"]

    ms1, evals1 = timed(alone)
    torch.cuda.synchronize()
    same = bool((out_d.view(torch.int32) == ref_d.view(torch.int32)).all().item()) and evals == evals1
    assert same, "slab result differs from vi_run"
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": evals / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "levels": clip.levels, "slabs": args.slabs,
                       "slab_devices": "all on this GPU, one stream"},
            "exchanged_bytes_per_step": nbytes, "identical_to_vi_run": same,
            "vi_run": {"ms_per_step": ms1, "value": evals1 / (ms1 / 1e3), "unit": UNIT},
            "roofline": None, "note": "the coarsest level runs in every slab's context"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=sorted(WORKLOADS) + [BATCH_WORKLOAD, SERVE_WORKLOAD])
    ap.add_argument("--slabs", type=int, default=1,
                    help="split one clip by frames over this many contexts on this GPU (vi_run_slabs)")
    ap.add_argument("--requests", type=int, default=200, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=4.0, help="serving: mean arrivals per second")
    ap.add_argument("--serve-pool", type=int, default=16, help="serving: distinct clips")
    ap.add_argument("--hbm-budget-gb", type=float, default=96.0, help="serving: admission budget")
    ap.add_argument("--slots", type=int, default=32, help="serving: most requests admitted at once")
    ap.add_argument("--serve-backend", default="native", choices=["streams", "batch", "native"],
                    help="serving: one stream per request by size priority (Python front), one shared batch, "
                         "or the library server (vi_server_*)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"],
                    help="channel storage: fp32, or fp16 copies screened before the FP32 distance")
    ap.add_argument("--rs-mode", default="eq3", choices=["eq3", "multi"],
                    help="random search: one radius per iteration (Eq. 3) or every radius")
    ap.add_argument("--sub-sweeps", type=int, default=2,
                    help="propagation sweeps per iteration (2, the library's default)")
    ap.add_argument("--realign", action="store_true",
                    help="AlignVideo (Sec. 3.4) before and UnwarpVideo after every inpainting")
    ap.add_argument("--tune-save", default=None, help="write the lanes autotuning table after warm-up")
    ap.add_argument("--tune-load", default=None, help="import a lanes autotuning table before warm-up")
    ap.add_argument("--lanes", type=int, default=0,
                    help="GPU lanes per target in the search kernels (0: chosen per level)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == BATCH_WORKLOAD:
        return run_batch(args)
    if args.workload == SERVE_WORKLOAD:
        return run_serve(args)
    if args.slabs > 1:
        return run_slabs(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
