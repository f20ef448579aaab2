#!/usr/bin/env python
"""Benchmark of the inpainting hot path on GB300.

Default workload (batch48): 48 synthetic layered-motion clips of uneven sizes
(W ~ logU[160, 640], H ~ logU[120, 480], frames ~ logU[20, 80], 3-12%
occlusion tubes; 163M voxels, levels by the rule of Sec. 3.6), inpainted as
one batch through the C ABI (vi_batch_add_many / vi_batch_run /
vi_batch_fetch / vi_batch_remove): pyramids and features, initialisations,
onion peels, per level the PatchMatch search and reconstruction rounds until
each clip's stopping rule, level transitions and the final best-patch step.
A step is the whole batch. Storage: FP16 copies screening the random-search
candidates at levels larger than L2 (--storage fp16, the default; results
identical to --storage fp32). --workload layered_320x240x60 / layered_1280x720x100 runs one
clip per step through vi_run; serve_poisson4 the serving stream.

Output: one JSON line (rank 0). `value` is inpainted (occluded) voxels per
second over the whole job (all ranks), inputs resident in device memory when
the timed region starts; `evals_per_s` is the patch-distance evaluation rate
of the same run (every candidate of Algorithm 1 that lands in D~, whether or
not exact pruning let it skip its gather). `e2e` is the same metric with the
inputs uploaded from pinned host buffers and every result fetched to host
memory inside the timed region (`e2e.phases`: one more such step, untimed,
split into adding the clips, the rounds and fetching). `roofline` is the PatchMatch step kernel's
gathered source bytes over its CUDA-event time against the measured HBM copy
bandwidth, with the per-evaluation count beside it. `cpu_baseline` times the
CPU oracle on the host cores, one clip per core, on a bounded sample of the
same workload.

Multi-GPU (torchrun): replicas only -- each rank inpaints its own clips; no
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

METRIC = "patch-distance evals/s and inpainted voxels/s vs HBM roofline; serving p50/p99"
UNIT = "inpainted voxels/s"
WORKLOAD = "batch48"
BYTES_PER_VOXEL_FP32_C5 = 5 * 4           # one source voxel: 5 FP32 channels
BYTES_PER_EVAL_FP32_C5 = 125 * BYTES_PER_VOXEL_FP32_C5   # a whole source patch
BYTES_PER_VOXEL_FP16 = 4 * 2             # channels c0..c3 of a voxel from the FP16 copy

# DRAM bytes (read + write) of the PatchMatch step kernel per gathered source
# voxel, from one ncu capture of a few launches of that kernel (the profiles
# directory names the command), keyed by (workload, storage, propagation
# sweeps per iteration). A run of the same configuration scales it by the
# source voxels its launches gathered. Empty while the kernels have changed
# since the capture.
NCU_STEP_TRAFFIC = {
    # 1,440 launches of one batch step of the first 8 clips (61.89 GB read +
    # 2.05 GB written over 18.33 G gathered voxels), scaled to the 48 clips by
    # gathered voxels (profiles/k_ann_step_batch_warp_batch48_8clips.md)
    ("batch48", "fp32", 2): (61.89e9 + 2.045e9) / 18.33e9,
    # 1,800 launches of one batch step of the first 14 clips with FP16
    # storage (142.1 GB read + 9.68 GB written over 43.17 G gathered voxels:
    # 39.45 G from FP32 channels, 3.71 G from FP16 copies), scaled the same way
    # (profiles/k_ann_step_batch_warp_batch48_14clips_fp16.md)
    ("batch48", "fp16", 2): (142.10e9 + 9.678e9) / 43.166e9,
}

# What the ncu counters of the step kernel show binds it (the roofline object
# reports the gather against the HBM copy bandwidth; this says what actually
# limits it).
STEP_LIMITER = ("latency of dependent gathers served by L1/L2 (ncu: long-scoreboard stalls dominate, "
                "L1 throughput the next limit, DRAM throughput low); not HBM bandwidth")


def step_traffic(args, workload, gathered, gathered_h, launches):
    key = (workload, args.storage, args.sub_sweeps)
    per_voxel = NCU_STEP_TRAFFIC.get(key)
    if per_voxel is None or not launches or args.lanes or getattr(args, "realign", False) or \
            getattr(args, "rs_mode", "eq3") != "eq3":
        return None
    return per_voxel * (gathered + gathered_h) / launches


def step_roofline(gathered, gathered_h, step_evals, step_ms, wall_ms, peak, peak_kind, kernel, traffic,
                  launches):
    """The roofline object of the step kernel: bytes it gathers (20 B per FP32
    source voxel, 8 B per FP16 one) over its CUDA-event time against the
    measured HBM copy bandwidth; beside it the same launches counted at a
    whole patch per evaluation (125 voxels x 20 B)."""
    if step_ms <= 0:
        return None
    gbytes = gathered * BYTES_PER_VOXEL_FP32_C5 + gathered_h * BYTES_PER_VOXEL_FP16
    achieved = gbytes / (step_ms / 1e3) / 1e9
    full = step_evals * BYTES_PER_EVAL_FP32_C5 / (step_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
            "unit_of_work": "one gathered source voxel: 20 B (5 FP32 channels) or 8 B (FP16 copy of c0..c3)",
            "gathered_bytes_per_launch": gbytes / launches if launches else None,
            "launches_timed": launches,
            "gathered_voxels_per_eval": (gathered + gathered_h) / step_evals if step_evals else None,
            "limiter": STEP_LIMITER,
            "per_evaluation_unit": {
                "bytes_per_eval": BYTES_PER_EVAL_FP32_C5, "achieved": full, "frac": full / peak,
                "evals_per_s_in_kernel": step_evals / (step_ms / 1e3),
                "note": "every counted evaluation at a whole 125-voxel FP32 patch; exact pruning skips most "
                        "of each patch and L1/L2 serve most of the rest, so this is not a bandwidth"},
            "kernel_ms_share": step_ms / wall_ms if wall_ms > 0 else None}


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


def make_clip(rank, workload="layered_320x240x60"):
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
    shift map from the oracle's initialisation. The search is the one the GPU
    path runs (the Jacobi schedule with its propagation sweeps per
    iteration), so its evaluation counts are comparable."""

    def __init__(self, clip, sub_sweeps=2, schedule="JAC"):
        import numpy as np
        from oracle import oracle as O
        self.O = O
        self.sub_sweeps = sub_sweeps
        self.schedule = schedule
        levels = clip.levels or 1
        lv = O.build_pyramid(clip.rgb, clip.mask, levels, True)[0]
        lv.x[lv.hole == 1] = 0.5
        lv.phi = O.init_nnf(lv.htilde, lv.dtilde, (1503, 0), O.tag(O.PURPOSE_INIT, 0))
        lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
        self.lv = lv
        self.T = lv.hole.shape[0]
        self.next_t = 2

    def slab(self, frames):
        """One ANN search (rescore + 10 PatchMatch iterations of Algorithm 1)
        over the targets of `frames` consecutive frames. Returns (evals,
        seconds)."""
        import numpy as np
        lv = self.lv
        t0 = self.next_t
        self.next_t = 2 + (self.next_t - 2 + frames) % max(self.T - 4 - frames, 1)
        tgt = np.zeros_like(lv.htilde)
        tgt[t0:t0 + frames] = lv.htilde[t0:t0 + frames]
        phi = lv.phi.copy()
        d2 = lv.d2.copy()
        s = time.perf_counter()
        ev = self.O.ann(lv.x, tgt, lv.dtilde, phi, d2, n_pm=10, schedule=self.schedule, key=(1503, 0),
                        tag_base=self.O.tag(self.O.PURPOSE_SEARCH, 0, 0), sub_sweeps=self.sub_sweeps)
        return ev, time.perf_counter() - s


def _oracle_worker(conn, clip_spec, sub_sweeps):
    """A spawned process holding one clip's oracle sample: answers each
    number of seconds received with (evaluations, seconds, frames) of
    two-frame slab searches run for at least that long; None ends it."""
    clip = _make_clip_from_spec(clip_spec)
    smp = OracleSample(clip, sub_sweeps=sub_sweeps)
    conn.send(("ready", clip.name))
    while True:
        seconds = conn.recv()
        if seconds is None:
            break
        evals, el, frames = 0, 0.0, 0
        while el < seconds:
            ev, dt = smp.slab(2)
            evals += ev
            el += dt
            frames += 2
        conn.send((evals, el, frames))
    conn.close()


class OracleWorkers:
    """One spawned process per host core, each with its own clip of the
    workload (clips spread one per core), for timing the CPU oracle on all
    cores at once. Spawned, not forked: the parent may hold a CUDA context."""

    def __init__(self, specs, sub_sweeps):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.procs, self.conns = [], []
        for spec in specs:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, spec, sub_sweeps), daemon=True)
            p.start()
            self.procs.append(p)
            self.conns.append(a)
        self.names = [c.recv()[1] for c in self.conns]

    def run(self, seconds):
        """(evaluations of all workers, wall seconds, frames) of one bounded
        sample: every worker searches for about `seconds`."""
        t = time.perf_counter()
        for c in self.conns:
            c.send(seconds)
        res = [c.recv() for c in self.conns]
        return sum(r[0] for r in res), time.perf_counter() - t, sum(r[2] for r in res)

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)
            if p.is_alive():
                p.terminate()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(specs, seconds, sub_sweeps, evals_per_voxel, workload):
    """The oracle on the host cores, one clip per core (one core for a single
    clip), as it stands: its Jacobi search over two-frame slabs of each
    clip's level-0 targets for about `seconds`. Its evaluation rate, divided
    by the evaluations the GPU run made per inpainted voxel (the oracle makes
    the same evaluations for the same state), gives the extrapolated
    inpainted voxels/s."""
    w = OracleWorkers(specs, sub_sweeps)
    try:
        evals, wall, frames = w.run(seconds)
    finally:
        w.close()
    rate = evals / wall
    return {"value": rate / evals_per_voxel, "unit": UNIT, "cores": len(specs), "kind": "oracle",
            "evals_per_s": rate,
            "sample": f"{workload}: {len(specs)} clip(s), one per core; the oracle's search (rescore + 10 "
                      f"PatchMatch iterations, {sub_sweeps} propagation sweeps each) over two-frame slabs of "
                      f"each clip's level-0 targets, {frames} frames in all, {evals} evaluations in "
                      f"{wall:.1f} s; inpainted voxels/s extrapolated by the GPU run's "
                      f"{evals_per_voxel:.0f} evaluations per inpainted voxel"}


def run_reference(args):
    """The CPU oracle as the reference arm: on the host cores, one clip per
    core, each step a bounded sample (every worker searches two-frame slabs of
    its clip's level-0 targets for about --ref-seconds), reported in the GPU
    arm's unit by the workload's evaluations per inpainted voxel."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    workload = args.workload
    if workload not in EVALS_PER_HOLE_VOXEL or EVALS_PER_HOLE_VOXEL[workload] is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no evaluation count per inpainted voxel "
                                                                f"stored for {workload}"}), flush=True)
        return 0
    epv = EVALS_PER_HOLE_VOXEL[workload]
    specs = oracle_specs(workload)
    w = OracleWorkers(specs, args.sub_sweeps)
    try:
        for _ in range(args.warmup):
            w.run(args.ref_seconds)
        evals, wall, frames = 0, 0.0, 0
        for _ in range(args.steps):
            ev, dt, fr = w.run(args.ref_seconds)
            evals += ev
            wall += dt
            frames += fr
    finally:
        w.close()
    rate = evals / wall
    value = rate / epv
    sample = (f"each step: {len(specs)} clip(s) of {workload}, one per core; the oracle's search (rescore + "
              f"10 PatchMatch iterations, {args.sub_sweeps} propagation sweeps each) over two-frame slabs of "
              f"each clip's level-0 targets for about {args.ref_seconds:.1f} s; inpainted voxels/s "
              f"extrapolated by {epv:.0f} evaluations per inpainted voxel")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "sub_sweeps": args.sub_sweeps, "sample": sample},
            "evals_per_s": rate,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(specs), "kind": "oracle",
                             "evals_per_s": rate, "sample": sample},
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
    storage = {"fp32": 0, "fp16": 1, "fp16-all": 2}[args.storage]
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
    evals_per_voxel = evals / (n_hole * args.steps)
    line = {
        "metric": METRIC, "value": hole_tot * args.steps / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "levels": clip.levels, "channels": 5, "storage": args.storage,
                   "random_search": args.rs_mode, "sub_sweeps": args.sub_sweeps,
                   "realign": bool(args.realign),
                   "hole_voxels": n_hole, "parallelism": f"replicas x{world}",
                   "lanes_per_target": args.lanes or "auto",
                   "l2": "inputs larger than L2: level-0 state about 0.3 GB per clip, rebuilt every step"},
        "evals_per_s": evals_tot / (ms_max / 1e3),
        "evals_per_step": evals / args.steps,
        "evals_per_inpainted_voxel": evals_per_voxel,
        "gathered_evals_per_s": ((step_gathered * BYTES_PER_VOXEL_FP32_C5 + step_gathered_h * BYTES_PER_VOXEL_FP16)
                                 / BYTES_PER_EVAL_FP32_C5 * world / (ms_max / 1e3)),
        "outer_iterations_per_level": outer[:clip.levels],
        "energy_level0": {"E_H": energy[0], "E_Htilde": energy[1]},
        "realign_ms_per_step": realign_ms,
        "screening": ({"screened": screened, "passed": passed,
                       "pass_rate": passed / screened if screened else None,
                       "fp16_voxels": step_gathered_h, "fp32_voxels": step_gathered}
                      if storage else None),
        "roofline": step_roofline(step_gathered, step_gathered_h, step_evals, step_ms, ms, peak, peak_kind,
                                  "k_ann_step_warp + k_ann_step (PatchMatch propagation + random search, "
                                  "every level)",
                                  step_traffic(args, args.workload, step_gathered, step_gathered_h, step_launches),
                                  step_launches),
        "e2e": {"value": hole_tot * args.steps / e2e_max, "unit": UNIT,
                "h2d_bytes_per_step": int(clip.rgb.nbytes + clip.mask.nbytes),
                "d2h_bytes_per_step": int(clip.rgb.nbytes)},
        "gpu_launches": launches,
        "lanes_tuned": vi.tune_export().splitlines(),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(oracle_specs(args.workload), args.cpu_seconds, args.sub_sweeps,
                                            evals_per_voxel, args.workload)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


BATCH_WORKLOAD = "batch48"


def make_batch_clip(rank, i, n=48):
    """Clip i of the 48 layered clips of uneven sizes (W ~ logU[160, 640],
    H ~ logU[120, 480], frames ~ logU[20, 80], hole 3-12%); levels by the
    rule of Sec. 3.6."""
    from paper_1503_05528_gb300 import synth
    W, H, T, frac = synth.batch_sizes(n)[i]
    return synth.layered_clip(W, H, T, 3, (16, 48), frac, 0, synth.BASE_SEED + 200 + 1000 * rank + i,
                              name=f"batch_{i}")


def make_batch_clips(rank, n=48):
    return [make_batch_clip(rank, i, n) for i in range(n)]


def _make_clip_from_spec(spec):
    """("batch", rank, i) or ("clip", rank, workload)."""
    if spec[0] == "batch":
        return make_batch_clip(spec[1], spec[2])
    return make_clip(spec[1], spec[2])


def oracle_specs(workload, rank=0):
    """The clips the CPU oracle is timed on: one per host core for the batch
    (the first min(cores, 48) clips), the clip itself for a single clip."""
    if workload == BATCH_WORKLOAD:
        return [("batch", rank, i) for i in range(min(host_cores(), 48))]
    return [("clip", rank, workload)]


# Evaluations per inpainted voxel of a whole inpainting of each workload in
# the default configuration (two propagation sweeps per iteration, Eq. 3
# random search): a property of the workload, not a timing -- the GPU path's
# count, which equals the oracle's for the same state (tests compare the
# counts). The GPU arm measures it on every run; the --impl reference arm,
# which has no GPU, converts the oracle's evaluation rate with it.
# (Measured on GB300: batch48 11,715,304,841 evaluations for 13,414,074
# occluded voxels; layered_320x240x60 the same way.)
EVALS_PER_HOLE_VOXEL = {"batch48": 11715304841 / 13414074, "layered_320x240x60": 506.897988193932,
                        "layered_1280x720x100": None}


def run_batch(args):
    """A step inpaints 48 uneven clips as one batch (vi_batch_*): add and
    prepare every clip (concurrently, vi_batch_add_many), rounds until all are
    done, fetch every result; the inputs are resident in device memory. The e2e leg repeats the step from
    pinned host buffers to host buffers. The same clips one after another
    through vi_run give the single-clip comparison (bit-identical results)."""
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
    clips = [make_batch_clip(rank, i) for i in range(min(args.clips, 48))]
    dev = [(torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()) for c in clips]
    outs = [torch.empty_like(r) for r, _ in dev]
    n_hole = sum(int(c.mask.sum()) for c in clips)
    n_vox = sum(int(c.mask.size) for c in clips)
    stream = torch.cuda.current_stream()
    storage = {"fp32": 0, "fp16": 1, "fp16-all": 2}[args.storage]
    kw = dict(levels=0, lanes_per_target=args.lanes, storage=storage, sub_sweeps=args.sub_sweeps)
    b = vi.Batch(stream=stream.cuda_stream, **kw)
    counter = vi.Context(**kw)      # reads the library's launch counter

    def add_all(inputs):
        # every clip uploaded and prepared concurrently (vi_batch_add_many)
        return b.add_many([(r, m, dict(levels=0, seed=1503 + i, clip=i)) for i, (r, m) in enumerate(inputs)])

    def step(inputs, outputs):
        ids = add_all(inputs)
        b.run()
        for cid, o in zip(ids, outputs):
            b.fetch(cid, o)
        for cid in ids:
            b.remove(cid)

    for _ in range(args.warmup):
        step(dev, outs)
    _tune_save(args, vi)
    b.profile(True)
    s0 = b.stats()
    l0 = counter.stats()["launches"]
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
        step(dev, outs)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    s1 = b.stats()
    launches = counter.stats()["launches"] - l0
    b.profile(False)
    ms = e0.elapsed_time(e1)
    evals = s1["evals"] - s0["evals"]
    step_ms = s1["step_ms"] - s0["step_ms"]
    step_evals = s1["step_evals"] - s0["step_evals"]
    gathered = s1["gathered"] - s0["gathered"]
    gathered_h = s1["gathered_h"] - s0["gathered_h"]
    screened = s1["screened"] - s0["screened"]
    passed = s1["screen_passed"] - s0["screen_passed"]
    rounds = (s1["rounds"] - s0["rounds"]) / args.steps
    step_launches = (s1["rounds"] - s0["rounds"]) * 10 * args.sub_sweeps   # n_pm sweeps x sub-sweeps per round

    # where one step's time goes (one more step, outside the timed region):
    # adding and preparing the clips (upload, pyramid, initialisation, onion
    # peel), the rounds, fetching and removing
    torch.cuda.synchronize()
    phase = {}
    t = time.perf_counter()
    ids = add_all(dev)
    torch.cuda.synchronize()
    phase["add_ms"] = 1e3 * (time.perf_counter() - t)
    t = time.perf_counter()
    b.run()
    torch.cuda.synchronize()
    phase["rounds_ms"] = 1e3 * (time.perf_counter() - t)
    t = time.perf_counter()
    for cid, o in zip(ids, outs):
        b.fetch(cid, o)
    for cid in ids:
        b.remove(cid)
    torch.cuda.synchronize()
    phase["fetch_remove_ms"] = 1e3 * (time.perf_counter() - t)

    # end to end through host buffers: every step uploads its clips from
    # pinned host memory and fetches every result to pinned host memory
    e2e_steps = 0 if args.device_only else max(1, min(args.steps, 5))
    e2e_s = 0.0
    e2e_phase = {}
    if e2e_steps:
        host_in = [(torch.from_numpy(c.rgb).pin_memory().numpy(), torch.from_numpy(c.mask).pin_memory().numpy())
                   for c in clips]
        host_out = [torch.empty(c.rgb.shape, dtype=torch.float32).pin_memory().numpy() for c in clips]
        step(host_in, host_out)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            step(host_in, host_out)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t
        assert all((h == o.cpu().numpy()).all() for h, o in zip(host_out, outs)), "host and device runs differ"
        # where one host-buffer step's time goes (one more step, untimed):
        # adding the clips from pinned host memory (the uploads included), the
        # rounds, fetching every result into pinned host memory
        torch.cuda.synchronize()
        t = time.perf_counter()
        ids = add_all(host_in)
        torch.cuda.synchronize()
        e2e_phase["add_ms"] = 1e3 * (time.perf_counter() - t)
        t = time.perf_counter()
        b.run()
        torch.cuda.synchronize()
        e2e_phase["rounds_ms"] = 1e3 * (time.perf_counter() - t)
        t = time.perf_counter()
        for cid, o in zip(ids, host_out):
            b.fetch(cid, o)
        e2e_phase["fetch_ms"] = 1e3 * (time.perf_counter() - t)
        for cid in ids:
            b.remove(cid)

    # the same clips one after another through the single-clip path
    torch.cuda.synchronize()
    t = time.perf_counter()
    single_evals = 0
    for i, (r, m) in enumerate([] if args.device_only else dev):
        with vi.Context(seed=1503 + i, clip=i, stream=stream.cuda_stream, **kw) as ctx:
            ctx.upload(r, m)
            ctx.run()
            ctx.fetch_result(outs[i])
            single_evals += ctx.stats()["evals"]
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t
    b.close()
    counter.close()

    mx, sm = combine_ranks([ms, float(evals), float(n_hole), single_s, float(single_evals), e2e_s], dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    ms_max, evals_tot, hole_tot = mx[0], sm[1], sm[2]
    peak, peak_kind = _peaks()
    evals_per_voxel = evals / (n_hole * args.steps)
    line = {
        "metric": METRIC, "value": hole_tot * args.steps / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD if len(clips) == 48 else f"{BATCH_WORKLOAD}[:{len(clips)}]",
                   "clips": len(clips), "voxels": n_vox, "hole_voxels": n_hole,
                   "levels": "rule of Sec. 3.6 per clip", "channels": 5, "storage": args.storage,
                   "sub_sweeps": args.sub_sweeps, "random_search": "eq3",
                   "parallelism": f"replicas x{world}", "lanes_per_target": args.lanes or "auto",
                   "rounds_per_step": rounds,
                   "l2": "inputs larger than L2: about 10 GB of clip state rebuilt every step"},
        "evals_per_s": evals_tot / (ms_max / 1e3),
        "evals_per_step": evals / args.steps,
        "evals_per_inpainted_voxel": evals_per_voxel,
        "gathered_evals_per_s": (gathered * 20 + gathered_h * 8) / BYTES_PER_EVAL_FP32_C5 * world / (ms_max / 1e3),
        "step_phases": phase,
        "screening": ({"screened": screened, "passed": passed,
                       "pass_rate": passed / screened if screened else None} if storage else None),
        "single_clip_path": ({"value": sm[2] / mx[3], "unit": UNIT, "evals_per_s": sm[4] / mx[3],
                              "seconds": mx[3],
                              "note": "the same clips one after another through vi_run; bit-identical results"}
                             if not args.device_only else None),
        "roofline": step_roofline(gathered, gathered_h, step_evals, step_ms, ms, peak, peak_kind,
                                  "k_ann_step_batch_warp + k_ann_step_batch (PatchMatch step, all clips)",
                                  step_traffic(args, BATCH_WORKLOAD, gathered, gathered_h, step_launches),
                                  step_launches),
        "e2e": ({"value": hole_tot * e2e_steps / mx[5], "unit": UNIT,
                 "steps": e2e_steps,
                 "h2d_bytes_per_step": int(sum(c.rgb.nbytes + c.mask.nbytes for c in clips)),
                 "d2h_bytes_per_step": int(sum(c.rgb.nbytes for c in clips)),
                 "phases": e2e_phase} if e2e_steps else None),
        "gpu_launches": launches,
        "lanes_tuned": vi.tune_export().splitlines(),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline and not args.device_only:
        line["cpu_baseline"] = cpu_baseline(oracle_specs(BATCH_WORKLOAD), args.cpu_seconds, args.sub_sweeps,
                                            evals_per_voxel, BATCH_WORKLOAD)
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
    storage = {"fp32": 0, "fp16": 1, "fp16-all": 2}[args.storage]
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
        "metric": METRIC, "value": sm[2] / mx[0], "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * mx[0],
        "evals_per_s": sm[1] / mx[0],
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
        "plain_fp32_path": {"value": sm[2] / mx[3], "unit": UNIT, "evals_per_s": sm[4] / mx[3],
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
        "e2e": {"value": sm[2] / mx[0], "unit": UNIT,
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
    n_hole = int(clip.mask.sum())
    line = {"metric": METRIC, "value": n_hole / (ms / 1e3), "unit": UNIT, "evals_per_s": evals / (ms / 1e3),
            "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "levels": clip.levels, "slabs": args.slabs,
                       "slab_devices": "all on this GPU, one stream"},
            "exchanged_bytes_per_step": nbytes, "identical_to_vi_run": same,
            "vi_run": {"ms_per_step": ms1, "value": n_hole / (ms1 / 1e3), "unit": UNIT},
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
    ap.add_argument("--device-only", action="store_true",
                    help="batch: time the device-resident steps only (no e2e, single-clip or CPU legs), "
                         "for profiler runs")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU baseline: seconds of oracle search per core")
    ap.add_argument("--ref-seconds", type=float, default=2.0,
                    help="--impl reference: seconds of oracle search per core and step")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=sorted(WORKLOADS) + [BATCH_WORKLOAD, SERVE_WORKLOAD])
    ap.add_argument("--clips", type=int, default=48,
                    help="batch: the first N of the 48 clips (a smaller case for profiling)")
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
    ap.add_argument("--storage", default="fp16", choices=["fp32", "fp16", "fp16-all"],
                    help="channel storage: fp32; fp16 copies that screen random-search candidates before the "
                         "FP32 distance at levels larger than L2 (fp16) or at every level (fp16-all)")
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
    if args.workload == BATCH_WORKLOAD and args.slabs <= 1:
        return run_batch(args)
    if args.workload == SERVE_WORKLOAD:
        return run_serve(args)
    if args.slabs > 1:
        if args.workload not in WORKLOADS:
            args.workload = "layered_320x240x60"
        return run_slabs(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
