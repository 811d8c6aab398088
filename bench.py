"""Benchmark: marginal-gain throughput of the GB300 path on the seeded synthetic workloads.

Default (N=1), one JSON line:
- headline: the large workload, 800x800x200 voxels at 0.05 m, a 2000-node RRT of depth <= 15,
  320x240 rays, K = 36 yaws, 8 m range. One step = one whole-tree evaluation (every node, yaw and
  ray: count, ancestor test, yaw argmax, depth render) through the device-resident call.
    value = marginal-gain rays per second = nodes * K * W * H / device time, inputs resident in HBM,
            CUDA events on the library's stream, L2 flushed between steps;
    e2e   = the same metric through the public host-array call (mig_tree_eval), host<->device copies
            inside the timed region;
- paper_scale: the same measurement on the 400x400x100, 500-node, 160x120, K = 16 workload;
- batched: 64 trees on 64 maps (50-2000 nodes, ray grids 64x48 ... 320x240) in one batched call
  against 64 sequential plain calls, repeated, with the spread;
- serving: 16 robots on 4 maps with Poisson arrivals through the continuous-batching server against
  the same requests as lone calls: at the specified 20 Hz per robot (far above capacity: the queue
  grows) and at a load the GPU can keep up with; p50 / p99 latency and replans/s;
- roofline of the dominant kernel, cpu_baseline (the CPU oracle on this host's cores, on a bounded
  sample of the large workload), the gap of the depth-buffer gain to the exact one.
Multi-GPU (torchrun, one rank per GPU): replicas only. Every rank evaluates its own seeded tree per
step, no collective on the data path; value = all ranks' rays / max-over-ranks time.

--impl reference: the CPU oracle (the plain C restatement of the method) timed on this host's cores
on a bounded sample of the same workload, same metric and unit.
--workload large | paper_scale | tiny | batched | batched_small | serving: one part alone (the
single-tree workloads also time every gain mode through the public call and report each mode's gap
to the exact marginal gain from the oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "marginal-gain rays/s & replans/s; p50/p99 replan latency, batched vs plain"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
DTYPE = "int32/int64 fixed point (u8 map)"
DATA = "synthetic (seeded; stands in for the paper's Gazebo worlds)"


# ----------------------------------------------------------------------------- utilities
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def l2_flush_buffer(torch, dev):
    return torch.empty(int(256 * 2 ** 20), dtype=torch.uint8, device=dev)


def max_over_ranks(x, device=None):
    """Largest value over all ranks (a no-op on one process); gloo or NCCL."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def spread(xs):
    xs = [float(x) for x in xs]
    return {"median": float(np.median(xs)), "min": min(xs), "max": max(xs), "n": len(xs)}


# -------------------------------------------------------------------- kernels and roofline
# Source files whose code (comments and blank lines removed) an ncu summary is tied to.
KERNEL_SOURCES = {
    "cast_kernel": ("voxcount.cu", "voxcount.cuh", "voxitems.cuh", "dev_path.cuh", "kernels.h"),
    "voxel_kernel": ("voxcount.cu", "voxcount.cuh", "voxitems.cuh", "dev_path.cuh", "kernels.h"),
    "node_kernel": ("voxcount.cu", "voxcount.cuh", "voxitems.cuh", "dev_path.cuh", "kernels.h"),
    "count_kernel": ("kernels.cu", "kernels.h", "dev_path.cuh"),
    "render_kernel": ("kernels.cu", "kernels.h", "dev_path.cuh"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2609_40297_gb300", "csrc", f)) as fh:
            txt = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [ln.split("//", 1)[0].rstrip() for ln in txt.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def profiled(kernel, workload):
    """Figures of a committed ncu summary (profiles/<kernel>_<workload>.md) taken on the current
    kernel source (the summary records the source hash), else None: DRAM bytes per launch over a
    whole evaluation (a one-pass capture), and from a full capture of one launch its issue
    activity, threads per instruction, L2 hit rate, L2-to-SM read rate (GB/s) and the bytes used
    per 32-byte sector of its global loads."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    mh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not mh or mh.group(1) != kernel_source_hash(kernel):
        return None
    out = {}
    for key in ("dram_bytes_per_launch", "issue_active_pct", "threads_per_inst", "l2_hit_pct", "l2_to_sm_gbs",
                "global_load_bytes_per_sector"):
        m = re.search(rf"{key}:\s*([0-9.eE+]+)", txt)
        if m:
            out[key] = float(m.group(1))
    return out or None


# Algorithmic bytes per unit of work (the roofline's per-unit figures, applied to the units each
# kernel processes): a voxel step or a brick jump reads 1 B; a cast ray reads its 16 B ray-table
# entry and writes its 2 B step count; an enumerated voxel reads 1 B; a counted sample reads its
# owner pixel's 2 B step count and 16 B ray entry; an ancestor test that reaches the buffer reads
# a 4 B depth texel; a rendered pixel writes a 4 B texel.
def kernel_units(kernel, st):
    if kernel == "cast_kernel":
        return (st["cast_steps"] + st["cast_jumps"] + 18 * st["cast_rays"],
                "voxel steps + brick jumps (1 B each) + cast rays (16 B ray entry + 2 B step count)")
    if kernel in ("voxel_kernel", "node_kernel"):
        return (st["voxel_candidates"] + 18 * st["owned_samples"] + 4 * st["voxel_depth_reads"],
                "enumerated voxels (1 B) + counted samples (2 B step count + 16 B ray entry) + depth reads (4 B)")
    if kernel == "count_kernel":
        return (st["dda_steps"] + 4 * st["depth_reads"], "DDA steps (1 B) + depth reads (4 B)")
    return (st["render_steps"] + 4 * st["render_rays"], "render DDA steps (1 B) + texels written (4 B)")


def method_bytes(st):
    """The ray-by-ray method's own algorithmic bytes per evaluation (the roofline's per-unit
    figures on the method's units: 1 B per DDA step of every ray, 4 B per ancestor depth read,
    4 B per rendered texel), counted by the instrumented pass."""
    return st["dda_steps"] + 4 * st["depth_reads"] + 4 * st["render_rays"]


# ----------------------------------------------------------------------------- workloads
WORKLOAD_DESC = {
    "paper_scale": "paper-scale: 400x400x100 voxels @0.1 m (rooms, 5 prior scans), 500-node RRT depth<=10, "
                   "160x120 rays, 90x60 deg, 6 m, K=16 yaws",
    "tiny": "tiny: 64x64x32 @0.2 m, 20-node RRT depth<=4, 36x24 rays, 4 m, K=8",
    "large": "large: 800x800x200 @0.05 m (Perlin terrain + boxes, 5 prior scans), 2000-node RRT depth<=15, "
             "320x240 rays, 90x60 deg, 8 m, K=36 yaws",
}


def make_problem(workload, rank):
    import synth
    if workload == "paper_scale":
        return synth.paper_scale(seed=202 + 1000 * rank)
    if workload == "tiny":
        return synth.tiny(seed=101 + 1000 * rank)
    if workload == "large":
        return synth.large(seed=303 + 1000 * rank)
    raise ValueError(workload)


def init_dist(local):
    import torch
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    return torch.device("cuda", local)


# ----------------------------------------------------------------------------- one tree
COUNT_PASSES = {"auto": 0, "rays": 1, "pairs": 2, "nodes": 3}


def measure_single(workload, steps, warmup, with_modes=False, count_pass="auto", first_nodes=0):
    """Times `steps` whole-tree evaluations of one workload on the device-resident path (after
    `warmup`), then the host-array path end to end; returns the benchmark's fields. `count_pass`
    picks the counting kernels (auto: the library's choice; rays: ray by ray; pairs / nodes: the
    owned-voxel pass per (node, yaw) or per node). `first_nodes` > 0 keeps only the tree's first nodes
    (parents precede children, so they form a sub-tree): a smaller case of the same kernels."""
    import torch

    import paper_2609_40297_gb300 as mig
    import synth

    ws, rank, local = dist_env()
    dev = init_dist(local)
    prob = make_problem(workload, rank)
    desc = WORKLOAD_DESC[workload]
    if 0 < first_nodes < prob.tree.n:
        prob.tree = synth.Tree(prob.tree.parent[:first_nodes].copy(), prob.tree.pos[:first_nodes].copy())
        desc += f" (its first {first_nodes} nodes)"
    s = prob.sensor
    n = prob.tree.n
    max_depth = int(prob.tree.depth().max())
    rays_per_step = n * s.yaw_bins * s.width * s.height
    ctx = mig.Context(local)
    ctx.set_count_kernel(COUNT_PASSES[count_pass])
    stream = torch.cuda.current_stream(dev)
    m = mig.Map(ctx, prob.map.grid, prob.map.voxel_size, prob.map.origin)
    par = torch.from_numpy(prob.tree.parent).to(dev)
    pos = torch.from_numpy(prob.tree.pos).to(dev)
    outs = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(3)]
    flush = l2_flush_buffer(torch, dev)

    def step():
        mig.tree_eval_device(m, par, pos, s, max_depth, *outs)

    for _ in range(warmup):
        step()
    ctx.sync()
    # algorithmic work of one step (instrumented pass, untimed; it re-runs the ray-by-ray count
    # kernel beside the owned-voxel one for the method's own work counts and checks they agree)
    ref_out, stats = mig.tree_eval_stats(m, prob.tree.parent, prob.tree.pos, s)
    # ---- timed region: K steps, device time per step with CUDA events, L2 flushed between steps
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    ktimes = ctx.profile_read()
    ctx.profile(False)
    clocks = sampler.stop()
    ctx.sync()
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    got = [o.cpu().numpy() for o in outs]
    ok = all(np.array_equal(a, ref_out[k]) for a, k in zip(got, ("abs", "marg", "yaw")))
    value = ws * rays_per_step * steps / (total_ms / 1e3)
    # ---- end to end: host arrays through the public call (copies in the timed region)
    e2e_ms = []
    for i in range(max(3, min(steps, 5))):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mig.tree_eval(m, prob.tree.parent, prob.tree.pos, s)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = max_over_ranks(float(np.sum(e2e_ms)), dev)
    e2e_value = ws * rays_per_step * len(e2e_ms) / (e2e_total / 1e3)
    modes = with_modes and rank == 0 and run_modes(mig, torch, m, prob, rays_per_step) or None
    # ---- roofline of the dominant kernel: its algorithmic bytes per launch over its average launch
    # time, against the measured HBM copy bandwidth
    kms = {k: ktimes[f"{k}_ms"] for k in ("cast", "voxel", "count", "render")}
    dom = max(kms, key=kms.get)
    # the voxel kind times whichever voxel pass ran: per (node, yaw) pair or per node
    kernel = "node_kernel" if dom == "voxel" and stats.get("voxel_pass") == 3 else f"{dom}_kernel"
    launches = max(1, int(ktimes[f"{dom}_launches"]))
    lps = launches / steps
    avg_launch_s = kms[dom] / 1e3 / launches
    units, unit_desc = kernel_units(kernel, stats)
    alg_bytes_launch = units / lps
    achieved = alg_bytes_launch / avg_launch_s / 1e9
    peak, peak_kind = load_peaks()
    prof = profiled(kernel, workload)
    count_pass_ms = (kms["cast"] + kms["voxel"] + kms["count"]) / steps
    n_launches = int(ktimes["count_launches"] + ktimes["select_launches"] + ktimes["render_launches"] +
                     ktimes["plan_launches"] * 4 + ktimes["cast_launches"] + ktimes["voxel_launches"])
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    res = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws, "steps": steps, "warmup": warmup,
        "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE, "data": DATA,
        "config": {"workload": desc, "nodes": n, "yaw_bins": s.yaw_bins,
                   "rays_per_node_yaw": s.width * s.height, "max_depth": max_depth,
                   "inputs_sha256_16": synth.sha256(prob.map.grid, prob.tree.parent, prob.tree.pos)[:16],
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}",
                   "count_pass": count_pass},
        "replans_per_s": ws * steps / (total_ms / 1e3),
        "nodes_per_s": ws * n * steps / (total_ms / 1e3),
        "replan_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "results_match_host_path": bool(ok),
        "e2e": {"value": e2e_value, "unit": "rays/s", "h2d_bytes_per_step": int(n * 16),
                "d2h_bytes_per_step": int(n * 12), "ms_per_step": e2e_total / len(e2e_ms)},
        "gpu_launches": n_launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": prof["dram_bytes_per_launch"] if prof and "dram_bytes_per_launch" in prof else None,
                     "kernel": kernel, "algorithmic_bytes_per_launch": alg_bytes_launch,
                     "avg_launch_ms": avg_launch_s * 1e3, "launches_per_step": lps,
                     "units": unit_desc, "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "ncu": prof,
                     "note": "the kernel is bound by integer issue and L2-served gathers, not by HBM: its data "
                             "(map, step counts, depth buffers) stays L2-resident between its loads"},
        "method_work": {"bytes_per_step": method_bytes(stats),
                        "gb_per_s_over_count_pass": method_bytes(stats) / (count_pass_ms / 1e3) / 1e9,
                        "count_pass_ms": count_pass_ms,
                        "note": "the ray-by-ray method's algorithmic bytes (1 B per DDA step of every ray, 4 B per "
                                "ancestor depth read, 4 B per rendered texel) over the count pass's time: the work "
                                "rate the same results would need from a ray-by-ray walk (not a roofline: the "
                                "owned-voxel kernels do not execute that walk)"},
        "modes": modes,
        "work_per_step": stats,
        "kernel_ms_per_step": {k.replace("_ms", ""): v / steps for k, v in ktimes.items() if k.endswith("_ms")},
        "sm_count": sm_count,
        "clocks": clocks,
    }
    m.close()
    ctx.close()
    return res


def run_modes(mig, torch, m, prob, rays_per_step):
    """The gain modes side by side (Table 2's absolute vs marginal columns, the paper's screen-space
    interval overlap against voxel-centre samples, panoramic counting), each through the public
    host-array call: median of 3 after one warm-up (a mode slower than 2 s: that first call alone)."""
    s = prob.sensor
    modes, yaws = {}, {}
    for name, md in (("marginal_samples", mig.MODE_MARGINAL), ("marginal_intervals", mig.MODE_INTERVAL),
                     ("single_parent", mig.MODE_SINGLE_PARENT), ("absolute", mig.MODE_ABSOLUTE),
                     ("panoramic", mig.MODE_PANORAMIC)):
        if md == mig.MODE_PANORAMIC and s.pitch_deg != 0:
            continue
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = mig.tree_eval(m, prob.tree.parent, prob.tree.pos, s, mode=md)
        first_ms = (time.perf_counter() - t0) * 1e3
        ts = []
        for _ in range(3 if first_ms < 2000 else 0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = mig.tree_eval(m, prob.tree.parent, prob.tree.pos, s, mode=md)
            ts.append((time.perf_counter() - t0) * 1e3)
        ms = float(np.median(ts)) if ts else first_ms
        modes[name] = {"ms_per_replan": ms, "rays_per_s": rays_per_step / (ms / 1e3),
                       "marg_sum": int(g["marg"].sum()), "abs_sum": int(g["abs"].sum())}
        if md == mig.MODE_PANORAMIC:
            modes[name]["note"] = ("rays_per_s counts the pinhole rays the mode stands in for (nodes x K x W x H); "
                                   "it casts nodes x A x H with A azimuth columns")
        yaws[name] = g["yaw"]
    for name in modes:  # how often each mode picks the same viewpoint as voxel-centre samples
        modes[name]["same_yaw_as_samples"] = float(np.mean(yaws[name] == yaws["marginal_samples"]))
    return modes


# ----------------------------------------------------------------------------- batched (config 4)
def golden_batched_check(probs, outs):
    """True/False against the stored oracle results of the 64-tree workload when present and the
    inputs match; None otherwise."""
    import synth
    path = os.path.join(ROOT, "tests", "golden", "batched_oracle.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    off = g["offsets"]
    if len(off) - 1 != len(probs):
        return None
    for i, p in enumerate(probs):
        if synth.sha256(p.map.grid, p.tree.parent, p.tree.pos) != str(g["inputs_sha256"][i]):
            return None
    return all(np.array_equal(o[k], g[k][off[i]:off[i + 1]]) for i, o in enumerate(outs) for k in ("abs", "marg", "yaw"))


def batched_compare(repeats=3, small=False):
    """64 trees on 64 maps: one batched call per step (graph replay) against the same trees evaluated
    by 64 sequential plain calls; both end to end through the host-array calls (plans up, results
    down inside the timed region), alternating, `repeats` times each."""
    import torch

    import paper_2609_40297_gb300 as mig
    import synth

    ws, rank, local = dist_env()
    init_dist(local)
    if small:
        probs = synth.batched_small(seed_base=606 + 1000 * rank)
    else:
        probs = synth.batched(seed_base=404 + 1000 * rank, n_trees=int(os.environ.get("MIG_BATCH_TREES", "64")))
    n_trees = len(probs)
    stream = torch.cuda.Stream(local)
    ctx = mig.Context(local, stream=stream)
    dev_maps = {}  # one device map per distinct map (small trees share their map)
    for p in probs:
        if id(p.map) not in dev_maps:
            dev_maps[id(p.map)] = mig.Map(ctx, p.map.grid, p.map.voxel_size, p.map.origin)
    maps = [dev_maps[id(p.map)] for p in probs]
    trees = [(p.tree.parent, p.tree.pos, p.sensor) for p in probs]
    rays = sum(p.tree.n * p.sensor.yaw_bins * p.sensor.width * p.sensor.height for p in probs)
    nodes = sum(p.tree.n for p in probs)

    def batched_step():
        return mig.tree_eval_batch(ctx, trees, maps)

    def plain_step():
        return [mig.tree_eval(m, *t) for m, t in zip(maps, trees)]

    ref = batched_step()
    plain = plain_step()
    same = all(np.array_equal(a[k], b[k]) for a, b in zip(ref, plain) for k in ("abs", "marg", "yaw"))
    golden = None if small else golden_batched_check(probs, ref)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    # both batch engines; the faster one is the batched figure (the tile autotuner's choice)
    engine_ms = {}
    tw, th, cps, eng0 = ctx.get_tiles()
    for eng in (0, 1):
        ctx.set_tiles(tw, th, cps, eng)
        batched_step()
        t0 = time.perf_counter()
        batched_step()
        engine_ms[eng] = (time.perf_counter() - t0) * 1e3
    best_engine = min(engine_ms, key=engine_ms.get)
    ctx.set_tiles(tw, th, cps, best_engine)
    batched_step()
    tb, tp = [], []
    for _ in range(repeats):
        t0 = time.perf_counter()
        batched_step()
        tb.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        plain_step()
        tp.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    caps, reps = ctx.graph_stats()
    for mm in dev_maps.values():
        mm.close()
    ctx.close()
    tbm, tpm = float(np.median(tb)), float(np.median(tp))
    desc = ((f"batched small trees: {n_trees} trees, 16 per map on {len(dev_maps)} rooms maps 400x400x100 @0.1 m, "
             "trees U[20,60] nodes, depth U[2,5], 64x48 rays, K=16, 6 m (short-horizon replans; not one of the "
             "paper's configurations)") if small else
            (f"batched: {n_trees} trees on {n_trees} rooms maps 400x400x100 @0.1 m, trees U[50,2000] nodes, "
             "depth U[3,15], ray grids 64x48..320x240, K=16, 6 m"))
    return {
        "workload": desc, "trees": n_trees, "nodes": nodes, "rays_per_step": rays,
        "repeats": repeats,
        "batched": {"ms": spread([x * 1e3 for x in tb]), "replans_per_s": n_trees / tbm, "rays_per_s": rays / tbm,
                    "engine": ["persistent_dataflow", "stream_chains"][best_engine]},
        "plain": {"ms": spread([x * 1e3 for x in tp]), "replans_per_s": n_trees / tpm, "rays_per_s": rays / tpm,
                  "launches": f"{n_trees} sequential mig_tree_eval calls"},
        "batched_vs_plain_speedup": tpm / tbm,
        "speedup_range": [min(tp) / max(tb), max(tp) / min(tb)],
        "results_identical_to_plain": bool(same),
        "results_identical_to_oracle": golden,
        "engine_ms": {"persistent_dataflow": engine_ms[0], "stream_chains": engine_ms[1]},
        "graph": {"captures": caps, "replays": reps},
        "e2e": {"h2d_bytes_per_step": int(sum(p.tree.n * 16 for p in probs)), "d2h_bytes_per_step": int(nodes * 12)},
        "l2": f"inputs ({len(dev_maps)} maps, {len(dev_maps) * 16} MB) larger than L2",
        "clocks": clocks,
    }


# ----------------------------------------------------------------------------- serving (config 5)
def serving_compare(window_s, rate_hz, inflight=4):
    """16 robots on 4 rooms maps, Poisson arrivals (rate_hz each) for window_s seconds, a 10 % map
    update before each request, trees of U[100,1500] nodes. Served arm: the continuous-batching
    server, arrivals replayed in real time, latency = arrival -> results on the host. Plain arm:
    the same requests in arrival order through lone mig_tree_eval calls, as a FIFO single-server
    queue on the measured service times."""
    import torch

    import paper_2609_40297_gb300 as mig
    import synth

    ws, rank, local = dist_env()
    init_dist(local)
    maps_spec, pools, events, sensor, updates = synth.serving_requests(seed=505 + 1000 * rank, duration_s=window_s,
                                                                       rate_hz=rate_hz, update_seed=77 + rank)
    ctx = mig.Context(local, stream=torch.cuda.Stream(local))

    def fresh_maps():
        return [mig.Map(ctx, mm.grid, mm.voxel_size, mm.origin) for mm in maps_spec]

    wm = fresh_maps()
    t0_tree = pools[0][1][0]
    for _ in range(3):
        mig.tree_eval(wm[0], t0_tree.parent, t0_tree.pos, sensor)
    for mm in wm:
        mm.close()
    # ---- served arm: real-time replay
    maps = fresh_maps()
    srv = mig.Server(ctx, arena_budget_bytes=8 << 30, max_inflight=inflight)
    tickets = [None] * len(events)
    start = time.perf_counter()

    def submitter():
        for i, (t_arr, rid, mi, ti) in enumerate(events):
            delay = start + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            (x0, y0, z0, dx, dy, dz), vox = updates[i]
            srv.map_update(maps[mi], x0, y0, z0, vox)
            tr = pools[rid][1][ti]
            tickets[i] = srv.submit(maps[mi], tr.parent, tr.pos, sensor)

    sampler = ClockSampler(local)
    sampler.start()
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat, done_at = [], []
    for i, (t, _) in enumerate(tickets):
        while not srv.poll(t, timeout_us=10_000_000):
            pass
        tm = srv.timing(t)
        lat.append(tm["done_us"] / 1e3)
        done_at.append(events[i][0] + tm["done_us"] / 1e6)  # relative to the first arrival's clock
    t_end = time.perf_counter()
    clocks = sampler.stop()
    served_results = [out for _, out in tickets]
    srv.close()
    for mm in maps:
        mm.close()
    served_span = t_end - start
    # ---- plain arm: the same requests one by one (FIFO queue on measured service times)
    maps = fresh_maps()
    finish, lat_plain, service = 0.0, [], []
    same = True
    for i, (t_arr, rid, mi, ti) in enumerate(events):
        (x0, y0, z0, dx, dy, dz), vox = updates[i]
        tr = pools[rid][1][ti]
        t0 = time.perf_counter()
        maps[mi].update(x0, y0, z0, vox)
        out = mig.tree_eval(maps[mi], tr.parent, tr.pos, sensor)
        sv = time.perf_counter() - t0
        service.append(sv)
        finish = max(finish, t_arr) + sv
        lat_plain.append((finish - t_arr) * 1e3)
        same &= all(np.array_equal(out[k], served_results[i][k]) for k in ("abs", "marg", "yaw"))
    for mm in maps:
        mm.close()
    ctx.close()
    n = len(events)
    plain_span = finish
    rays = sum(pools[rid][1][ti].n for (_, rid, _, ti) in events) * sensor.yaw_bins * sensor.width * sensor.height
    backlog = int(sum(1 for d in done_at if d > window_s))
    return {
        "workload": (f"serving: 16 robots on 4 rooms maps 400x400x100 @0.1 m, Poisson {rate_hz:g} Hz each for "
                     f"{window_s:g} s of arrivals ({n} requests), trees U[100,1500] nodes, 160x120 rays, K=16, "
                     "10% map update before each request"),
        "requests": n, "max_inflight": inflight,
        "offered_replans_per_s": n / window_s,
        "served": {"replans_per_s": n / served_span, "rays_per_s": rays / served_span, "span_s": served_span,
                   "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}},
        "plain": {"replans_per_s": n / plain_span, "rays_per_s": rays / plain_span, "span_s": plain_span,
                  "latency_ms": {"p50": float(np.percentile(lat_plain, 50)),
                                 "p99": float(np.percentile(lat_plain, 99))},
                  "mean_service_ms": float(np.mean(service)) * 1e3},
        "served_vs_plain_replans": plain_span / served_span,
        "queue": {"backlog_at_window_end": backlog,
                  "growth_per_s": max(0.0, n / window_s - n / served_span),
                  "note": "requests not yet completed when the last arrival came, and the offered minus the served "
                          "rate: positive when the offered load exceeds the GPU's capacity"},
        "results_identical_alone_vs_mix": bool(same),
        "e2e": {"h2d_bytes_per_step": int(np.mean([pools[r][1][t].n * 16 for (_, r, _, t) in events])),
                "d2h_bytes_per_step": int(np.mean([pools[r][1][t].n * 12 for (_, r, _, t) in events]))},
        "clocks": clocks,
    }


# ----------------------------------------------------------------------------- CPU oracle
def cpu_model():
    """The host CPU as /proc/cpuinfo names it: the model name, or on Arm the implementer and part
    codes (0x41 / 0xd4f is an Arm Neoverse V2, the Grace core), plus the machine type."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" in line:
                    k, v = (x.strip() for x in line.split(":", 1))
                    fields.setdefault(k, v)
    except OSError:
        pass
    name = fields.get("model name") or " ".join(
        f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part") if k in fields)
    return f"{platform.machine()}: {name or 'unknown'}"


def cpu_baseline(workload, sample_depth=None, with_gap=False, with_mode_gaps=False, n_threads=0):
    """The oracle as it stands, on this host's cores (n_threads = 0: all of them), on a bounded,
    ancestor-closed sample of the workload (all nodes up to a depth), reported in the benchmark's
    unit."""
    import oracle
    prob = make_problem(workload, 0)
    s = prob.sensor
    d = prob.tree.depth()
    if sample_depth is None:
        sample_depth = {"tiny": 10, "paper_scale": 10, "large": 2}.get(workload, 3)
    mask = (d <= sample_depth).astype(np.uint8)
    m = int(mask.sum())
    t0 = time.perf_counter()
    db = oracle.eval_tree(prob.map.grid, prob.map.voxel_size, prob.map.origin, prob.tree.parent, prob.tree.pos, s,
                          node_mask=mask, n_threads=n_threads)
    dt = time.perf_counter() - t0
    rays = m * s.yaw_bins * s.width * s.height
    full_rays = prob.tree.n * s.yaw_bins * s.width * s.height
    out = {"value": rays / dt, "unit": "rays/s", "cores": n_threads or os.cpu_count(), "cpu": cpu_model(),
           "kind": "oracle",
           "sample": f"{m} of {prob.tree.n} nodes (all nodes of depth <= {sample_depth}), all {s.yaw_bins} yaws, "
                     f"{s.width}x{s.height} rays; {dt:.1f} s",
           "seconds": dt, "full_tree_seconds_extrapolated": full_rays / (rays / dt)}
    if with_gap:
        # gap of the depth-buffer marginal gain to the exact one (Eq. 2 with the same yaws, Sec. V-A),
        # both from the oracle on the same sample (the CUDA path is bit-identical to the oracle's DB part)
        off, ids = oracle.visible_sets(prob.map.grid, prob.map.voxel_size, prob.map.origin, prob.tree.pos, db["yaw"],
                                       s, node_mask=mask)
        ex = oracle.exact_dfs(prob.tree.parent, off, ids, prob.map.grid.size, node_mask=mask)
        sel = mask.astype(bool)
        rep = oracle.gap_report(d[sel], db["marg"][sel], ex[sel], abs_gain=db["abs"][sel])
        rep["nodes"] = m
        out["gap_to_exact"] = rep
        if with_mode_gaps:
            # the same report for the paper's interval overlap (Eq. 5-7) and for panoramic counting,
            # each with its own yaws (exact sets are the pinhole visible sets at those yaws)
            for key, md in (("gap_to_exact_intervals", oracle.MODE_INTERVAL),
                            ("gap_to_exact_panoramic", oracle.MODE_PANORAMIC)):
                if md == oracle.MODE_PANORAMIC and s.pitch_deg != 0:
                    continue
                iv = oracle.eval_tree(prob.map.grid, prob.map.voxel_size, prob.map.origin, prob.tree.parent,
                                      prob.tree.pos, s, node_mask=mask, mode=md)
                off, ids = oracle.visible_sets(prob.map.grid, prob.map.voxel_size, prob.map.origin, prob.tree.pos,
                                               iv["yaw"], s, node_mask=mask)
                exi = oracle.exact_dfs(prob.tree.parent, off, ids, prob.map.grid.size, node_mask=mask)
                repi = oracle.gap_report(d[sel], iv["marg"][sel], exi[sel], abs_gain=iv["abs"][sel])
                repi["nodes"] = m
                repi["same_yaw_as_samples"] = float(np.mean(iv["yaw"][sel] == db["yaw"][sel]))
                out[key] = repi
            # the exact-yaw variant (each node's yaw chosen by its exact Eq. 2 gain, given its
            # ancestors' exact choices), on the nodes of depth <= 4: how often the depth-buffer
            # method picks the same viewpoint, and the exact gain of both choices of yaws
            m4 = (d <= min(4, sample_depth)).astype(np.uint8)
            s4 = m4.astype(bool)
            ey, eE = oracle.exact_yaw(prob.map.grid, prob.map.voxel_size, prob.map.origin, prob.tree.parent,
                                      prob.tree.pos, s, node_mask=m4)
            off, ids = oracle.visible_sets(prob.map.grid, prob.map.voxel_size, prob.map.origin, prob.tree.pos,
                                           db["yaw"], s, node_mask=m4)
            edb = oracle.exact_dfs(prob.tree.parent, off, ids, prob.map.grid.size, node_mask=m4)
            out["exact_yaw"] = {"nodes": int(s4.sum()), "same_yaw_as_depth_buffer": float(np.mean(ey[s4] == db["yaw"][s4])),
                                "exact_gain_with_depth_buffer_yaws": int(edb[s4].sum()),
                                "exact_gain_with_exact_yaws": int(eE[s4].sum()),
                                "ratio": float(edb[s4].sum() / max(1, eE[s4].sum()))}
    return out


def add_cpu_baseline(res, workload, with_modes):
    cb = cpu_baseline(workload, with_gap=True, with_mode_gaps=with_modes)
    res["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "cpu", "kind", "sample",
                                              "full_tree_seconds_extrapolated")}
    for key in ("gap_to_exact", "gap_to_exact_intervals", "gap_to_exact_panoramic", "exact_yaw"):
        if cb.get(key):
            res[key] = cb[key]
    # the same oracle on one core, on a smaller sample (a few seconds)
    c1 = cpu_baseline(workload, sample_depth={"tiny": 10, "paper_scale": 3, "large": 0}[workload], n_threads=1)
    res["cpu_baseline_single_thread"] = {k: c1[k] for k in ("value", "unit", "cores", "cpu", "kind", "sample")}


# ----------------------------------------------------------------------------- reference arm
REFERENCE_SAMPLE_DEPTH = {"large": 1, "paper_scale": 3, "tiny": 10}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    workload = args.workload if args.workload in REFERENCE_SAMPLE_DEPTH else "large"
    cb = None
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(workload, sample_depth=REFERENCE_SAMPLE_DEPTH[workload])
        if i >= args.warmup:
            vals.append(r["value"])
        cb = r
    value = float(np.mean(vals))
    cb = dict(cb)
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cb["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64 fixed point (u8 map)", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[workload], "sample": cb["sample"]},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "cpu", "kind", "sample")},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- main
def summary(r):
    keys = ("value", "unit", "ms_per_step", "replans_per_s", "nodes_per_s", "replan_latency_ms", "e2e",
            "results_match_host_path", "kernel_ms_per_step", "roofline", "method_work", "config")
    return {k: r[k] for k in keys if k in r}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "large", "paper_scale", "tiny", "batched", "batched_small", "serving"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the per-mode comparison (interval, absolute)")
    ap.add_argument("--no-extras", action="store_true", help="headline: skip the batched and serving parts")
    ap.add_argument("--serve-rate-hz", type=float, default=20.0, help="serving: Poisson request rate per robot")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="serving: arrival window (the workload specifies 30 s; at 20 Hz per robot the queue "
                         "grows by ~280 requests per second, so the default run replays the first 3 s)")
    ap.add_argument("--batch-repeats", type=int, default=3)
    ap.add_argument("--count-pass", default="auto", choices=sorted(COUNT_PASSES),
                    help="single-tree workloads: the counting kernels (default: the library's choice)")
    ap.add_argument("--first-nodes", type=int, default=0,
                    help="single-tree workloads: evaluate only the tree's first N nodes (a smaller case)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, _ = dist_env()
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res))
        return
    res = None
    if args.workload in ("batched", "batched_small"):
        b = batched_compare(repeats=max(args.batch_repeats, args.steps), small=args.workload == "batched_small")
        if rank == 0:
            tb = b["batched"]["ms"]["median"] / 1e3
            res = {"metric": METRIC, "value": ws * b["rays_per_step"] / tb, "unit": "rays/s", "n_gpus": ws,
                   "steps": b["repeats"], "warmup": args.warmup, "ms_per_step": tb * 1e3, "higher_is_better": True,
                   "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": DATA,
                   "config": {"workload": b["workload"], "parallelism": f"replicas x{ws}"},
                   "e2e": {"value": ws * b["rays_per_step"] / tb, "unit": "rays/s", **b["e2e"]},
                   "gpu_launches": None, "batched": b, "clocks": b["clocks"]}
    elif args.workload == "serving":
        sv = serving_compare(args.serve_seconds, args.serve_rate_hz)
        if rank == 0:
            res = {"metric": METRIC, "value": ws * sv["served"]["replans_per_s"], "unit": "replans/s", "n_gpus": ws,
                   "steps": sv["requests"], "warmup": args.warmup, "ms_per_step": 1e3 / sv["served"]["replans_per_s"],
                   "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE,
                   "data": "synthetic (seeded Poisson trace; stands in for robots replanning online)",
                   "config": {"workload": sv["workload"], "parallelism": f"replicas x{ws}"},
                   "e2e": {"value": ws * sv["served"]["replans_per_s"], "unit": "replans/s", **sv["e2e"]},
                   "gpu_launches": None, "serving": sv, "clocks": sv["clocks"]}
    else:
        workload = "large" if args.workload == "headline" else args.workload
        res = measure_single(workload, args.steps, args.warmup,
                             with_modes=not args.no_modes and args.workload != "headline", count_pass=args.count_pass,
                             first_nodes=args.first_nodes)
        if args.workload == "headline" and ws == 1 and not args.no_extras:
            res["paper_scale"] = summary(measure_single("paper_scale", args.steps, args.warmup))
            res["batched"] = batched_compare(repeats=args.batch_repeats)
            res["serving"] = {
                "as_specified": serving_compare(args.serve_seconds, args.serve_rate_hz),
                "feasible_load": serving_compare(10.0, 2.0),
            }
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            add_cpu_baseline(res, workload, with_modes=not args.no_modes and args.workload != "headline")
    if ws > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
