"""Benchmark: marginal-gain throughput of the GB300 path on the seeded synthetic workloads.

Default (N=1): the paper-scale workload, 400x400x100 voxels at 0.1 m, a 500-node RRT of depth
<= 10, 160x120 rays, K = 16 yaws, 6 m range. One step = one whole-tree evaluation (every node,
yaw and ray: count, ancestor test, yaw argmax, depth render).
  value = marginal-gain rays per second = nodes * K * W * H / device time, inputs resident in HBM,
          timed with CUDA events on the library's stream, L2 flushed between steps;
  e2e   = the same metric through the public host-array call (mig_tree_eval), host<->device
          copies inside the timed region.
Multi-GPU (torchrun, one rank per GPU): replicas only. Every rank evaluates its own seeded tree
per step, no collective on the data path; value = all ranks' rays / max-over-ranks time.

--impl reference: the CPU oracle (the plain C restatement of the method) timed on this host's
cores on a bounded sample of the same workload, same metric and unit.
--workload batched | serving | large | tiny: the other configurations (64 trees batched against 64
plain calls; the serving loop with p50/p99 latency; the 800x800x200 large workload; the tiny one).
The single-tree workloads also time every gain mode through the public call (`modes`) and, from the
oracle, report each mode's gap to the exact marginal gain.
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


def kernel_source_hash():
    """Hash of the count kernel's code (its source files with comments and blank lines removed), so
    that an ncu summary stays tied to the code it measured, not to its comments."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.h", "dev_path.cuh"):
        with open(os.path.join(ROOT, "paper_2609_40297_gb300", "csrc", f)) as fh:
            txt = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [ln.split("//", 1)[0].rstrip() for ln in txt.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernel
    source (the summary records the source hash); else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    mh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    mt = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mt or mh.group(1) != kernel_source_hash():
        return None
    return float(mt.group(1))


# Algorithmic integer operations per unit of work, from the fixed-point specification:
#  - a DDA step: 6 cross products, 3 comparisons, axis choice (2), step budget check and decrement (2),
#    face distance, voxel index and address updates (3), voxel load and code test (2) = 18;
#  - an owner test: offsets (3), Z and U and V (3 x 5), pixel-slab products (4) and comparisons (4) = 26;
#  - an ancestor projection: offsets (3), Z, U, V (15), image bounds (4), pixel floors (4), depth read
#    and comparison (2), float estimate (2) = 30.
OPS_PER_STEP, OPS_PER_OWNER_TEST, OPS_PER_ANCESTOR_TEST = 18, 26, 30


def issue_peak_ops(sm_clock_mhz=None):
    """Integer issue ceiling of a GB300: 152 SMs x 4 schedulers x 32 lanes per clock, at the SM clock
    seen under load (else the 2070 MHz maximum)."""
    mhz = sm_clock_mhz or 2070.0
    return 152 * 4 * 32 * mhz * 1e6


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


# ----------------------------------------------------------------------------- workloads
def make_problem(workload, rank):
    import synth
    if workload == "paper_scale":
        return synth.paper_scale(seed=202 + 1000 * rank)
    if workload == "tiny":
        return synth.tiny(seed=101 + 1000 * rank)
    if workload == "large":
        return synth.large(seed=303 + 1000 * rank)
    raise ValueError(workload)


WORKLOAD_DESC = {
    "paper_scale": "paper-scale: 400x400x100 voxels @0.1 m (rooms, 5 prior scans), 500-node RRT depth<=10, "
                   "160x120 rays, 90x60 deg, 6 m, K=16 yaws",
    "tiny": "tiny: 64x64x32 @0.2 m, 20-node RRT depth<=4, 36x24 rays, 4 m, K=8",
    "large": "large: 800x800x200 @0.05 m (Perlin terrain), 2000-node RRT depth<=15, 320x240 rays, 8 m, K=36",
}


def oracle_sample_mask(tree, max_depth_sample):
    d = tree.depth()
    return (d <= max_depth_sample).astype(np.uint8)


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    import paper_2609_40297_gb300 as mig
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = make_problem(args.workload, rank)
    s = prob.sensor
    n = prob.tree.n
    max_depth = int(prob.tree.depth().max())
    rays_per_step = n * s.yaw_bins * s.width * s.height
    ctx = mig.Context(local)
    stream = torch.cuda.current_stream(dev)
    m = mig.Map(ctx, prob.map.grid, prob.map.voxel_size, prob.map.origin)
    par = torch.from_numpy(prob.tree.parent).to(dev)
    pos = torch.from_numpy(prob.tree.pos).to(dev)
    outs = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(3)]
    flush = l2_flush_buffer(torch, dev)

    def step():
        mig.tree_eval_device(m, par, pos, s, max_depth, *outs)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    # algorithmic work of one step (instrumented pass, untimed)
    ref_out, stats = mig.tree_eval_stats(m, prob.tree.parent, prob.tree.pos, s)
    # ---- timed region: K steps, device time per step with CUDA events, L2 flushed between steps
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    ktimes = ctx.profile_read()
    ctx.profile(False)
    clocks = sampler.stop()
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    got = [o.cpu().numpy() for o in outs]
    ok = all(np.array_equal(a, ref_out[k]) for a, k in zip(got, ("abs", "marg", "yaw")))
    value = ws * rays_per_step * args.steps / (total_ms / 1e3)
    # ---- end to end: host arrays through the public call (copies in the timed region)
    e2e_ms = []
    for i in range(max(3, min(args.steps, 10))):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mig.tree_eval(m, prob.tree.parent, prob.tree.pos, s)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = max_over_ranks(float(np.sum(e2e_ms)), dev)
    e2e_value = ws * rays_per_step * len(e2e_ms) / (e2e_total / 1e3)
    # ---- the gain modes side by side (Table 2's absolute vs marginal columns, and the paper's
    # screen-space interval overlap against voxel-centre samples), each through the public host-array
    # call, outside the timed region: median of 3 after one warm-up (a mode slower than 2 s per call:
    # that first call alone)
    modes, yaws = {}, {}
    if rank == 0 and not args.no_modes:
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
            for _ in range(3 if first_ms < 2000 else 0):  # slow modes: the first call alone
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
    # ---- roofline of the dominant kernel (count pass). It is bound by integer issue: achieved =
    # algorithmic integer operations per launch / average launch time, against the issue ceiling.
    # The gather roofline (algorithmic voxel + depth bytes against HBM) is reported beside it.
    count_launches = max(1, int(ktimes["count_launches"]))
    launches_per_step = count_launches / args.steps
    avg_launch_s = ktimes["count_ms"] / 1e3 / count_launches
    alg_ops_launch = (stats["dda_steps"] * OPS_PER_STEP + stats["unknown_visits"] * OPS_PER_OWNER_TEST +
                      stats["ancestor_tests"] * OPS_PER_ANCESTOR_TEST) / launches_per_step
    alg_bytes_launch = (stats["dda_steps"] * 1 + stats["depth_reads"] * 4) / launches_per_step
    achieved_ops = alg_ops_launch / avg_launch_s / 1e9
    peak_ops = issue_peak_ops((clocks or {}).get("sm_mhz")) / 1e9
    achieved = alg_bytes_launch / avg_launch_s / 1e9
    peak, peak_kind = load_peaks()
    # the random-gather ceiling for the count pass's scattered loads, measured here by a probe:
    # 1-byte loads from a map-sized buffer (L2-resident) and 4-byte loads from an arena-sized one
    grid_bytes = int(prob.map.grid.size)
    gp_voxel = mig.probe_gather(ctx, grid_bytes, 1)
    gp_texel = mig.probe_gather(ctx, max(4096, int(prob.tree.n) * s.width * s.height * 4), 4)
    gathers_launch = (stats["dda_steps"] + stats["depth_reads"]) / launches_per_step
    gather_rate = gathers_launch / avg_launch_s
    gather_peak = (stats["dda_steps"] + stats["depth_reads"]) / (stats["dda_steps"] / gp_voxel + stats["depth_reads"] / gp_texel)
    traffic = profiled_traffic("count_kernel", args.workload)
    n_launches = int(ktimes["count_launches"] + ktimes["select_launches"] + ktimes["render_launches"] +
                     ktimes["plan_launches"] * 4)
    res = None
    if rank == 0:
        res = {
            "metric": METRIC,
            "value": value,
            "unit": "rays/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int32/int64 fixed point (u8 map)",
            "data": "synthetic (seeded; stands in for the paper's Gazebo worlds)",
            "config": {"workload": WORKLOAD_DESC[args.workload], "nodes": n, "yaw_bins": s.yaw_bins,
                       "rays_per_node_yaw": s.width * s.height, "max_depth": max_depth,
                       "inputs_sha256_16": synth.sha256(prob.map.grid, prob.tree.parent, prob.tree.pos)[:16],
                       "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}"},
            "replans_per_s": ws * args.steps / (total_ms / 1e3),
            "nodes_per_s": ws * n * args.steps / (total_ms / 1e3),
            "replan_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "results_match_host_path": bool(ok),
            "e2e": {"value": e2e_value, "unit": "rays/s", "h2d_bytes_per_step": int(n * 16),
                    "d2h_bytes_per_step": int(n * 12), "ms_per_step": e2e_total / len(e2e_ms)},
            "gpu_launches": n_launches,
            "roofline": {"bound": "alu", "achieved": achieved_ops, "peak": peak_ops, "unit": "Gop/s",
                         "frac": achieved_ops / peak_ops, "traffic": traffic, "kernel": "count_kernel",
                         "algorithmic_ops_per_launch": alg_ops_launch, "avg_launch_ms": avg_launch_s * 1e3,
                         "peak_source": "issue ceiling: 152 SMs x 4 schedulers x 32 lanes x the SM clock sampled under load",
                         "note": f"ops/unit: DDA step {OPS_PER_STEP}, owner test {OPS_PER_OWNER_TEST}, "
                                 f"ancestor projection {OPS_PER_ANCESTOR_TEST}; traffic = ncu DRAM bytes of one "
                                 "launch (level 8) when the committed summary matches the kernel source"},
            "gather_roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                                "algorithmic_bytes_per_launch": alg_bytes_launch,
                                "note": "algorithmic bytes = DDA voxel gathers (1 B) + ancestor depth reads (4 B); "
                                        "ncu: L2 sector hit 99 %, 3.6 sectors per load request"},
            "gather_rate_roofline": {"bound": "l2_random_gather", "achieved": gather_rate / 1e9,
                                     "peak": gather_peak / 1e9, "unit": "Gloads/s", "frac": gather_rate / gather_peak,
                                     "peak_source": "measured by mig_probe_gather on this GPU (random 1-byte loads from a "
                                                    f"{grid_bytes >> 20} MiB map-sized buffer: {gp_voxel / 1e9:.0f} G/s; "
                                                    f"random 4-byte loads from an arena-sized buffer: {gp_texel / 1e9:.0f} G/s), "
                                                    "weighted by the launch's voxel and depth-texel loads",
                                     "gathers_per_launch": gathers_launch,
                                     "note": "the probe's loads are fully random (32 sectors per warp request); the "
                                             "kernel's neighbouring rays load neighbouring voxels (3.6 sectors per "
                                             "request and 69 % L1 hits, ncu level 8), so its L2 sector traffic is far "
                                             "below this ceiling (47.7 G sectors/s under ncu, ~15 %); integer issue "
                                             "(roofline) is the binding resource"},
            "modes": modes or None,
            "work_per_step": stats,
            "kernel_ms_per_step": {k.replace("_ms", ""): v / args.steps for k, v in ktimes.items() if k.endswith("_ms")},
            "clocks": clocks,
        }
    m.close()
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return res


# ----------------------------------------------------------------------------- batched (config 4)
def run_batched(args):
    """64 trees on 64 maps: one persistent launch per step (graph replay), against the same trees
    evaluated by 64 sequential plain launches. value = batched rays/s; both arms end to end
    through the host-array calls (plans up, results down inside the timed region)."""
    import torch

    import paper_2609_40297_gb300 as mig
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    small = args.workload == "batched_small"
    if small:
        probs = synth.batched_small(seed_base=606 + 1000 * rank)
        n_trees = len(probs)
    else:
        n_trees = int(os.environ.get("MIG_BATCH_TREES", "64"))
        probs = synth.batched(seed_base=404 + 1000 * rank, n_trees=n_trees)
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

    for _ in range(args.warmup):
        ref = batched_step()
    plain = plain_step()
    same = all(np.array_equal(a[k], b[k]) for a, b in zip(ref, plain) for k in ("abs", "marg", "yaw"))
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    # both batch engines; the faster one is the batched figure (the tile autotuner's choice)
    engine_ms = {}
    tw, th, cps, eng0 = ctx.get_tiles()
    for eng in (0, 1):
        ctx.set_tiles(tw, th, cps, eng)
        for _ in range(2):
            batched_step()
        t0 = time.perf_counter()
        batched_step()
        engine_ms[eng] = (time.perf_counter() - t0) * 1e3
    best_engine = min(engine_ms, key=engine_ms.get)
    ctx.set_tiles(tw, th, cps, best_engine)
    batched_step()
    tb = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        batched_step()
        tb.append(time.perf_counter() - t0)
    tp = []
    for _ in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        plain_step()
        tp.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    caps, reps = ctx.graph_stats()
    tbatch, tplain = max_over_ranks(float(np.sum(tb)), torch.device("cuda", local)), float(np.mean(tp))
    value = ws * rays * len(tb) / tbatch
    res = None
    if rank == 0:
        res = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": tbatch / len(tb) * 1e3, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "int32/int64 fixed point (u8 map)",
               "data": "synthetic (seeded; stands in for the paper's Gazebo worlds)",
               "config": {"workload": (f"batched small trees: {n_trees} trees, 16 per map on {len(dev_maps)} rooms maps "
                                       "400x400x100 @0.1 m, trees U[20,60] nodes, depth U[2,5], 64x48 rays, K=16, 6 m "
                                       "(short-horizon replans; not one of the paper's configurations)") if small else
                                      (f"batched: {n_trees} trees on {n_trees} rooms maps 400x400x100 @0.1 m, "
                                       "trees U[50,2000] nodes, depth U[3,15], ray grids 64x48..320x240, K=16, 6 m"),
                          "nodes": nodes, "rays_per_step": rays,
                          "l2": f"inputs ({len(dev_maps)} maps, {len(dev_maps) * 16} MB) larger than L2",
                          "parallelism": f"replicas x{ws}"},
               "replans_per_s": ws * n_trees * len(tb) / tbatch,
               "plain": {"ms_per_step": tplain * 1e3, "rays_per_s": rays / tplain,
                         "replans_per_s": n_trees / tplain, "launches": f"{n_trees} sequential mig_tree_eval calls"},
               "batched_vs_plain_speedup": tplain / (tbatch / len(tb)),
               "results_identical_to_plain": bool(same),
               "graph": {"captures": caps, "replays": reps},
               "engine_ms": {"persistent_dataflow": engine_ms[0], "stream_chains": engine_ms[1]},
               "engine": ["persistent_dataflow", "stream_chains"][best_engine],
               "e2e": {"value": value, "unit": "rays/s",
                       "h2d_bytes_per_step": int(sum(p.tree.n * 16 for p in probs)),
                       "d2h_bytes_per_step": int(nodes * 12)},
               "gpu_launches": int(len(tb) * (sum(3 * (int(p.tree.depth().max()) + 1) - 1 for p in probs)
                                             if best_engine == 1 else 1)),
               "clocks": clocks}
    for m in dev_maps.values():
        m.close()
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return res


# ----------------------------------------------------------------------------- serving (config 5)
def run_serving(args):
    """16 robots on 4 rooms maps, Poisson arrivals (20 Hz each), a 10 % map update before each
    request, trees of U[100,1500] nodes. Served arm: the continuous-batching server, arrivals
    replayed in real time for a bounded window, latency = submit -> results on the host. Plain
    arm: the same requests in arrival order through lone mig_tree_eval calls, as a FIFO
    single-server queue on the measured service times."""
    import torch

    import paper_2609_40297_gb300 as mig
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    window = float(os.environ.get("MIG_SERVE_SECONDS", "2.0"))
    rate = float(args.serve_rate_hz)
    maps_spec, pools, events, sensor = synth.serving_trace(seed=505 + 1000 * rank, duration_s=window, rate_hz=rate)
    rng = np.random.default_rng(77 + rank)
    updates = [synth.map_update_box(rng, maps_spec[mi], 0.10) for (_, _, mi, _) in events]
    ctx = mig.Context(local, stream=torch.cuda.Stream(local))

    def fresh_maps():
        return [mig.Map(ctx, m.grid, m.voxel_size, m.origin) for m in maps_spec]

    # ---- warm-up (camera tables, kernels, allocator pools)
    wm = fresh_maps()
    t0_tree = pools[0][1][0]
    for _ in range(args.warmup):
        mig.tree_eval(wm[0], t0_tree.parent, t0_tree.pos, sensor)
    for m in wm:
        m.close()
    # ---- served arm: real-time replay
    maps = fresh_maps()
    inflight = int(os.environ.get("MIG_SERVE_INFLIGHT", "4"))
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
    lat = []
    for t, _ in tickets:
        while not srv.poll(t, timeout_us=10_000_000):
            pass
        lat.append(srv.timing(t)["done_us"] / 1e3)
    t_end = time.perf_counter()
    clocks = sampler.stop()
    served_results = [out for _, out in tickets]
    srv.close()
    for m in maps:
        m.close()
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
    for m in maps:
        m.close()
    ctx.close()
    n = len(events)
    plain_span = finish
    rays = sum(pools[rid][1][ti].n for (_, rid, _, ti) in events) * sensor.yaw_bins * sensor.width * sensor.height
    res = None
    if rank == 0:
        res = {"metric": METRIC, "value": ws * n / served_span, "unit": "replans/s", "n_gpus": ws,
               "steps": n, "warmup": args.warmup, "ms_per_step": served_span / n * 1e3, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "int32/int64 fixed point (u8 map)",
               "data": "synthetic (seeded Poisson trace; stands in for robots replanning online)",
               "config": {"workload": f"serving: 16 robots on 4 rooms maps 400x400x100 @0.1 m, Poisson {rate:g} Hz each "
                                      f"for {window:g} s of arrivals ({n} requests), trees U[100,1500] nodes, "
                                      "160x120 rays, K=16, 10% map update before each request",
                          "max_inflight": inflight, "parallelism": f"replicas x{ws}"},
               "served": {"replans_per_s": n / served_span, "rays_per_s": rays / served_span,
                          "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}},
               "plain": {"replans_per_s": n / plain_span, "rays_per_s": rays / plain_span,
                         "latency_ms": {"p50": float(np.percentile(lat_plain, 50)),
                                        "p99": float(np.percentile(lat_plain, 99))},
                         "mean_service_ms": float(np.mean(service)) * 1e3},
               "served_vs_plain_replans": (n / served_span) / (n / plain_span),
               "results_identical_alone_vs_mix": bool(same),
               "e2e": {"value": ws * n / served_span, "unit": "replans/s",
                       "h2d_bytes_per_step": int(np.mean([pools[r][1][t].n * 16 for (_, r, _, t) in events])),
                       "d2h_bytes_per_step": int(np.mean([pools[r][1][t].n * 12 for (_, r, _, t) in events]))},
               "gpu_launches": None, "clocks": clocks}
    return res


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
    out = {"value": rays / dt, "unit": "rays/s", "cores": n_threads or os.cpu_count(), "cpu": cpu_model(),
           "kind": "oracle",
           "sample": f"{m} of {prob.tree.n} nodes (all nodes of depth <= {sample_depth}), all {s.yaw_bins} yaws, "
                     f"{s.width}x{s.height} rays; {dt:.1f} s", "seconds": dt}
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


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    cb = None
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(args.workload)
        if i >= args.warmup:
            vals.append(r["value"])
        cb = r
    value = float(np.mean(vals))
    cb = dict(cb)
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cb["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64 fixed point (u8 map)", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload], "sample": cb["sample"]},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "cpu", "kind", "sample")},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_scale",
                    choices=["paper_scale", "tiny", "large", "batched", "batched_small", "serving"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the per-mode comparison (interval, absolute)")
    ap.add_argument("--serve-rate-hz", type=float, default=20.0,
                    help="serving workload: Poisson request rate per robot (20 Hz offers ~9x the GPU's capacity)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res))
        return
    if args.workload in ("batched", "batched_small"):
        res = run_batched(args)
    elif args.workload == "serving":
        res = run_serving(args)
    else:
        res = run_ours(args)
    ws, rank, _ = dist_env()
    if rank == 0 and res is not None:
        if ws == 1 and not args.no_cpu_baseline and args.workload in ("paper_scale", "tiny", "large"):
            cb = cpu_baseline(args.workload, with_gap=True, with_mode_gaps=not args.no_modes)
            res["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "cpu", "kind", "sample")}
            res["gap_to_exact"] = cb.get("gap_to_exact")
            for key in ("gap_to_exact_intervals", "gap_to_exact_panoramic", "exact_yaw"):
                if cb.get(key):
                    res[key] = cb[key]
            # the same oracle on one core, on a smaller sample (a few seconds)
            c1 = cpu_baseline(args.workload, sample_depth={"tiny": 10, "paper_scale": 3, "large": 0}[args.workload],
                              n_threads=1)
            res["cpu_baseline_single_thread"] = {k: c1[k] for k in ("value", "unit", "cores", "cpu", "kind", "sample")}
        print(json.dumps(res))


if __name__ == "__main__":
    main()
