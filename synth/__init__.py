"""Seeded synthetic inputs for the marginal-gain path (maps, RRT trees, sensors, traces).

This module is the ONLY code shared by the CUDA path's tests/benchmarks and the CPU
oracle. It holds none of the method's arithmetic: no fixed-point DDA, no projection,
no counting. Maps are made with a plain float ray-march of its own (a stand-in for
a mapping pipeline), trees with a plain RRT (a stand-in for the planner that
builds the complete tree before gain evaluation, Sec. IV-D).

The paper's own worlds (Gazebo school / maze / multi-story, Table 1) and its
real-world data are not available; the recipes below stand in for them with the
same structure: tri-state voxel maps (free / occupied / unknown, Sec. III-A),
an explored region around the robot, and RRTs with bounded edge length, depth
and branching (Table 1 step sizes).

Voxel codes: 0 = unknown, 1 = free, 2 = occupied. Grids are numpy uint8 arrays of
shape (nz, ny, nx) (x fastest in memory). Positions are float32 metres in the world
frame (z up); the grid origin is the world position of voxel (0,0,0)'s low corner.

Determinism: numpy's PCG64 generator is platform independent; float work here
(trig in the scan directions, Perlin noise) may differ in the last bit between an
x86 and an Arm host, so a map is reproducible per platform. Parity never depends
on that: the CUDA path and the oracle always consume the same in-process arrays.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass, field

import numpy as np

UNKNOWN, FREE, OCCUPIED = 0, 1, 2


@dataclass
class Sensor:
    hfov_deg: float = 90.0
    vfov_deg: float = 60.0
    width: int = 36
    height: int = 24
    range_m: float = 4.0
    yaw_bins: int = 8
    pitch_deg: float = 0.0


@dataclass
class MapSpec:
    grid: np.ndarray                 # uint8 (nz, ny, nx)
    voxel_size: float
    origin: tuple = (0.0, 0.0, 0.0)
    truth: np.ndarray | None = None  # optional ground-truth occupancy (bool), for map updates

    @property
    def dims(self):
        nz, ny, nx = self.grid.shape
        return nx, ny, nz


@dataclass
class Tree:
    parent: np.ndarray   # int32 [n], -1 = root
    pos: np.ndarray      # float32 [n, 3] metres

    @property
    def n(self):
        return int(self.parent.shape[0])

    def depth(self) -> np.ndarray:
        d = np.zeros(self.n, np.int32)
        for i in range(self.n):  # parents precede children in generated trees
            p = self.parent[i]
            d[i] = 0 if p < 0 else d[p] + 1
        return d


@dataclass
class Problem:
    name: str
    map: MapSpec
    tree: Tree
    sensor: Sensor
    meta: dict = field(default_factory=dict)


def sha256(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


# ----------------------------------------------------------------------------------
# ground-truth worlds
# ----------------------------------------------------------------------------------

def _boxes_until(rng, shape, frac, emin, emax, occ=None):
    nz, ny, nx = shape
    occ = np.zeros(shape, bool) if occ is None else occ
    total = occ.size
    count = int(occ.sum())
    while count < frac * total:
        ex, ey, ez = (int(v) for v in rng.integers(emin, emax + 1, size=3))
        ex, ey, ez = min(ex, nx), min(ey, ny), min(ez, nz)
        x0 = int(rng.integers(0, nx - ex + 1))
        y0 = int(rng.integers(0, ny - ey + 1))
        z0 = int(rng.integers(0, nz - ez + 1))
        sl = occ[z0:z0 + ez, y0:y0 + ey, x0:x0 + ex]
        count += int(sl.size - sl.sum())
        sl[...] = True
    return occ


def world_rooms(rng, nx=400, ny=400, nz=100, wall=2, slab=2, target=0.10):
    """Room-and-pillar ground truth: floor/ceiling slabs, a jittered wall grid with
    door gaps, and pillars; pillars are added until `target` of the voxels are occupied."""
    occ = np.zeros((nz, ny, nx), bool)
    occ[:slab] = True
    occ[nz - slab:] = True
    door_h = min(nz - slab - 1, 24)

    def cuts(n):
        xs, x = [], int(rng.integers(30, 60))
        while x < n - 20:
            xs.append(x)
            x += int(rng.integers(55, 95))
        return xs

    xcuts, ycuts = cuts(nx), cuts(ny)
    # walls normal to x (planes x = c), split into segments between y cuts, each with a door
    ybounds = [0] + ycuts + [ny]
    for c in xcuts:
        occ[:, :, c:c + wall] = True
        for a, b in zip(ybounds[:-1], ybounds[1:]):
            if b - a > 20:
                w = min(int(rng.integers(10, 17)), b - a - 6)  # leaves room for the door's offset
                s = int(rng.integers(a + 3, b - w - 2))
                occ[slab:slab + door_h, s:s + w, c:c + wall] = False
    xbounds = [0] + xcuts + [nx]
    for c in ycuts:
        occ[:, c:c + wall, :] = True
        for a, b in zip(xbounds[:-1], xbounds[1:]):
            if b - a > 20:
                w = min(int(rng.integers(10, 17)), b - a - 6)  # leaves room for the door's offset
                s = int(rng.integers(a + 3, b - w - 2))
                occ[slab:slab + door_h, c:c + wall, s:s + w] = False
    # pillars (full height) and low furniture boxes until the target fraction
    total = occ.size
    count = int(occ.sum())
    while count < target * total:
        if rng.random() < 0.5:
            px, py = (int(v) for v in rng.integers(0, [nx - 4, ny - 4]))
            sl = occ[:, py:py + 4, px:px + 4]
        else:
            ex, ey, ez = (int(v) for v in rng.integers([6, 6, 4], [30, 30, 15]))
            px = int(rng.integers(0, nx - ex))
            py = int(rng.integers(0, ny - ey))
            sl = occ[slab:slab + ez, py:py + ey, px:px + ex]
        count += int(sl.size - np.count_nonzero(sl))
        sl[...] = True
    return occ


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def perlin_improved(x, y, z, perm):
    """Ken Perlin's 'improved noise' (SIGGRAPH 2002): 12 gradient directions chosen by
    a permutation hash, quintic fade, trilinear blend. Vectorised over numpy arrays."""
    X = np.floor(x).astype(np.int64) & 255
    Y = np.floor(y).astype(np.int64) & 255
    Z = np.floor(z).astype(np.int64) & 255
    x = x - np.floor(x)
    y = y - np.floor(y)
    z = z - np.floor(z)
    u, v, w = _fade(x), _fade(y), _fade(z)
    p = np.concatenate([perm, perm])

    def grad(h, x, y, z):
        h = h & 15
        a = np.where(h < 8, x, y)
        b = np.where(h < 4, y, np.where((h == 12) | (h == 14), x, z))
        return np.where(h & 1 == 0, a, -a) + np.where(h & 2 == 0, b, -b)

    A = p[X] + Y
    AA, AB = p[A] + Z, p[A + 1] + Z
    B = p[X + 1] + Y
    BA, BB = p[B] + Z, p[B + 1] + Z

    def lerp(t, a, b):
        return a + t * (b - a)

    return lerp(w,
                lerp(v, lerp(u, grad(p[AA], x, y, z), grad(p[BA], x - 1, y, z)),
                     lerp(u, grad(p[AB], x, y - 1, z), grad(p[BB], x - 1, y - 1, z))),
                lerp(v, lerp(u, grad(p[AA + 1], x, y, z - 1), grad(p[BA + 1], x - 1, y, z - 1)),
                     lerp(u, grad(p[AB + 1], x, y - 1, z - 1), grad(p[BB + 1], x - 1, y - 1, z - 1))))


def world_terrain(rng, nx=800, ny=800, nz=200, target=0.12):
    """Perlin heightfield terrain plus boxes; the terrain height scale is bisected (on a 4x column
    subsample) so that about `target` of all voxels are occupied."""
    perm = rng.permutation(256).astype(np.int64)
    gy, gx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    h = np.zeros((ny, nx))
    amp, freq = 1.0, 1.0 / 160.0
    for _ in range(4):
        h += amp * perlin_improved(gx * freq, gy * freq, np.full_like(gx, 0.5), perm)
        amp *= 0.5
        freq *= 2.0
    h = (h - h.min()) / (h.max() - h.min() + 1e-12)  # [0,1]
    boxes = _boxes_until(rng, (nz, ny, nx), 0.025, 8, 60)
    zc = np.arange(nz, dtype=np.float64)[:, None, None]
    hs, bs = h[::4, ::4], boxes[:, ::4, ::4]
    lo, hi = 0.0, float(nz)
    mid = 0.5 * (lo + hi)
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        f = ((zc < (mid * 0.5 + hs * mid)[None]) | bs).mean()
        if abs(f - target) < 0.002:
            break
        if f < target:
            lo = mid
        else:
            hi = mid
    return (zc < (mid * 0.5 + h * mid)[None]) | boxes


# ----------------------------------------------------------------------------------
# prior exploration: which voxels a robot has already seen (float ray march)
# ----------------------------------------------------------------------------------

def explore(truth, voxel_size, origin, viewpoints, range_m, az_step_deg=0.5, el_deg=(-30.0, 30.0),
            el_step_deg=0.5):
    """Map = unknown everywhere except what 360deg x 60deg scans from `viewpoints` saw in
    `truth`: marched samples before the first occupied sample become free, that sample's
    voxel becomes occupied. A plain float march at 1/2 voxel spacing (a mapping stand-in)."""
    nz, ny, nx = truth.shape
    grid = np.zeros(truth.shape, np.uint8)
    az = np.deg2rad(np.arange(0.0, 360.0, az_step_deg))
    el = np.deg2rad(np.arange(el_deg[0], el_deg[1] + 1e-9, el_step_deg))
    A, E = np.meshgrid(az, el, indexing="ij")
    dirs = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    step = 0.5 * voxel_size
    n_steps = int(math.ceil(range_m / step))
    org = np.asarray(origin, np.float64)
    flat_truth = truth.reshape(-1)
    flat_grid = grid.reshape(-1)
    for vp in viewpoints:
        p0 = (np.asarray(vp, np.float64) - org) / voxel_size      # voxel units
        dv = dirs * (step / voxel_size)
        alive = np.arange(dirs.shape[0])
        for s in range(n_steps):
            pts = p0[None, :] + s * dv[alive]
            idx = np.floor(pts).astype(np.int64)
            inside = ((idx[:, 0] >= 0) & (idx[:, 0] < nx) & (idx[:, 1] >= 0) & (idx[:, 1] < ny)
                      & (idx[:, 2] >= 0) & (idx[:, 2] < nz))
            alive, idx = alive[inside], idx[inside]
            if alive.size == 0:
                break
            lin = (idx[:, 2] * ny + idx[:, 1]) * nx + idx[:, 0]
            hit = flat_truth[lin]
            flat_grid[lin[~hit]] = FREE
            flat_grid[lin[hit]] = OCCUPIED
            alive = alive[~hit]
    return grid


# ----------------------------------------------------------------------------------
# planning trees
# ----------------------------------------------------------------------------------

def _segment_free(grid, voxel_size, origin, a, b):
    nz, ny, nx = grid.shape
    L = float(np.linalg.norm(b - a))
    m = max(2, int(math.ceil(L / (0.25 * voxel_size))) + 1)
    t = np.linspace(0.0, 1.0, m)[:, None]
    pts = a[None] + t * (b - a)[None]
    idx = np.floor((pts - np.asarray(origin)) / voxel_size).astype(np.int64)
    if np.any(idx < 0) or np.any(idx[:, 0] >= nx) or np.any(idx[:, 1] >= ny) or np.any(idx[:, 2] >= nz):
        return False
    return not np.any(grid[idx[:, 2], idx[:, 1], idx[:, 0]] == OCCUPIED)


def local_box(m: MapSpec, root, half_xy, dz_lo, dz_hi):
    """Sampling box around the robot, clipped to the grid less one voxel."""
    nz, ny, nx = m.grid.shape
    v = m.voxel_size
    org = np.asarray(m.origin, np.float64)
    glo = org + v
    ghi = org + np.array([nx, ny, nz]) * v - v
    r = np.asarray(root, np.float64)
    lo = np.maximum(glo, r - np.array([half_xy, half_xy, dz_lo]))
    hi = np.minimum(ghi, r + np.array([half_xy, half_xy, dz_hi]))
    return lo, hi


def rrt(rng, m: MapSpec, root, n_nodes, max_depth, step_m, max_children=None, box=None,
        max_tries=None):
    """Plain RRT: uniform samples in `box` (default: the grid box less one voxel),
    nearest node that may still take a child (depth < max_depth, children < cap),
    steer by at most `step_m`, accept if the segment crosses no occupied map voxel.
    Nodes are stored in insertion order, so parent[i] < i."""
    nz, ny, nx = m.grid.shape
    v = m.voxel_size
    org = np.asarray(m.origin, np.float64)
    if box is None:
        lo = org + v
        hi = org + np.array([nx, ny, nz]) * v - v
    else:
        lo, hi = (np.asarray(x, np.float64) for x in box)
    pos = np.zeros((n_nodes, 3), np.float64)
    parent = np.full(n_nodes, -1, np.int32)
    depth = np.zeros(n_nodes, np.int32)
    kids = np.zeros(n_nodes, np.int32)
    pos[0] = root
    n = 1
    tries = 0
    max_tries = max_tries or 400 * n_nodes
    while n < n_nodes:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"rrt: only {n}/{n_nodes} nodes after {tries} samples")
        s = lo + rng.random(3) * (hi - lo)
        ok = depth[:n] < max_depth
        if max_children is not None:
            ok &= kids[:n] < max_children
        if not ok.any():
            raise RuntimeError("rrt: no node can take a child")
        d2 = np.sum((pos[:n] - s) ** 2, axis=1)
        d2[~ok] = np.inf
        j = int(np.argmin(d2))
        dist = math.sqrt(float(d2[j]))
        if dist < 1e-6:
            continue
        q = pos[j] + (s - pos[j]) * min(1.0, step_m / dist)
        vi = np.floor((q - org) / v).astype(np.int64)
        if np.any(vi < 0) or vi[0] >= nx or vi[1] >= ny or vi[2] >= nz:
            continue
        if m.grid[vi[2], vi[1], vi[0]] == OCCUPIED:
            continue
        if not _segment_free(m.grid, v, org, pos[j], q):
            continue
        pos[n] = q
        parent[n] = j
        depth[n] = depth[j] + 1
        kids[j] += 1
        n += 1
    return Tree(parent=parent, pos=pos.astype(np.float32))


def _free_spot(rng, truth, voxel_size, origin, lo_vox, hi_vox, z_vox, clearance=4):
    nz, ny, nx = truth.shape
    for _ in range(10000):
        x = int(rng.integers(lo_vox[0], hi_vox[0]))
        y = int(rng.integers(lo_vox[1], hi_vox[1]))
        z = int(z_vox)
        c = clearance
        if x - c < 0 or y - c < 0 or x + c >= nx or y + c >= ny:
            continue
        if not truth[z - 1:z + 2, y - c:y + c + 1, x - c:x + c + 1].any():
            return np.asarray(origin) + (np.array([x, y, z]) + 0.5) * voxel_size
    raise RuntimeError("no free spot")


# ----------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------

SENSOR_TINY = Sensor(90.0, 60.0, 36, 24, 4.0, 8, 0.0)
SENSOR_PAPER = Sensor(90.0, 60.0, 160, 120, 6.0, 16, 0.0)
SENSOR_LARGE = Sensor(90.0, 60.0, 320, 240, 8.0, 36, 0.0)


def tiny(seed=101, n_nodes=20, max_depth=4) -> Problem:
    """64x64x32 grid at 0.2 m: random occupied boxes (edges 1-8 voxels) until >=15 %
    occupied, a known-free sphere of 3 m around the grid centre, the rest unknown.
    20-node RRT rooted at the grid centre, edges <= 1.5 m, depth <= 4."""
    rng = np.random.default_rng(seed)
    nx, ny, nz, v = 64, 64, 32, 0.2
    occ = _boxes_until(rng, (nz, ny, nx), 0.15, 1, 8)
    grid = np.zeros((nz, ny, nx), np.uint8)
    grid[occ] = OCCUPIED
    c = np.array([nx, ny, nz]) / 2.0
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    r2 = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2
    grid[r2 <= (3.0 / v) ** 2] = FREE
    m = MapSpec(grid, v, (0.0, 0.0, 0.0), truth=occ)
    root = c * v
    tree = rrt(rng, m, root, n_nodes, max_depth, 1.5)
    return Problem("tiny", m, tree, SENSOR_TINY, {"seed": seed})


def rooms_map(seed, nx=400, ny=400, nz=100, v=0.1, n_views=5, scan_range=6.0, scan_step_deg=0.5):
    rng = np.random.default_rng(seed)
    truth = world_rooms(rng, nx, ny, nz)
    org = (0.0, 0.0, 0.0)
    zv = int(round(1.5 / v))
    vp0 = _free_spot(rng, truth, v, org, (nx // 2 - 40, ny // 2 - 40), (nx // 2 + 40, ny // 2 + 40), zv)
    vps = [vp0]
    c0 = np.floor((vp0 - np.asarray(org)) / v).astype(int)
    while len(vps) < n_views:
        vps.append(_free_spot(rng, truth, v, org, (c0[0] - 80, c0[1] - 80), (c0[0] + 80, c0[1] + 80), zv))
    grid = explore(truth, v, org, vps, scan_range, az_step_deg=scan_step_deg, el_step_deg=scan_step_deg)
    return MapSpec(grid, v, org, truth=truth), vps, rng


def paper_scale(seed=202, n_nodes=500, max_depth=10) -> Problem:
    """400x400x100 grid at 0.1 m: room-and-pillar world (~10 % occupied); the map is
    unknown except for what 5 seeded 360x60 deg scans (6 m) saw. 500-node RRT rooted at
    the latest scan pose, depth <= 10, 1-6 children, step 1.5 m (Table 1, large maze)."""
    m, vps, rng = rooms_map(seed)
    tree = rrt(rng, m, vps[0], n_nodes, max_depth, 1.5, max_children=6,
               box=local_box(m, vps[0], 8.0, 1.0, 1.5))
    return Problem("paper_scale", m, tree, SENSOR_PAPER, {"seed": seed, "viewpoints": [list(map(float, p)) for p in vps]})


def large(seed=303, n_nodes=2000, max_depth=15) -> Problem:
    """800x800x200 grid at 0.05 m: Perlin terrain plus boxes (12 % occupied), explored by
    5 seeded scans (8 m); 2000-node RRT, depth <= 15, step 2.0 m, 1-6 children."""
    rng = np.random.default_rng(seed)
    nx, ny, nz, v = 800, 800, 200, 0.05
    truth = world_terrain(rng, nx, ny, nz)
    org = (0.0, 0.0, 0.0)
    # viewpoints 1.5 m above the local terrain column top
    vps = []
    c = np.array([nx // 2, ny // 2])
    while len(vps) < 5:
        x, y = (int(t) for t in rng.integers(c - 120, c + 120))
        col = truth[:, y, x]
        top = int(np.nonzero(col)[0].max()) + 1 if col.any() else 0
        z = top + int(1.5 / v)
        if z >= nz - 5 or truth[min(nz - 1, z), y, x]:
            continue
        if truth[max(0, z - 2):z + 3, max(0, y - 3):y + 4, max(0, x - 3):x + 4].any():
            continue
        vps.append(np.asarray(org) + (np.array([x, y, z]) + 0.5) * v)
    grid = explore(truth, v, org, vps, 8.0, az_step_deg=0.5, el_step_deg=0.5)
    m = MapSpec(grid, v, org, truth=truth)
    tree = rrt(rng, m, vps[0], n_nodes, max_depth, 2.0, max_children=6,
               box=local_box(m, vps[0], 10.0, 1.5, 2.5))
    return Problem("large", m, tree, SENSOR_LARGE, {"seed": seed})


RAY_GRIDS = [(64, 48), (96, 72), (128, 96), (160, 120), (240, 180), (320, 240)]


def _batched_one(args):
    seed, n_range, depth_range = args
    m, vps, rng = rooms_map(seed, scan_step_deg=1.0)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    dmax = int(rng.integers(depth_range[0], depth_range[1] + 1))
    w, h = RAY_GRIDS[int(rng.integers(0, len(RAY_GRIDS)))]
    n = min(n, sum(6 ** d for d in range(dmax + 1)) // 2)  # at most half a full 6-ary tree of that depth
    tree = rrt(rng, m, vps[0], n, dmax, 1.5, max_children=6, box=local_box(m, vps[0], 8.0, 1.0, 1.5))
    s = Sensor(90.0, 60.0, w, h, 6.0, 16, 0.0)
    m.truth = None  # not needed downstream; keeps the pickled result small
    return Problem(f"batched_{seed}", m, tree, s, {"seed": seed})


def batched(seed_base=404, n_trees=64, n_range=(50, 2000), depth_range=(3, 15), workers=None):
    """64 independent problems on 64 seeded rooms maps (config-2 type, scans at 1 deg): tree sizes
    U[50,2000] (capped at half the nodes of a full 6-ary tree of the drawn depth), depth limits U[3,15], ray grids drawn from RAY_GRIDS, K=16, 6 m. Built in a pool
    of spawned worker processes when workers > 1."""
    jobs = [(seed_base + i, n_range, depth_range) for i in range(n_trees)]
    workers = workers if workers is not None else min(16, os.cpu_count() or 1)
    if workers <= 1 or n_trees <= 1:
        return [_batched_one(j) for j in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batched_one, jobs))


def _batched_small_one(args):
    seed, trees_per_map, n_range, depth_range, grid = args
    m, vps, rng = rooms_map(seed, scan_step_deg=1.0)
    m.truth = None
    out = []
    for t in range(trees_per_map):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        dmax = int(rng.integers(depth_range[0], depth_range[1] + 1))
        n = min(n, sum(6 ** d for d in range(dmax + 1)) // 2)
        start = vps[t % len(vps)]
        tree = rrt(rng, m, start, n, dmax, 1.5, max_children=6, box=local_box(m, start, 8.0, 1.0, 1.5))
        out.append(Problem(f"small_{seed}_{t}", m, tree, Sensor(90.0, 60.0, grid[0], grid[1], 6.0, 16, 0.0),
                           {"seed": seed, "tree": t}))
    return out


def batched_small(seed_base=606, n_maps=16, trees_per_map=16, n_range=(20, 60), depth_range=(2, 5), grid=(64, 48),
                  workers=None):
    """Many short-horizon replans: n_maps seeded rooms maps (config-2 type), trees_per_map small trees on
    each (U[20,60] nodes, depth limits U[2,5], 64x48 rays, K=16, 6 m), started from the map's scan
    poses. Trees on the same map share its MapSpec object."""
    jobs = [(seed_base + i, trees_per_map, n_range, depth_range, grid) for i in range(n_maps)]
    workers = workers if workers is not None else min(16, os.cpu_count() or 1)
    if workers <= 1 or n_maps <= 1:
        groups = [_batched_small_one(j) for j in jobs]
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            groups = list(ex.map(_batched_small_one, jobs))
    return [p for g in groups for p in g]


def map_update_box(rng, m: MapSpec, frac=0.10):
    """One axis-aligned box holding `frac` of the grid's voxels, re-labelled from the
    ground truth (occupied stays occupied, the rest becomes free): a mapping update."""
    nz, ny, nx = m.grid.shape
    vol = frac * nx * ny * nz
    ez = nz
    side = int(round(math.sqrt(vol / ez)))
    ex, ey = min(nx, side), min(ny, side)
    x0 = int(rng.integers(0, nx - ex + 1))
    y0 = int(rng.integers(0, ny - ey + 1))
    z0 = 0
    t = m.truth[z0:z0 + ez, y0:y0 + ey, x0:x0 + ex]
    vox = np.where(t, OCCUPIED, FREE).astype(np.uint8)
    return (x0, y0, z0, ex, ey, ez), np.ascontiguousarray(vox)


def serving_trace(seed=505, n_maps=4, robots_per_map=4, rate_hz=20.0, duration_s=30.0,
                  n_range=(100, 1500), trees_per_robot=4, update_frac=0.10):
    """Open-loop replanning trace: robots on shared rooms maps issue requests with
    Poisson arrivals; each request names a tree (uniform 100-1500 nodes, drawn from a
    small per-robot pool) and, before it, a map update of `update_frac` of the voxels."""
    rng = np.random.default_rng(seed)
    maps, pools = [], []
    for mi in range(n_maps):
        m, vps, mrng = rooms_map(seed + 1000 + mi)
        maps.append(m)
        for r in range(robots_per_map):
            pool = []
            for _ in range(trees_per_robot):
                n = int(mrng.integers(n_range[0], n_range[1] + 1))
                root = vps[r % len(vps)]
                pool.append(rrt(mrng, m, root, n, 10, 1.5, max_children=6,
                                box=local_box(m, root, 8.0, 1.0, 1.5)))
            pools.append((mi, pool))
    events = []
    for rid, (mi, pool) in enumerate(pools):
        t = 0.0
        while True:
            t += float(rng.exponential(1.0 / rate_hz))
            if t >= duration_s:
                break
            events.append((t, rid, mi, int(rng.integers(0, len(pool)))))
    events.sort()
    return maps, pools, events, SENSOR_PAPER


def serving_requests(seed=505, duration_s=30.0, rate_hz=20.0, update_seed=77, n_first=None):
    """The serving workload as a request sequence: serving_trace's maps, tree pools and Poisson
    events, plus the map update that precedes each request (a box of 10 % of the voxels,
    re-labelled from ground truth, drawn with its own seeded generator). n_first keeps the first
    requests only. Returns (maps, pools, events, sensor, updates); updates[i] =
    ((x0, y0, z0, dx, dy, dz), voxels[dz, dy, dx]) for events[i] = (t, robot, map, tree)."""
    maps, pools, events, sensor = serving_trace(seed=seed, duration_s=duration_s, rate_hz=rate_hz)
    if n_first is not None:
        events = events[:n_first]
    rng = np.random.default_rng(update_seed)
    updates = [map_update_box(rng, maps[mi], 0.10) for (_, _, mi, _) in events]
    return maps, pools, events, sensor, updates


def apply_update(grid, update):
    """The grid (nz, ny, nx) after one map update ((x0, y0, z0, dx, dy, dz), voxels), as a copy."""
    (x0, y0, z0, dx, dy, dz), vox = update
    g = grid.copy()
    g[z0:z0 + dz, y0:y0 + dy, x0:x0 + dx] = vox
    return g


def tiny_tree(positions, parents):
    return Tree(parent=np.asarray(parents, np.int32), pos=np.asarray(positions, np.float32))


def open_box_map(nx, ny, nz, v=0.2, fill=UNKNOWN):
    return MapSpec(np.full((nz, ny, nx), fill, np.uint8), v, (0.0, 0.0, 0.0))


def random_small(seed, nx=24, ny=20, nz=12, v=0.25, p_occ=0.08, p_free=0.4, n_nodes=12, max_depth=5,
                 sensor=None):
    """Small random tri-state map and tree for pin and parity tests (several tiles and a ragged tail)."""
    rng = np.random.default_rng(seed)
    u = rng.random((nz, ny, nx))
    grid = np.where(u < p_occ, OCCUPIED, np.where(u < p_occ + p_free, FREE, UNKNOWN)).astype(np.uint8)
    m = MapSpec(grid, v, (0.0, 0.0, 0.0))
    c = np.array([nx, ny, nz]) * v / 2.0
    gc = np.floor(c / v).astype(int)
    grid[gc[2] - 1:gc[2] + 2, gc[1] - 1:gc[1] + 2, gc[0] - 1:gc[0] + 2] = FREE  # room to grow the tree
    tree = rrt(rng, m, c + rng.uniform(-0.3 * v, 0.3 * v, 3), n_nodes, max_depth, 3 * v)
    s = sensor or Sensor(80.0, 55.0, 19, 13, 2.5, 6, 0.0)
    return Problem(f"random_small_{seed}", m, tree, s, {"seed": seed})


CONFIGS = {1: tiny, 2: paper_scale, 3: large}
