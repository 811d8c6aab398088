"""Pins of the CPU oracle against things other than itself (CPU only, no GPU).

Each pin ties one step of the oracle to an independent fact:
  - DDA (Sec. IV-B, Amanatides-Woo): brute-force exact-rational slab intersection of the
    quantised ray with every voxel (Python fractions), on tie-free random rays, including
    the hit depth; hand-written sequences for the documented tie rule (x, then y, then z).
  - Camera and projection (Eq. 5): an independent float64 pinhole built from rotation
    matrices (numpy), for ray directions and for pixel indices of projected points.
  - Depth buffer (Sec. IV-A): closed-form z of a fronto-parallel wall, and of the range
    endpoint when nothing is hit.
  - Absolute gain (Eq. 1): voxel-centric brute force of the owner-visible set, and the
    closed-form frustum-ball volume Omega R^3 / 3 on an all-unknown map.
  - Marginal gain (Eq. 2): root marginal == absolute; marginal <= absolute per yaw;
    g_abs >= g_sp >= g_all with one fixed yaw; disjoint frusta give marginal == absolute;
    an identical pose gives exact marginal 0; an all-free map gives 0 everywhere.
  - Exact routes: hash-set merge == depth-first reference counts == sorted merge, and the
    telescoping identity: along every root-to-leaf path the exact gains sum to the size of
    the union of the visible sets.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from synth import Sensor

Q16 = 1 << 16
Q30 = 1 << 30


# ----------------------------------------------------------------------------- DDA
def brute_ray(grid, P, d, Tq):
    """Voxels whose interior the ray P + t d, 0 <= t < T crosses, by exact slab tests,
    in order of entry, cut after the first occupied one. Returns (list, hit_t or None),
    or None when the ray grazes an edge/corner (a tie) somewhere."""
    nz, ny, nx = grid.shape
    p = [Fr(int(P[a]), Q16) for a in range(3)]
    dd = [Fr(int(d[a]), Q30) for a in range(3)]
    T = Fr(int(Tq), Q16)
    dims = (nx, ny, nz)
    # tie check: all face-crossing times of different axes must differ
    times = {}
    for a in range(3):
        if dd[a] == 0:
            continue
        for b in range(0, dims[a] + 1):
            t = (b - p[a]) / dd[a]
            if 0 <= t < T:
                if t in times and times[t] != a:
                    return None
                times[t] = a
    hits = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                v = (x, y, z)
                lo, hi = Fr(-10 ** 9), Fr(10 ** 9)
                ok = True
                for a in range(3):
                    if dd[a] == 0:
                        if not (v[a] <= p[a] < v[a] + 1):
                            ok = False
                        continue
                    t0 = (v[a] - p[a]) / dd[a]
                    t1 = (v[a] + 1 - p[a]) / dd[a]
                    if t0 > t1:
                        t0, t1 = t1, t0
                    lo, hi = max(lo, t0), min(hi, t1)
                if not ok or not (lo < hi) or not (hi > 0):
                    continue
                entry = max(lo, Fr(0))
                if entry < T:
                    hits.append((entry, v))
    hits.sort()
    out = []
    hit_t = None
    for t, v in hits:
        out.append(v)
        if grid[v[2], v[1], v[0]] == 2:
            hit_t = t
            break
    return out, hit_t


def rand_dir(rng):
    while True:
        v = rng.normal(size=3)
        n = np.linalg.norm(v)
        if n > 1e-3:
            q = np.rint(v / n * Q30).astype(np.int64)
            if np.all(q != 0):
                return q


def test_dda_matches_exact_slab_brute_force(oracle_lib):
    rng = np.random.default_rng(7)
    nx, ny, nz = 9, 8, 7
    checked = 0
    for trial in range(160):
        u = rng.random((nz, ny, nx))
        grid = np.where(u < 0.06, 2, np.where(u < 0.5, 1, 0)).astype(np.uint8)
        P = np.array([rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)], np.int64) * Q16 \
            + rng.integers(1, Q16, size=3)
        d = rand_dir(rng)
        Tq = int(rng.integers(Q16, 14 * Q16))
        dzc = int(rng.integers(Q30 // 2, Q30))
        br = brute_ray(grid, P, d, Tq)
        if br is None:
            continue
        exp, hit_t = br
        vox, codes, hit, D = oracle_lib.trace(grid, P, d, Tq, dzc)
        assert [tuple(v) for v in vox.tolist()] == exp, f"trial {trial}"
        assert hit == (hit_t is not None)
        if hit:
            # depth of the entry point: floor(t * dzc * 2^16 / 2^30)
            assert D == math.floor(hit_t * dzc * Q16 / Q30)
        else:
            assert D == (Tq * dzc) // Q30
        checked += 1
    assert checked >= 140


def test_dda_tie_rule_x_then_y_then_z(oracle_lib):
    grid = np.ones((8, 8, 8), np.uint8)
    Tq = 20 * Q16  # directions below are not unit length: t advances 2-3 per voxel
    # 45 deg in the xy plane from a voxel centre: every crossing is an x/y tie
    P = np.array([Q16 // 2] * 3, np.int64)
    vox, _, hit, _ = oracle_lib.trace(grid, P, [Q30 // 2, Q30 // 2, 0], Tq, Q30)
    assert not hit
    assert [tuple(v) for v in vox.tolist()][:7] == [(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 1, 0), (2, 2, 0),
                                                      (3, 2, 0), (3, 3, 0)]
    # main diagonal: triple ties
    vox, _, _, _ = oracle_lib.trace(grid, P, [Q30 // 2, Q30 // 2, Q30 // 2], Tq, Q30)
    assert [tuple(v) for v in vox.tolist()][:7] == [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 1, 1),
                                                      (2, 2, 1), (2, 2, 2)]
    # start exactly on a corner going down in all axes: three zero-length steps at t = 0
    P = np.array([4 * Q16] * 3, np.int64)
    vox, _, _, _ = oracle_lib.trace(grid, P, [-(Q30 // 2), -(Q30 // 3), -(Q30 // 5)], Tq, Q30)
    assert [tuple(v) for v in vox.tolist()][:4] == [(4, 4, 4), (3, 4, 4), (3, 3, 4), (3, 3, 3)]


def test_dda_stops_at_range_and_grid(oracle_lib):
    grid = np.ones((4, 4, 30), np.uint8)
    P = np.array([Q16 // 2, 2 * Q16 + 5, 2 * Q16 + 7], np.int64)
    # along +x: voxel m is entered at t = m - 1/2; T = 10 visits m = 0..10
    vox, _, hit, _ = oracle_lib.trace(grid, P, [Q30, 0, 0], 10 * Q16, Q30)
    assert [v[0] for v in vox.tolist()] == list(range(11))
    # T exactly at a crossing: entry t = 9.5 is not < 9.5
    vox, _, _, _ = oracle_lib.trace(grid, P, [Q30, 0, 0], 9 * Q16 + Q16 // 2, Q30)
    assert [v[0] for v in vox.tolist()] == list(range(10))
    # leaving the grid ends the ray without a hit
    vox, _, hit, D = oracle_lib.trace(grid, P, [-Q30, 0, 0], 10 * Q16, Q30)
    assert [tuple(v) for v in vox.tolist()] == [(0, 2, 2)] and not hit and D == 10 * Q16


# ------------------------------------------------------------------- camera model
def float_camera(sensor, k):
    """Independent pinhole: rotation camera->world = Rz(psi) Ry(pitch) R_cb, with the camera
    x right, y down, z forward and the body x forward, y left, z up."""
    W, H, K = sensor.width, sensor.height, sensor.yaw_bins
    fx = (W / 2) / math.tan(math.radians(sensor.hfov_deg) / 2)
    fy = (H / 2) / math.tan(math.radians(sensor.vfov_deg) / 2)
    R_cb = np.array([[0, 0, 1], [-1, 0, 0], [0, -1, 0]], float)
    th = math.radians(sensor.pitch_deg)
    Ry = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    ps = 2 * math.pi * k / K
    Rz = np.array([[math.cos(ps), -math.sin(ps), 0], [math.sin(ps), math.cos(ps), 0], [0, 0, 1]])
    return Rz @ Ry @ R_cb, fx, fy, W / 2, H / 2


@pytest.mark.parametrize("sensor", [Sensor(90, 60, 36, 24, 4.0, 8, 0.0), Sensor(87, 58, 48, 28, 5.0, 12, 10.0),
                                    Sensor(70, 50, 17, 11, 3.0, 5, -20.0)])
def test_ray_directions_match_float_pinhole(oracle_lib, sensor):
    dirs = oracle_lib.ray_dirs(sensor).astype(np.float64) / Q30
    W, H = sensor.width, sensor.height
    j, i = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for k in range(sensor.yaw_bins):
        R, fx, fy, cx, cy = float_camera(sensor, k)
        cam = np.stack([(i + 0.5 - cx) / fx, (j + 0.5 - cy) / fy, np.ones_like(i, float)], -1)
        cam /= np.linalg.norm(cam, axis=-1, keepdims=True)
        world = cam @ R.T
        assert np.max(np.abs(dirs[k] - world)) < 4.0 / Q30
    # pixel (0,0) looks up and to the left of the optical axis
    assert dirs[0, 0, 0, 1] > 0 and dirs[0, 0, 0, 2] > 0 or sensor.pitch_deg > 0


@pytest.mark.parametrize("sensor", [Sensor(90, 60, 36, 24, 4.0, 8, 0.0), Sensor(87, 58, 48, 28, 5.0, 12, 10.0)])
def test_projection_matches_float_pinhole(oracle_lib, sensor):
    rng = np.random.default_rng(3)
    P = np.array([20 * Q16 + 12345, 20 * Q16 + 777, 10 * Q16 + 4242], np.int64)
    vox = rng.integers(0, 40, size=(4000, 3)).astype(np.int32)
    vox[:, 2] = rng.integers(0, 20, size=4000)
    n_cmp = 0
    for k in range(sensor.yaw_bins):
        out = oracle_lib.project(sensor, k, P, vox)
        R, fx, fy, cx, cy = float_camera(sensor, k)
        r = (vox + 0.5) - P / Q16
        c = r @ R  # world -> camera: R^T r
        front = c[:, 2] > 1e-6
        assert np.array_equal(out[:, 0].astype(bool), front)
        u = fx * c[front, 0] / c[front, 2] + cx
        v = fy * c[front, 1] / c[front, 2] + cy
        # compare where the pixel decision matters (within two image widths of it); far
        # outside, grazing points (z ~ 0) amplify the Q16 rounding of the projection rows
        near = (np.abs(u - cx) < 2 * sensor.width) & (np.abs(v - cy) < 2 * sensor.height)
        safe = near & (np.abs(u - np.round(u)) > 0.02) & (np.abs(v - np.round(v)) > 0.02)
        assert np.array_equal(out[front, 1][safe], np.floor(u[safe]).astype(np.int64))
        assert np.array_equal(out[front, 2][safe], np.floor(v[safe]).astype(np.int64))
        n_cmp += int(safe.sum())
    assert n_cmp > 1000


# --------------------------------------------------------------------- depth buffer
def single_node(pos_m):
    return np.array([-1], np.int32), np.asarray([pos_m], np.float32)


def test_depth_of_fronto_parallel_wall(oracle_lib):
    v = 0.25
    grid = np.ones((24, 40, 48), np.uint8)
    X0 = 31
    grid[:, :, X0] = 2
    P_vox = np.array([13.37, 20.41, 11.23])
    parent, pos = single_node(P_vox * v)
    s = Sensor(90, 60, 36, 24, 30 * v, 4, 0.0)
    r = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s, want_depth=True)
    assert r["yaw"][0] == 0 and r["abs"][0] == 0
    Pq = oracle_lib.quantize(pos, (0, 0, 0), v, (48, 40, 24))[0]
    expect = (X0 * Q16 - Pq[0])  # z-depth of a wall normal to the optical axis is constant
    D = r["depth"][0].astype(np.int64)
    assert np.all(np.abs(D - expect) <= 1), (D.min(), D.max(), expect)


def test_depth_of_range_endpoint(oracle_lib):
    v = 0.2
    grid = np.ones((30, 30, 30), np.uint8)
    parent, pos = single_node(np.array([15.5, 15.25, 15.125]) * v)
    s = Sensor(80, 50, 20, 14, 2.0, 3, 15.0)
    r = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s, want_depth=True)
    W, H = s.width, s.height
    j, i = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    fx = (W / 2) / math.tan(math.radians(s.hfov_deg) / 2)
    fy = (H / 2) / math.tan(math.radians(s.vfov_deg) / 2)
    cam = np.stack([(i + 0.5 - W / 2) / fx, (j + 0.5 - H / 2) / fy, np.ones((H, W))], -1)
    dzc = 1.0 / np.linalg.norm(cam, axis=-1)
    T = 2.0 / v
    expect = np.floor(T * dzc * Q16)
    assert np.all(np.abs(r["depth"][0].astype(np.float64) - expect) <= 1)


def test_ancestor_test_is_smaller_or_equal(oracle_lib):
    """Sec. IV-B: a sample is observed when its depth is smaller than OR EQUAL to the stored
    depth. At yaw 0, pitch 0 the camera z axis is world +x exactly, so the camera z of a
    voxel centre is known exactly: (x + 1/2) - P_x, in Q16 units (x+1/2)*2^16 - P_x."""
    s = Sensor(90, 60, 36, 24, 4.0, 1, 0.0)
    rng = np.random.default_rng(5)
    P = np.array([10 * Q16 + 9876, 12 * Q16 + 3210, 6 * Q16 + 4444], np.int64)
    R, fx, fy, cx, cy = float_camera(s, 0)
    n_checked = 0
    for _ in range(300):
        vox = np.array([rng.integers(11, 30), rng.integers(0, 25), rng.integers(0, 13)], np.int32)
        c = ((vox + 0.5) - P / Q16) @ R
        u, v = fx * c[0] / c[2] + cx, fy * c[1] / c[2] + cy
        if not (0.05 < u < s.width - 0.05 and 0.05 < v < s.height - 0.05):
            continue
        if min(abs(u - round(u)), abs(v - round(v))) < 0.02:
            continue
        zq = int((int(vox[0]) * Q16 + Q16 // 2) - P[0])
        D = np.full((s.height, s.width), 0, np.uint32)
        D[int(v), int(u)] = zq
        assert oracle_lib.observed(s, 0, P, D, vox)          # z == stored depth: observed
        D[int(v), int(u)] = zq - 1
        assert not oracle_lib.observed(s, 0, P, D, vox)      # z just behind: not observed
        D[int(v), int(u)] = 0xFFFFFFFF >> 6
        assert oracle_lib.observed(s, 0, P, D, vox)
        n_checked += 1
    assert n_checked > 100


# -------------------------------------------------------------------- absolute gain
def test_owner_set_equals_voxel_centric_brute_force(oracle_lib):
    rng = np.random.default_rng(11)
    nx, ny, nz, v = 20, 18, 10, 0.25
    u = rng.random((nz, ny, nx))
    grid = np.where(u < 0.05, 2, np.where(u < 0.3, 1, 0)).astype(np.uint8)
    s = Sensor(80, 55, 15, 11, 2.0, 4, 5.0)
    Pm = np.array([9.3, 8.6, 4.7]) * v
    grid[4, 8, 9] = 1
    parent, pos = single_node(Pm)
    r = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s, want_counts=True)
    Pq = oracle_lib.quantize(pos, (0, 0, 0), v, (nx, ny, nz))[0]
    dirs = oracle_lib.ray_dirs(s)
    Tq = oracle_lib.range_q16(s.range_m, v)
    unk = np.argwhere(grid == 0)[:, ::-1].astype(np.int32)  # (x,y,z)
    cache = {}
    for k in range(s.yaw_bins):
        proj = oracle_lib.project(s, k, Pq, unk)
        count = 0
        for (ok, pu, pv, _), vx in zip(proj, unk):
            if not ok or not (0 <= pu < s.width and 0 <= pv < s.height):
                continue
            key = (k, pu, pv)
            if key not in cache:
                vox, _, _, _ = oracle_lib.trace(grid, Pq, dirs[k, pv, pu], Tq, Q30)
                cache[key] = {tuple(t) for t in vox.tolist()}
            if tuple(vx.tolist()) in cache[key]:
                count += 1
        assert count == r["cnt_abs"][0, k], k
        assert r["cnt_marg"][0, k] == r["cnt_abs"][0, k]


def test_absolute_gain_frustum_volume_closed_form(oracle_lib):
    # all unknown, no occupied voxel: |I| ~ Omega R^3 / 3 with
    # Omega = 4 asin(sin(hfov/2) sin(vfov/2)) the solid angle of the rectangular frustum;
    # the buffer follows the resolution rule of Sec. IV-A (one pixel ~ one voxel at range).
    R = 20
    grid = np.zeros((48, 48, 48), np.uint8)
    v = 0.1
    s = Sensor(90, 60, 40, 24, R * v, 1, 0.0)
    parent, pos = single_node(np.array([24.31, 24.17, 24.43]) * v)
    r = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s)
    omega = 4 * math.asin(math.sin(math.radians(45)) * math.sin(math.radians(30)))
    vol = omega * R ** 3 / 3
    assert 0.85 * vol < r["abs"][0] < 1.1 * vol, (r["abs"][0], vol)


def test_all_free_map_gives_zero(oracle_lib):
    p = synth.random_small(5)
    grid = np.where(p.map.grid == 2, 2, 1).astype(np.uint8)
    r = oracle_lib.eval_tree(grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    assert not r["abs"].any() and not r["marg"].any() and not r["yaw"].any()


# -------------------------------------------------------------------- marginal gain
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_marginal_invariants(oracle_lib, seed):
    p = synth.random_small(seed)
    r = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                             want_counts=True)
    root = int(np.nonzero(p.tree.parent < 0)[0][0])
    assert r["marg"][root] == r["abs"][root]
    assert np.array_equal(r["cnt_marg"][root], r["cnt_abs"][root])
    assert np.all(r["cnt_marg"] <= r["cnt_abs"]) and np.all(r["cnt_marg"] >= 0)
    assert np.all(r["marg"] <= r["abs"])
    assert np.array_equal(r["abs"], r["cnt_abs"].max(axis=1))
    K = p.sensor.yaw_bins
    for n in range(p.tree.n):
        m = r["cnt_marg"][n]
        assert r["yaw"][n] == int(np.argmax(m)) and r["marg"][n] == m.max()
    assert np.all((r["yaw"] >= 0) & (r["yaw"] < K))


def test_result_independent_of_thread_count(oracle_lib):
    """The oracle parallelises over the nodes of a level and the yaws of a node; each (node, yaw)
    count is written by one thread, so one core and every core give the same result in every mode,
    and a one-thread call leaves later calls on every core."""
    p = synth.tiny()
    for mode in (oracle_lib.MODE_MARGINAL, oracle_lib.MODE_INTERVAL, oracle_lib.MODE_PANORAMIC):
        one = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                                   mode=mode, want_counts=True, want_depth=True, n_threads=1)
        every = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                                     mode=mode, want_counts=True, want_depth=True)
        assert one.keys() == every.keys()
        for k in one:
            assert np.array_equal(one[k], every[k]), (mode, k)


def test_fixed_yaw_ordering_abs_sp_all(oracle_lib):
    p = synth.random_small(4, n_nodes=14)
    s = Sensor(80, 55, 19, 13, 2.5, 1, 0.0)  # one yaw: every mode sees the same viewpoints
    args = (p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, s)
    a = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_ABSOLUTE)
    sp = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_SINGLE_PARENT)
    al = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_MARGINAL)
    assert np.array_equal(a["abs"], a["marg"])
    assert np.all(a["abs"] >= sp["marg"]) and np.all(sp["marg"] >= al["marg"])
    depth = p.tree.depth()
    assert np.array_equal(sp["marg"][depth == 1], al["marg"][depth == 1])
    assert np.any(sp["marg"] > al["marg"])


def test_disjoint_frusta_and_identical_pose(oracle_lib):
    rng = np.random.default_rng(2)
    nx, ny, nz, v = 40, 40, 16, 0.2
    u = rng.random((nz, ny, nx))
    grid = np.where(u < 0.03, 2, np.where(u < 0.2, 1, 0)).astype(np.uint8)
    grid[7:10, 19:22, 19:22] = 1
    c = np.array([20.3, 20.6, 8.2]) * v
    parent = np.array([-1, 0], np.int32)
    pos = np.stack([c, c]).astype(np.float32)
    # two yaws 180 deg apart and hfov < 180: the child's frustum at the other yaw is
    # behind the root camera, so nothing it sees is excluded
    s = Sensor(90, 60, 24, 16, 3.0, 2, 0.0)
    r = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s, want_counts=True)
    k_other = 1 - r["yaw"][0]
    assert r["cnt_marg"][1, k_other] == r["cnt_abs"][1, k_other] > 0
    # one yaw: identical viewpoints, the exact marginal gain of the child is 0
    s1 = Sensor(90, 60, 24, 16, 3.0, 1, 0.0)
    r1 = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s1)
    off, ids = oracle_lib.visible_sets(grid, v, (0, 0, 0), pos, r1["yaw"], s1)
    E = oracle_lib.exact_dfs(parent, off, ids, grid.size)
    assert E[1] == 0 and E[0] == r1["abs"][0]
    # the depth-buffer method keeps a residual at occlusion edges: a voxel clipped by its
    # owner ray just before an occupied voxel has its centre behind the stored depth
    # (the overestimate of Sec. V-A); speckle maps have many such edges
    assert r1["marg"][1] <= 0.15 * r1["abs"][1]


# -------------------------------------------------------------------- exact routes
@pytest.mark.parametrize("seed", [1, 2, 6])
def test_exact_routes_agree_and_telescope(oracle_lib, seed):
    p = synth.random_small(seed, n_nodes=16)
    r = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor,
                             want_counts=True)
    off, ids = oracle_lib.visible_sets(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.pos, r["yaw"], p.sensor)
    n = p.tree.n
    sizes = np.diff(off)
    assert np.array_equal(sizes, r["cnt_abs"][np.arange(n), r["yaw"]])  # abs == |I| (Sec. V-A)
    E1 = oracle_lib.exact_hash_merge(p.tree.parent, off, ids)
    E2 = oracle_lib.exact_dfs(p.tree.parent, off, ids, p.map.grid.size)
    E3 = oracle_lib.exact_sorted_merge(p.tree.parent, off, ids)
    assert np.array_equal(E1, E2) and np.array_equal(E1, E3)
    assert np.all(E1 <= sizes)
    # telescoping: sum of exact marginal gains on a root path == |union of its sets|
    parent = p.tree.parent
    is_leaf = np.ones(n, bool)
    is_leaf[parent[parent >= 0]] = False
    for leaf in np.nonzero(is_leaf)[0]:
        path, q = [], int(leaf)
        while q >= 0:
            path.append(q)
            q = int(parent[q])
        union = set()
        for q in path:
            union |= set(ids[off[q]:off[q + 1]].tolist())
        assert sum(int(E1[q]) for q in path) == len(union)


def test_tiny_config_gap_is_small_and_positive(oracle_lib):
    p = synth.tiny()
    r = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    off, ids = oracle_lib.visible_sets(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.pos, r["yaw"], p.sensor)
    E = oracle_lib.exact_dfs(p.tree.parent, off, ids, p.map.grid.size)
    rep = oracle_lib.gap_report(p.tree.depth(), r["marg"], E)
    # the depth-buffer method overestimates the exact marginal gain a little (Sec. V-A)
    assert 1.0 <= rep["sum_ratio"] < 1.15


def test_regression_tiny_depth_buffer_gain_not_below_exact(oracle_lib):
    """Regression check, not a pin: on this seed every node's depth-buffer marginal gain is at
    least its exact one. The method does not guarantee it (an ancestor's buffer can cover a
    voxel centre that its owner ray missed, which the exact sets do not count as observed); the
    check only flags a change of the tiny workload's result."""
    p = synth.tiny()
    r = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    off, ids = oracle_lib.visible_sets(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.pos, r["yaw"], p.sensor)
    E = oracle_lib.exact_dfs(p.tree.parent, off, ids, p.map.grid.size)
    assert np.all(r["marg"] >= E)


def test_invalid_inputs_rejected(oracle_lib):
    p = synth.random_small(1)
    g, v, o, par, pos, s = p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor
    bad = par.copy()
    bad[3] = 3
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.eval_tree(g, v, o, bad, pos, s)
    two_roots = par.copy()
    two_roots[2] = -1
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.eval_tree(g, v, o, two_roots, pos, s)
    outside = pos.copy()
    outside[1, 0] = -1.0
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.eval_tree(g, v, o, par, outside, s)
    g3 = g.copy()
    g3[0, 0, 0] = 7
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.eval_tree(g3, v, o, par, pos, s)


# ----------------------------------------------------------------------- path scoring
def test_score_closed_forms():
    """Eq. 3 and Eq. 4 on a straight chain with unit steps and equal gains: c(k) = k and
    o(k) = g v^3 sum_{j<=k} exp(-lambda j) (a geometric series); a branch picks the larger sum."""
    from oracle.score import score_tree
    n, v, lam = 6, 0.2, 0.5
    parent = np.arange(-1, n - 1)
    pos = np.stack([np.arange(n, dtype=float), np.zeros(n), np.zeros(n)], 1)
    gain = np.full(n, 1000)
    cost, obj, best = score_tree(parent, pos, gain, v, lam)
    assert np.allclose(cost, np.arange(n))
    g = 1000 * v ** 3
    expect = g * (1 - np.exp(-lam * np.arange(1, n + 1))) / (1 - np.exp(-lam))
    assert np.allclose(obj, expect, rtol=1e-12)
    assert best == n - 1
    # a root with two children: a 3-4-5 step with a large gain beats a unit step with a small one
    parent = np.array([-1, 0, 0])
    pos = np.array([[0, 0, 0], [3, 4, 0], [1, 0, 0]], float)
    cost, obj, best = score_tree(parent, pos, np.array([10, 500, 100]), 1.0, lam)
    assert np.allclose(cost, [0, 5, 1])
    assert np.isclose(obj[1], 10 + 500 * np.exp(-2.5)) and np.isclose(obj[2], 10 + 100 * np.exp(-0.5))
    assert best == 2  # 100 e^-0.5 = 60.7 > 500 e^-2.5 = 41.0
    # lambda = 0: the objective is the plain path sum of gains (a star: root + own gain)
    rng = np.random.default_rng(7)
    parent = np.array([-1, 0, 0, 1, 1, 3])
    pos = rng.normal(size=(6, 3))
    gain = np.array([5, 7, 11, 13, 17, 19])
    _, obj, best = score_tree(parent, pos, gain, 1.0, 0.0)
    assert np.allclose(obj, [5, 12, 16, 25, 29, 44]) and best == 5
    # equal objectives: the lowest index wins (two mirrored children of the root)
    parent = np.array([-1, 0, 0])
    pos = np.array([[0, 0, 0], [0, 1, 0], [0, -1, 0]], float)
    _, obj, best = score_tree(parent, pos, np.array([1, 9, 9]), 1.0, lam)
    assert obj[1] == obj[2] and best == 1
