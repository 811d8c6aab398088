"""Pins of the oracle's interval mode (Sec. IV-B, Eq. 5-7) against things other than itself.

The interval mode replaces the voxel-centre ancestor test by the paper's screen-space overlap:
each candidate ray is clipped to an ancestor's valid depth range, projected (Eq. 5), clipped to
the buffer (Liang-Barsky), walked pixel by pixel with a 2D DDA, and compared with the stored
depth at one inverse-depth sample per visited pixel (Eq. 6); the observed runs are the
intervals of Eq. 7. The pins tie each step to an independent float64 model built from rotation
matrices (the camera of test_oracle_pins.float_camera), to exact rational slab intersections,
and to closed forms:
  - the depth-clipped, image-clipped segment and its projected endpoints;
  - the walk's portions tile the clipped segment and each lies in its pixel;
  - each portion's depth sample is the perspective-correct depth at the portion's midpoint,
    compared "smaller or equal" (adversarial depth buffers set just above / below it);
  - a sample's screen parameter is the projection of the ray point (perspective-correct);
  - a voxel's sample is the midpoint of the ray's traversal of it;
  - tree-level invariants of Eq. 2 and a bounded gap to the exact marginal gain.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from synth import Sensor
from test_oracle_pins import Q16, Q30, float_camera, rand_dir

Z_NEAR = 1.0 / 1024.0


def _setup(rng, s, T_vox, spread=8.0):
    Pa = (rng.uniform(20, 40, 3) * Q16).astype(np.int64)
    P = Pa + (rng.uniform(-spread, spread, 3) * Q16).astype(np.int64)
    ka = int(rng.integers(0, s.yaw_bins))
    d = rand_dir(rng)
    return Pa, P, ka, d


def _model(s, ka, Pa, P, d, T_vox):
    """float64 camera-frame coordinates of the ray point at fraction lam."""
    R, fx, fy, cx, cy = float_camera(s, ka)
    p0 = np.asarray(P, float) / Q16 - np.asarray(Pa, float) / Q16
    dv = np.asarray(d, float) / Q30 * T_vox

    def cam(lam):
        c = (p0 + np.multiply.outer(np.atleast_1d(lam), dv)) @ R
        return c[:, 0], c[:, 1], c[:, 2]

    def proj(lam):
        x, y, z = cam(lam)
        return fx * x / z + cx, fy * y / z + cy, z

    return cam, proj


SENSORS = [Sensor(90, 60, 36, 24, 4.0, 8, 0.0), Sensor(87, 58, 48, 28, 4.0, 12, 10.0)]


@pytest.mark.parametrize("s", SENSORS)
def test_interval_segment_matches_float_camera(oracle_lib, s):
    rng = np.random.default_rng(11)
    v = 0.2
    Tq = oracle_lib.range_q16(s.range_m, v)
    T_vox = Tq / Q16
    D = np.zeros((s.height, s.width), np.uint32)
    n_vis = n_empty = 0
    lam_grid = np.linspace(0.0, 1.0, 4001)
    for _ in range(300):
        Pa, P, ka, d = _setup(rng, s, T_vox)
        r = oracle_lib.ray_intervals(s, ka, Pa, D, P, d, Tq)
        cam, proj = _model(s, ka, Pa, P, d, T_vox)
        u, vv, z = proj(lam_grid)
        zin = (z >= Z_NEAR) & (z <= T_vox)
        inside = zin & (u > 1e-3) & (u < s.width - 1e-3) & (vv > 1e-3) & (vv < s.height - 1e-3)
        if len(r["portions"]) == 0:
            n_empty += 1
            assert not inside.any()
            continue
        n_vis += 1
        lo, hi, Za, Zb, ua, va, ub, vb, wa, wb, s0, s1 = [float(x) for x in r["seg"]]
        # the depth clip: z >= Z_NEAR and z <= range, exactly where the model says
        ok = np.nonzero(zin)[0]
        assert abs(lo - lam_grid[ok[0]]) <= 3e-4 + 1e-4 and abs(hi - lam_grid[ok[-1]]) <= 3e-4 + 1e-4
        # projected clipped endpoints and their depths (Eq. 5); the oracle's rows are Q16, so camera
        # coordinates carry up to ~3 x 2^-17 x |offset| of rounding, which the pixel divides by z
        fmax = max(float_camera(s, ka)[1:3])
        for lam, Zx, ux, vx in ((lo, Za, ua, va), (hi, Zb, ub, vb)):
            mu, mv, mz = proj(lam)
            ez = 4e-4 + 1e-5 * mz[0]
            assert abs(Zx - mz[0]) <= ez
            if mz[0] > 0.05:
                eu = 2e-3 + fmax * ez / mz[0] * (1 + (abs(mu[0]) + abs(mv[0])) / fmax)
                assert abs(ux - mu[0]) <= eu and abs(vx - mv[0]) <= eu
        assert wa == pytest.approx(1.0 / Za, rel=1e-6) and wb == pytest.approx(1.0 / Zb, rel=1e-6)
        # Liang-Barsky: the 2D segment is inside the buffer exactly on [s0, s1] (to the float32
        # resolution of s times the segment's screen length)
        tol = 2e-3 + 3e-7 * max(abs(ub - ua), abs(vb - va))
        for sx in (s0, s1):
            px, py = ua + sx * (ub - ua), va + sx * (vb - va)
            assert -tol <= px <= s.width + tol and -tol <= py <= s.height + tol
        if s0 > 0:
            px, py = ua + s0 * (ub - ua), va + s0 * (vb - va)
            assert min(abs(px), abs(px - s.width), abs(py), abs(py - s.height)) < tol
        if s1 < 1:
            px, py = ua + s1 * (ub - ua), va + s1 * (vb - va)
            assert min(abs(px), abs(px - s.width), abs(py), abs(py - s.height)) < tol
    assert n_vis > 50 and n_empty > 20


@pytest.mark.parametrize("s", SENSORS)
def test_interval_walk_tiles_the_clipped_segment(oracle_lib, s):
    rng = np.random.default_rng(12)
    v = 0.2
    Tq = oracle_lib.range_q16(s.range_m, v)
    T_vox = Tq / Q16
    D = np.zeros((s.height, s.width), np.uint32)
    n_por = 0
    for _ in range(300):
        Pa, P, ka, d = _setup(rng, s, T_vox)
        r = oracle_lib.ray_intervals(s, ka, Pa, D, P, d, Tq)
        por, pix = r["portions"], r["pixels"]
        if len(por) == 0:
            continue
        lo, hi, Za, Zb, ua, va, ub, vb, wa, wb, s0, s1 = [float(x) for x in r["seg"]]
        assert por[0, 0] == np.float32(s0)
        assert np.array_equal(por[1:, 0], por[:-1, 1])  # contiguous
        steps = np.abs(np.diff(pix, axis=0)).sum(axis=1)
        assert np.all(steps == 1)  # 4-connected 2D DDA
        assert np.all((pix[:, 0] >= 0) & (pix[:, 0] < s.width) & (pix[:, 1] >= 0) & (pix[:, 1] < s.height))
        last = pix[-1]
        edge = last[0] in (0, s.width - 1) or last[1] in (0, s.height - 1)
        assert por[-1, 1] == np.float32(s1) or edge
        for q in range(len(por)):
            a, b = float(por[q, 0]), float(por[q, 1])
            if b - a < 1e-4:
                continue
            sm = 0.5 * (a + b)
            px, py = ua + sm * (ub - ua), va + sm * (vb - va)
            tol = 1e-3 + 3e-7 * max(abs(ub - ua), abs(vb - va))
            assert pix[q, 0] - tol <= px <= pix[q, 0] + 1 + tol and pix[q, 1] - tol <= py <= pix[q, 1] + 1 + tol
            n_por += 1
    assert n_por > 600


def _lam_of_screen(proj, lo, hi, target, axis):
    """Bisection for the ray fraction whose projection has coordinate `target` on `axis`."""
    a, b = lo, hi
    fa = proj(a)[axis][0] - target
    for _ in range(80):
        m = 0.5 * (a + b)
        fm = proj(m)[axis][0] - target
        if (fm < 0) == (fa < 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


@pytest.mark.parametrize("s", SENSORS)
def test_interval_depth_sample_is_perspective_midpoint_smaller_or_equal(oracle_lib, s):
    """Eq. 6 and the "smaller or equal" rule: for every portion, the buffer depth is set just above
    or just below the true depth of the ray point that projects to the portion's midpoint (found
    by bisection on the float64 model, not by the inverse-depth formula); the portion is observed
    exactly when the stored depth is above it."""
    rng = np.random.default_rng(13)
    v = 0.2
    Tq = oracle_lib.range_q16(s.range_m, v)
    T_vox = Tq / Q16
    n_chk = 0
    for _ in range(160):
        Pa, P, ka, d = _setup(rng, s, T_vox, spread=5.0)
        D0 = np.zeros((s.height, s.width), np.uint32)
        r = oracle_lib.ray_intervals(s, ka, Pa, D0, P, d, Tq)
        por, pix = r["portions"], r["pixels"]
        if len(por) == 0:
            continue
        lo, hi, Za, Zb, ua, va, ub, vb, wa, wb, s0, s1 = [float(x) for x in r["seg"]]
        cam, proj = _model(s, ka, Pa, P, d, T_vox)
        axis = 0 if abs(ub - ua) >= abs(vb - va) else 1
        if max(abs(ub - ua), abs(vb - va)) < 0.5:
            continue
        D = np.zeros((s.height, s.width), np.uint32)
        expect = {}
        for q in range(len(por)):
            a, b = float(por[q, 0]), float(por[q, 1])
            if b - a < 2e-3:
                continue
            sm = 0.5 * (a + b)
            target = (ua + sm * (ub - ua)) if axis == 0 else (va + sm * (vb - va))
            lam = _lam_of_screen(proj, lo, hi, target, axis)
            z = float(proj(lam)[2][0])
            delta = int(rng.choice([-200, 200]))  # 3e-3 voxel: above the Q16-row rounding of z
            Dq = int(math.floor(z * Q16)) + delta
            if Dq <= 0:
                continue
            D[pix[q, 1], pix[q, 0]] = Dq
            expect[q] = delta > 0
        if not expect:
            continue
        r2 = oracle_lib.ray_intervals(s, ka, Pa, D, P, d, Tq)
        for q, e in expect.items():
            assert bool(r2["portions"][q, 2]) == e, (q, e)
            n_chk += 1
    assert n_chk > 500


def test_interval_equal_depth_counts_as_observed(oracle_lib):
    """A ray at constant camera depth 4 voxels (yaw 0, pitch 0: camera z = world +x, the ray runs
    along world +y): every sample depth is exactly 4.0, so a buffer holding exactly 4.0 observes
    every portion and one holding 4.0 - 2^-16 none."""
    s = Sensor(90, 60, 36, 24, 4.0, 4, 0.0)
    Tq = 10 * Q16
    Pa = np.array([20 * Q16, 20 * Q16 + 1234, 10 * Q16 + 999], np.int64)
    P = Pa + np.array([4 * Q16, -3 * Q16, 0], np.int64)
    d = np.array([0, Q30, 0], np.int64)
    D = np.full((s.height, s.width), 4 * Q16, np.uint32)
    r = oracle_lib.ray_intervals(s, 0, Pa, D, P, d, Tq)
    assert len(r["portions"]) > 5
    assert np.all(r["portions"][:, 2] == 1)
    r = oracle_lib.ray_intervals(s, 0, Pa, D - 1, P, d, Tq)
    assert np.all(r["portions"][:, 2] == 0)


@pytest.mark.parametrize("s", SENSORS)
def test_interval_sample_parameter_is_perspective_correct(oracle_lib, s):
    rng = np.random.default_rng(14)
    v = 0.2
    Tq = oracle_lib.range_q16(s.range_m, v)
    T_vox = Tq / Q16
    D = np.zeros((s.height, s.width), np.uint32)
    n_chk = 0
    for _ in range(200):
        Pa, P, ka, d = _setup(rng, s, T_vox)
        lam = rng.uniform(0, 1, 64).astype(np.float32)
        r = oracle_lib.ray_intervals(s, ka, Pa, D, P, d, Tq, lam)
        if len(r["portions"]) == 0:
            continue
        lo, hi, Za, Zb, ua, va, ub, vb, wa, wb, s0, s1 = [float(x) for x in r["seg"]]
        if abs(Za - Zb) < 0.5:
            continue
        cam, proj = _model(s, ka, Pa, P, d, T_vox)
        fmax = max(float_camera(s, ka)[1:3])
        for q in range(lam.size):
            if r["lam_obs"][q] < 0:
                continue
            sv = float(r["lam_s"][q])
            mu, mv, mz = proj(float(lam[q]))
            # float32 resolution of s times the screen length, plus the Q16-row rounding over z
            tol = 3e-3 + 3e-7 * max(abs(ub - ua), abs(vb - va)) + fmax * (4e-4 + 1e-5 * mz[0]) / mz[0] * (
                1 + (abs(mu[0]) + abs(mv[0])) / fmax)
            assert abs(ua + sv * (ub - ua) - mu[0]) < tol and abs(va + sv * (vb - va) - mv[0]) < tol
            n_chk += 1
    assert n_chk > 1000


def test_interval_voxel_sample_is_traversal_midpoint(oracle_lib):
    """A voxel's sample is the midpoint of the ray's traversal of it (exact rational slab entry and
    exit, the exit capped at the range), as a fraction of the range."""
    rng = np.random.default_rng(15)
    grid = np.zeros((12, 14, 16), np.uint8)
    n_chk = 0
    for _ in range(60):
        P = (rng.uniform(2, 10, 3) * Q16).astype(np.int64)
        d = rand_dir(rng)
        Tq = int(rng.integers(3 * Q16, 9 * Q16))
        vox, codes, hit, Dd, lam = oracle_lib.trace(grid, P, d, Tq, Q30, want_lambda=True)
        p = [Fr(int(P[a]), Q16) for a in range(3)]
        dd = [Fr(int(d[a]), Q30) for a in range(3)]
        T = Fr(Tq, Q16)
        for m, vx in enumerate(vox.tolist()):
            tin, tout = Fr(0), T
            for a in range(3):
                if dd[a] == 0:
                    continue
                t0 = (vx[a] - p[a]) / dd[a]
                t1 = (vx[a] + 1 - p[a]) / dd[a]
                tin, tout = max(tin, min(t0, t1)), min(tout, max(t0, t1))
            expect = float((tin + tout) / 2 / T)
            assert abs(float(lam[m]) - expect) < 2e-6, (m, float(lam[m]), expect)
            n_chk += 1
    assert n_chk > 300


# ------------------------------------------------------------------- tree-level pins
@pytest.mark.parametrize("seed", [1, 4])
def test_interval_mode_invariants(oracle_lib, seed):
    p = synth.random_small(seed, n_nodes=14)
    args = (p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    r = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_INTERVAL, want_counts=True)
    r0 = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_MARGINAL, want_counts=True)
    root = int(np.nonzero(p.tree.parent < 0)[0][0])
    assert r["marg"][root] == r["abs"][root]
    assert np.all(r["cnt_marg"] <= r["cnt_abs"])
    assert np.array_equal(r["cnt_abs"], r0["cnt_abs"])  # the mode changes only the exclusion
    assert np.all(r["marg"] <= r["abs"])


def test_interval_mode_special_cases(oracle_lib):
    rng = np.random.default_rng(2)
    nx, ny, nz, v = 40, 40, 16, 0.2
    u = rng.random((nz, ny, nx))
    grid = np.where(u < 0.03, 2, np.where(u < 0.2, 1, 0)).astype(np.uint8)
    grid[7:10, 19:22, 19:22] = 1
    c = np.array([20.3, 20.6, 8.2]) * v
    parent = np.array([-1, 0], np.int32)
    pos = np.stack([c, c]).astype(np.float32)
    mode = oracle_lib.MODE_INTERVAL
    s = Sensor(90, 60, 24, 16, 3.0, 2, 0.0)
    r = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s, mode=mode, want_counts=True)
    k_other = 1 - r["yaw"][0]
    assert r["cnt_marg"][1, k_other] == r["cnt_abs"][1, k_other] > 0  # disjoint frusta
    s1 = Sensor(90, 60, 24, 16, 3.0, 1, 0.0)
    r1 = oracle_lib.eval_tree(grid, v, (0, 0, 0), parent, pos, s1, mode=mode)
    assert r1["marg"][1] <= 0.05 * r1["abs"][1]  # identical pose: (almost) everything observed
    free = np.ones_like(grid)
    rf = oracle_lib.eval_tree(free, v, (0, 0, 0), parent, pos, s, mode=mode)
    assert np.all(rf["abs"] == 0) and np.all(rf["marg"] == 0)


def test_interval_mode_gap_to_exact_tiny(oracle_lib):
    p = synth.tiny()
    args = (p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, p.sensor)
    r = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_INTERVAL)
    off, ids = oracle_lib.visible_sets(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.pos, r["yaw"], p.sensor)
    E = oracle_lib.exact_dfs(p.tree.parent, off, ids, p.map.grid.size)
    ratio = r["marg"].sum() / E.sum()
    assert 0.99 <= ratio <= 1.10, ratio
