"""Pins of the oracle's panoramic mode against things other than itself.

The panoramic mode casts each node's rays once over 360 degrees: A azimuth wedges ("columns"),
each a one-pixel-wide strip camera with the pinhole's rows; owned unknown voxels are counted per
column and a yaw bin's gain is the sum over the columns of its window. The pins tie it to:
  - a float64 model of the tables (wedge boundaries, strip rays, window placement by azimuth);
  - float64 azimuth / elevation of voxel centres for the owning cell;
  - a voxel-centric brute force of the owned set (each voxel's cell, that cell's ray traced);
  - the window-sum identity and the closed-form band volume on an all-unknown map;
  - the invariants of Eq. 2 (root marginal == absolute, marginal <= absolute, all-free map).
"""
import math

import numpy as np
import pytest

import synth
from synth import Sensor
from test_oracle_pins import Q16, Q30

SENSORS = [Sensor(90, 60, 36, 24, 4.0, 8, 0.0), Sensor(87, 58, 48, 28, 4.0, 12, 0.0), Sensor(60, 40, 20, 9, 3.0, 6, 0.0)]


def _wrap(a):
    return (a + 180.0) % 360.0 - 180.0


@pytest.mark.parametrize("s", SENSORS)
def test_pano_tables_match_float_model(oracle_lib, s):
    t = oracle_lib.pano_tables(s)
    A, Wc, step = t["A"], t["Wc"], t["step"]
    assert step == math.ceil(s.width * 360 / (s.hfov_deg * s.yaw_bins)) and A == step * s.yaw_bins
    # a column is no wider than the pinhole's central pixel, a window spans the horizontal field of view
    pix = 2 * math.degrees(math.atan(math.tan(math.radians(s.hfov_deg / 2)) / s.width))
    assert 360 / A <= pix + 1e-9
    assert abs(Wc * 360 / A - s.hfov_deg) <= 0.5 * 360 / A
    az = 2 * np.pi * np.arange(A) / A
    assert np.max(np.abs(t["bc"] / Q30 - np.stack([np.cos(az), np.sin(az)], 1))) < 2.0 / Q30
    th = 2 * np.pi * (np.arange(A) + 0.5) / A
    tv = math.tan(math.radians(s.vfov_deg / 2))
    el = np.arctan(-((2 * np.arange(s.height) + 1 - s.height) / s.height) * tv)
    d = np.stack([np.cos(th)[:, None] * np.cos(el)[None], np.sin(th)[:, None] * np.cos(el)[None],
                  np.broadcast_to(np.sin(el)[None], (A, s.height))], -1)
    assert np.max(np.abs(t["dirs"] / Q30 - d)) < 4.0 / Q30
    # window k: the Wc columns whose centre azimuths are nearest the yaw, centred on it
    for k in range(s.yaw_bins):
        psi = 360.0 * k / s.yaw_bins
        cols = (t["wstart"][k] + np.arange(Wc)) % A
        centre = np.degrees(th[cols])
        off = _wrap(centre - psi)
        assert np.all(np.abs(off) <= Wc * 180.0 / A + 1e-9)
        assert abs(off.mean()) <= 0.5 * 360 / A + 1e-9


@pytest.mark.parametrize("s", SENSORS[:2])
def test_pano_cells_match_float_azimuth_elevation(oracle_lib, s):
    rng = np.random.default_rng(21)
    t = oracle_lib.pano_tables(s)
    A = t["A"]
    P = np.array([30 * Q16 + 12345, 31 * Q16 + 2222, 20 * Q16 + 999], np.int64)
    vox = np.stack([rng.integers(5, 56, 6000), rng.integers(5, 56, 6000), rng.integers(5, 36, 6000)], 1).astype(np.int32)
    out = oracle_lib.pano_cells(s, P, vox)
    r = vox + 0.5 - P / Q16
    az = np.degrees(np.arctan2(r[:, 1], r[:, 0])) % 360.0
    col = np.floor(az / (360.0 / A)).astype(int)
    th = 2 * np.pi * (col + 0.5) / A
    rho = r[:, 0] * np.cos(th) + r[:, 1] * np.sin(th)
    tv = math.tan(math.radians(s.vfov_deg / 2))
    fy = (s.height / 2) / tv
    v = fy * (-r[:, 2]) / rho + s.height / 2
    frac_az = az / (360.0 / A) - col
    safe = (np.minimum(frac_az, 1 - frac_az) > 1e-4) & (np.abs(v - np.round(v)) > 1e-3)
    inside = (v >= 0) & (v < s.height) & (rho > 0)
    exp_c = np.where(inside, col, -1)
    exp_j = np.where(inside, np.floor(v).astype(int), -1)
    assert np.array_equal(out[safe, 0], exp_c[safe]) and np.array_equal(out[safe, 1], exp_j[safe])
    assert safe.sum() > 5000 and (out[:, 0] >= 0).sum() > 1000


@pytest.mark.parametrize("seed", [3, 8])
def test_pano_owner_set_equals_voxel_centric_brute_force(oracle_lib, seed):
    """Ray-centric per-column counts == voxel-centric: every unknown voxel's owning cell, whose ray
    is traced to check that it reaches the voxel. The node sits on a voxel-centre plane (y), so some
    voxel centres lie exactly on a wedge boundary and must be owned once."""
    rng = np.random.default_rng(seed)
    s = Sensor(90, 60, 12, 8, 2.0, 4, 0.0)
    nz, ny, nx = 14, 22, 22
    u = rng.random((nz, ny, nx))
    grid = np.where(u < 0.04, 2, np.where(u < 0.3, 1, 0)).astype(np.uint8)
    v = 0.2
    P = np.array([11 * Q16 + 2345, 11 * Q16 + Q16 // 2, 7 * Q16 + 4321], np.int64)
    grid[P[2] >> 16, P[1] >> 16, P[0] >> 16] = 1
    Tq = oracle_lib.range_q16(s.range_m, v)
    cols = oracle_lib.pano_node_columns(grid, P, s, Tq)
    t = oracle_lib.pano_tables(s)
    unk = np.argwhere(grid == 0)[:, ::-1].astype(np.int32)  # (x, y, z)
    cells = oracle_lib.pano_cells(s, P, unk)
    brute = np.zeros(t["A"], np.int64)
    for vx, cj in zip(unk, cells):
        c, j = int(cj[0]), int(cj[1])
        if c < 0:
            continue
        vis, codes, hit, D = oracle_lib.trace(grid, P, t["dirs"][c, j].astype(np.int64), Tq, Q30)
        if any((vis == vx).all(axis=1)):
            brute[c] += 1
    assert np.array_equal(cols, brute)
    assert brute.sum() > 100


@pytest.mark.parametrize("s", [SENSORS[0], SENSORS[2]])
def test_pano_window_sums_and_identity(oracle_lib, s):
    p = synth.random_small(5, n_nodes=1, sensor=s)
    r = oracle_lib.eval_tree(p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, s,
                             mode=oracle_lib.MODE_PANORAMIC, want_counts=True)
    P = oracle_lib.quantize(p.tree.pos, p.map.origin, p.map.voxel_size, p.map.grid.shape[::-1])[0]
    cols = oracle_lib.pano_node_columns(p.map.grid, P, s, oracle_lib.range_q16(s.range_m, p.map.voxel_size))
    t = oracle_lib.pano_tables(s)
    A, Wc = t["A"], t["Wc"]
    th = np.degrees(2 * np.pi * (np.arange(A) + 0.5) / A)
    for k in range(s.yaw_bins):
        win = np.abs(_wrap(th - 360.0 * k / s.yaw_bins)) < s.hfov_deg / 2  # centres inside the field of view
        assert win.sum() == Wc
        assert r["cnt_abs"][0, k] == cols[win].sum()
    if (Wc * s.yaw_bins) % A == 0:
        assert r["cnt_abs"][0].sum() == (Wc * s.yaw_bins // A) * cols.sum()
    assert np.array_equal(r["cnt_abs"], r["cnt_marg"])  # no ancestors: nothing excluded


def test_pano_all_unknown_band_volume(oracle_lib):
    """All-unknown map: the owned voxels fill the elevation band |el| <= vfov/2 of the range ball,
    volume (4 pi / 3) R^3 sin(vfov / 2), with R the range plus about half a voxel (a voxel is
    visited when the ray enters it before the range, so centres reach a little beyond it)."""
    s = Sensor(90, 60, 40, 30, 3.0, 8, 0.0)
    v = 0.1
    n = 72
    grid = np.zeros((n, n, n), np.uint8)
    P = np.array([36 * Q16 + 1234, 36 * Q16 + 5678, 36 * Q16 + 910], np.int64)
    Tq = oracle_lib.range_q16(s.range_m, v)
    cols = oracle_lib.pano_node_columns(grid, P, s, Tq)
    R = Tq / Q16 + 0.5
    expect = 4 * math.pi / 3 * R ** 3 * math.sin(math.radians(s.vfov_deg / 2))
    assert abs(cols.sum() / expect - 1) < 0.04, cols.sum() / expect
    # the same count at half the vertical field of view scales with sin(vfov / 2)
    s2 = Sensor(90, 30, 40, 15, 3.0, 8, 0.0)
    cols2 = oracle_lib.pano_node_columns(grid, P, s2, Tq)
    ratio = cols2.sum() / cols.sum()
    assert abs(ratio - math.sin(math.radians(15)) / math.sin(math.radians(30))) < 0.03, ratio


@pytest.mark.parametrize("seed", [1, 4])
def test_pano_mode_invariants(oracle_lib, seed):
    s = Sensor(90, 60, 16, 10, 2.0, 8, 0.0)
    p = synth.random_small(seed, n_nodes=14, sensor=s)
    args = (p.map.grid, p.map.voxel_size, p.map.origin, p.tree.parent, p.tree.pos, s)
    r = oracle_lib.eval_tree(*args, mode=oracle_lib.MODE_PANORAMIC, want_counts=True)
    root = int(np.nonzero(p.tree.parent < 0)[0][0])
    assert r["marg"][root] == r["abs"][root]
    assert np.all(r["cnt_marg"] <= r["cnt_abs"]) and np.all(r["marg"] <= r["abs"])
    assert np.all(r["yaw"] == np.argmax(r["cnt_marg"], axis=1))
    free = np.ones_like(p.map.grid)
    rf = oracle_lib.eval_tree(free, *args[1:], mode=oracle_lib.MODE_PANORAMIC)
    assert np.all(rf["abs"] == 0)
    with pytest.raises(oracle_lib.OracleError):  # level camera only
        oracle_lib.eval_tree(*args[:-1], Sensor(90, 60, 16, 10, 2.0, 8, 10.0), mode=oracle_lib.MODE_PANORAMIC)
