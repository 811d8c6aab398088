"""CPU oracle for path-dependent marginal information gain (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
package. It shares no code with the CUDA library (paper_2609_40297_gb300) and never
imports it. The arithmetic lives in mig_oracle.c (a plain C restatement of Sec. III-IV);
this module compiles it with gcc, loads it with ctypes and adds the hash-set route of the
exact marginal gain (exact.py).

Functions with no pin of their own: none — every entry point is pinned by
tests/test_oracle_*.py (see the pins listed there).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mig_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmig_oracle.so")
_lock = threading.Lock()
_lib = None

MODE_MARGINAL, MODE_SINGLE_PARENT, MODE_ABSOLUTE, MODE_INTERVAL, MODE_PANORAMIC = 0, 1, 2, 3, 4


_MUTANT = 0  # planted-mistake variant (pin-strength tests only); 0 = the oracle


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               f"-DORACLE_MUTANT={int(_MUTANT)}", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_variant(mutant: int):
    """A separate instance of this module bound to a build with one planted mistake
    (ORACLE_MUTANT=m). Used only to show that the pins catch each plausible mistake."""
    import importlib.util
    import sys
    name = f"oracle_mutant_{int(mutant)}"
    if name in sys.modules:
        return sys.modules[name]
    spec = importlib.util.spec_from_file_location(name, os.path.abspath(__file__))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._MUTANT = int(mutant)
    mod._LIB_PATH = os.path.join(_BUILD, f"libmig_oracle_m{int(mutant)}.so")
    sys.modules[name] = mod
    return mod


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            p = C.c_void_p
            i, f = C.c_int, C.c_float
            L.oracle_eval_tree.argtypes = [p, i, i, i, f, p, i, p, p, f, f, i, i, f, i, f, i, p, p, p, p, p, p, p, i]
            L.oracle_camera_tables.argtypes = [f, f, i, i, i, f, p, p, p, p, p, p]
            L.oracle_ray_dirs.argtypes = [f, f, i, i, i, f, p]
            L.oracle_trace.argtypes = [p, i, i, i, p, p, C.c_int64, C.c_int64, i, p, p, p, p, p]
            L.oracle_project.argtypes = [f, f, i, i, i, f, i, p, i, p, p]
            L.oracle_quantize.argtypes = [p, i, p, f, i, i, i, p]
            L.oracle_observed.argtypes = [f, f, i, i, i, f, i, p, p, p]
            L.oracle_visible_sets.argtypes = [p, i, i, i, f, p, i, p, p, f, f, i, i, f, i, f, p, p, p, i]
            L.oracle_exact_dfs.argtypes = [i, p, p, p, C.c_int64, p, p]
            L.oracle_ray_intervals.argtypes = [f, f, i, i, i, f, i, p, p, p, p, C.c_int64, i, p, p, i, p, p, p, p]
            i64 = C.c_int64
            L.oracle_sample_lambda.argtypes = [i64, i64, i64, i64, i64]
            L.oracle_sample_lambda.restype = C.c_float
            L.oracle_pano_tables.argtypes = [f, f, i, i, i, f, p, p, p, p, p]
            L.oracle_pano_cells.argtypes = [f, f, i, i, i, f, p, i, p, p]
            L.oracle_pano_node_columns.argtypes = [p, i, i, i, p, f, f, i, i, i, f, C.c_int64, p]
            L.oracle_exact_yaw.argtypes = [p, i, i, i, f, p, i, p, p, f, f, i, i, f, i, f, p, p, p, i]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleError(RuntimeError):
    pass


def eval_tree(grid, voxel, origin, parent, pos, sensor, mode=MODE_MARGINAL, node_mask=None,
              want_counts=False, want_depth=False, n_threads=0):
    """Depth-buffer method over the whole tree (or an ancestor-closed subset).

    grid: uint8 (nz, ny, nx) codes; parent int32 [n]; pos float32 [n,3] metres;
    sensor: object with hfov_deg, vfov_deg, width, height, range_m, yaw_bins, pitch_deg.
    Returns dict with abs, marg, yaw (int32 [n]) and optionally cnt_abs/cnt_marg [n,K],
    depth [n,H,W] (uint32, Q16 voxel units)."""
    grid = _c(grid, np.uint8)
    nz, ny, nx = grid.shape
    parent = _c(parent, np.int32)
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = parent.shape[0]
    K, W, H = sensor.yaw_bins, sensor.width, sensor.height
    org = _c(origin, np.float32)
    absv = np.zeros(n, np.int32)
    marg = np.zeros(n, np.int32)
    yaw = np.zeros(n, np.int32)
    ca = np.zeros((n, K), np.int32) if want_counts else None
    cm = np.zeros((n, K), np.int32) if want_counts else None
    dep = np.zeros((n, H, W), np.uint32) if want_depth else None
    mask = None if node_mask is None else _c(node_mask, np.uint8)
    rc = lib().oracle_eval_tree(_ptr(grid), nx, ny, nz, float(voxel), _ptr(org), n, _ptr(parent), _ptr(pos),
                                float(sensor.hfov_deg), float(sensor.vfov_deg), int(W), int(H), float(sensor.range_m),
                                int(K), float(sensor.pitch_deg), int(mode), _ptr(mask), _ptr(absv), _ptr(marg),
                                _ptr(yaw), _ptr(ca), _ptr(cm), _ptr(dep), int(n_threads))
    if rc != 0:
        raise OracleError(f"oracle_eval_tree failed: {rc}")
    out = {"abs": absv, "marg": marg, "yaw": yaw}
    if want_counts:
        out["cnt_abs"], out["cnt_marg"] = ca, cm
    if want_depth:
        out["depth"] = dep
    return out


def camera_tables(sensor):
    W, H, K = sensor.width, sensor.height, sensor.yaw_bins
    body = np.zeros((H, W, 3), np.int32)
    dzc = np.zeros((H, W), np.int32)
    ck = np.zeros(K, np.int32)
    sk = np.zeros(K, np.int32)
    M = np.zeros((K, 3, 3), np.int32)
    tv = np.zeros(4, np.float64)
    rc = lib().oracle_camera_tables(float(sensor.hfov_deg), float(sensor.vfov_deg), W, H, K, float(sensor.pitch_deg),
                                    _ptr(body), _ptr(dzc), _ptr(ck), _ptr(sk), _ptr(M), _ptr(tv))
    if rc != 0:
        raise OracleError(f"oracle_camera_tables failed: {rc}")
    return {"body": body, "dzc": dzc, "ck": ck, "sk": sk, "M": M, "t_h": tv[0], "t_v": tv[1], "cp": tv[2], "sp": tv[3]}


def ray_dirs(sensor):
    W, H, K = sensor.width, sensor.height, sensor.yaw_bins
    out = np.zeros((K, H, W, 3), np.int64)
    rc = lib().oracle_ray_dirs(float(sensor.hfov_deg), float(sensor.vfov_deg), W, H, K, float(sensor.pitch_deg),
                               _ptr(out))
    if rc != 0:
        raise OracleError(f"oracle_ray_dirs failed: {rc}")
    return out


def trace(grid, P, d, Tq, dzc, cap=100000, want_lambda=False):
    """One DDA ray; returns (voxels [m,3], codes [m], hit, D), plus the interval-mode sample
    fraction of each visited voxel when want_lambda."""
    grid = _c(grid, np.uint8)
    nz, ny, nx = grid.shape
    P = _c(P, np.int64)
    d = _c(d, np.int64)
    vox = np.zeros((cap, 3), np.int32)
    codes = np.zeros(cap, np.uint8)
    hit = np.zeros(1, np.int32)
    D = np.zeros(1, np.uint32)
    lam = np.zeros(cap, np.float32) if want_lambda else None
    m = lib().oracle_trace(_ptr(grid), nx, ny, nz, _ptr(P), _ptr(d), int(Tq), int(dzc), cap, _ptr(vox), _ptr(codes),
                           _ptr(hit), _ptr(D), _ptr(lam))
    if m < 0:
        raise OracleError("oracle_trace: invalid ray")
    if m > cap:
        raise OracleError("oracle_trace: cap exceeded")
    out = (vox[:m].copy(), codes[:m].copy(), bool(hit[0]), int(D[0]))
    return out + (lam[:m].copy(),) if want_lambda else out


def project(sensor, k, P, vox):
    vox = _c(vox, np.int32).reshape(-1, 3)
    P = _c(P, np.int64)
    out = np.zeros((vox.shape[0], 4), np.int64)
    rc = lib().oracle_project(float(sensor.hfov_deg), float(sensor.vfov_deg), sensor.width, sensor.height,
                              sensor.yaw_bins, float(sensor.pitch_deg), int(k), _ptr(P), vox.shape[0], _ptr(vox),
                              _ptr(out))
    if rc != 0:
        raise OracleError("oracle_project failed")
    return out


def observed(sensor, k, P, D, vox):
    """Is voxel `vox` observed by the camera at P (Q16) with yaw k and depth buffer D?"""
    D = _c(D, np.uint32)
    rc = lib().oracle_observed(float(sensor.hfov_deg), float(sensor.vfov_deg), sensor.width, sensor.height,
                               sensor.yaw_bins, float(sensor.pitch_deg), int(k), _ptr(_c(P, np.int64)), _ptr(D),
                               _ptr(_c(vox, np.int32)))
    if rc < 0:
        raise OracleError("oracle_observed failed")
    return bool(rc)


def ray_intervals(sensor, ka, Pa, D, P, d, Tq, lam=()):
    """The interval construction (Sec. IV-B, Eq. 5-7) of one candidate ray (origin P, Q16; direction
    d, Q30; range Tq, Q16) against one ancestor (position Pa, yaw bin ka, depth buffer D [H, W]).

    Returns a dict: seg (lo, hi, Za, Zb, ua, va, ub, vb, wa, wb, s0, s1), portions [m, 3]
    (s_in, s_out, observed) and their pixels [m, 2] in walk order, and for each ray fraction in
    `lam` its screen parameter and observation (-1 = outside the ancestor's depth range or image)."""
    W, H = sensor.width, sensor.height
    cap = W + H + 2
    lam = _c(np.asarray(lam, np.float32).reshape(-1), np.float32)
    seg = np.zeros(12, np.float32)
    por = np.zeros((cap, 3), np.float32)
    pix = np.zeros((cap, 2), np.int32)
    lo = np.zeros(max(1, lam.size), np.int32)
    ls = np.zeros(max(1, lam.size), np.float32)
    m = lib().oracle_ray_intervals(float(sensor.hfov_deg), float(sensor.vfov_deg), W, H, sensor.yaw_bins,
                                   float(sensor.pitch_deg), int(ka), _ptr(_c(Pa, np.int64)), _ptr(_c(D, np.uint32)),
                                   _ptr(_c(P, np.int64)), _ptr(_c(d, np.int64)), int(Tq), int(lam.size), _ptr(lam),
                                   _ptr(seg), cap, _ptr(por), _ptr(pix), _ptr(lo), _ptr(ls))
    if m < 0:
        raise OracleError("oracle_ray_intervals failed")
    return {"seg": seg, "portions": por[:m].copy(), "pixels": pix[:m].copy(), "lam_obs": lo[:lam.size].copy(),
            "lam_s": ls[:lam.size].copy()}


def sample_lambda(ne, ade, nx, adx, Tq):
    """Interval mode: a voxel's sample, the midpoint of the ray's traversal (entry ne/ade, exit
    nx/adx, capped at the range), as a fraction of the range."""
    return float(lib().oracle_sample_lambda(int(ne), int(ade), int(nx), int(adx), int(Tq)))


def pano_tables(sensor):
    """Panoramic mode tables: dict with A (columns), Wc (columns per yaw window), step (columns per
    yaw bin), bc [A, 2] (wedge boundary cos/sin, Q30), dirs [A, H, 3] (ray of each cell, Q30),
    rows [A, 6] (strip rows mv, mz, Q16) and wstart [K] (first column of each yaw's window)."""
    W, H, K = sensor.width, sensor.height, sensor.yaw_bins
    dims = np.zeros(3, np.int32)
    args = (float(sensor.hfov_deg), float(sensor.vfov_deg), W, H, K, float(sensor.pitch_deg))
    rc = lib().oracle_pano_tables(*args, _ptr(dims), None, None, None, None)
    if rc != 0:
        raise OracleError(f"oracle_pano_tables failed: {rc}")
    A = int(dims[0])
    bc = np.zeros((A, 2), np.int32)
    dirs = np.zeros((A, H, 3), np.int32)
    rows = np.zeros((A, 6), np.int32)
    ws = np.zeros(K, np.int32)
    lib().oracle_pano_tables(*args, _ptr(dims), _ptr(bc), _ptr(dirs), _ptr(rows), _ptr(ws))
    return {"A": A, "Wc": int(dims[1]), "step": int(dims[2]), "bc": bc, "dirs": dirs, "rows": rows, "wstart": ws}


def pano_cells(sensor, P, vox):
    """Owning (column, row) of each voxel seen from P (Q16) by search over every wedge; -1 = none."""
    vox = _c(vox, np.int32).reshape(-1, 3)
    out = np.zeros((vox.shape[0], 2), np.int32)
    rc = lib().oracle_pano_cells(float(sensor.hfov_deg), float(sensor.vfov_deg), sensor.width, sensor.height,
                                 sensor.yaw_bins, float(sensor.pitch_deg), _ptr(_c(P, np.int64)), vox.shape[0],
                                 _ptr(vox), _ptr(out))
    if rc != 0:
        raise OracleError("oracle_pano_cells failed")
    return out


def pano_node_columns(grid, P, sensor, Tq):
    """Per-column absolute counts of one node (no ancestors) in the panoramic mode."""
    grid = _c(grid, np.uint8)
    nz, ny, nx = grid.shape
    A = pano_tables(sensor)["A"]
    out = np.zeros(A, np.int64)
    rc = lib().oracle_pano_node_columns(_ptr(grid), nx, ny, nz, _ptr(_c(P, np.int64)), float(sensor.hfov_deg),
                                        float(sensor.vfov_deg), sensor.width, sensor.height, sensor.yaw_bins,
                                        float(sensor.pitch_deg), int(Tq), _ptr(out))
    if rc != 0:
        raise OracleError("oracle_pano_node_columns failed")
    return out


def quantize(pos, origin, voxel, dims):
    pos = _c(pos, np.float32).reshape(-1, 3)
    org = _c(origin, np.float32)
    P = np.zeros((pos.shape[0], 3), np.int64)
    rc = lib().oracle_quantize(_ptr(pos), pos.shape[0], _ptr(org), float(voxel), int(dims[0]), int(dims[1]),
                               int(dims[2]), _ptr(P))
    if rc != 0:
        raise OracleError("position outside the grid")
    return P


def range_q16(range_m, voxel):
    return int(np.rint((float(np.float32(range_m)) / float(np.float32(voxel))) * 65536.0))


def visible_sets(grid, voxel, origin, pos, yaws, sensor, node_mask=None, n_threads=0):
    """I(n, yaws[n]) for every node: (offsets int64 [n+1], ids int32 sorted per node)."""
    grid = _c(grid, np.uint8)
    nz, ny, nx = grid.shape
    pos = _c(pos, np.float32).reshape(-1, 3)
    yaws = _c(yaws, np.int32)
    n = pos.shape[0]
    org = _c(origin, np.float32)
    offsets = np.zeros(n + 1, np.int64)
    mask = None if node_mask is None else _c(node_mask, np.uint8)
    args = (_ptr(grid), nx, ny, nz, float(voxel), _ptr(org), n, _ptr(pos), _ptr(yaws), float(sensor.hfov_deg),
            float(sensor.vfov_deg), sensor.width, sensor.height, float(sensor.range_m), sensor.yaw_bins,
            float(sensor.pitch_deg), _ptr(mask))
    rc = lib().oracle_visible_sets(*args, _ptr(offsets), None, int(n_threads))
    if rc != 0:
        raise OracleError("oracle_visible_sets failed")
    ids = np.zeros(max(1, int(offsets[-1])), np.int32)
    rc = lib().oracle_visible_sets(*args, _ptr(offsets), _ptr(ids), int(n_threads))
    if rc != 0:
        raise OracleError("oracle_visible_sets failed")
    return offsets, ids[:int(offsets[-1])]


def exact_yaw(grid, voxel, origin, parent, pos, sensor, node_mask=None, n_threads=0):
    """The exact-yaw variant: each node takes the yaw maximising its exact marginal gain (Eq. 2)
    given its ancestors' own exact choices. Returns (yaw, E) int32 [n] (-1 outside node_mask)."""
    grid = _c(grid, np.uint8)
    nz, ny, nx = grid.shape
    parent = _c(parent, np.int32)
    pos = _c(pos, np.float32).reshape(-1, 3)
    n = parent.shape[0]
    yaw = np.full(n, -1, np.int32)
    E = np.full(n, -1, np.int32)
    mask = None if node_mask is None else _c(node_mask, np.uint8)
    rc = lib().oracle_exact_yaw(_ptr(grid), nx, ny, nz, float(voxel), _ptr(_c(origin, np.float32)), n, _ptr(parent),
                                _ptr(pos), float(sensor.hfov_deg), float(sensor.vfov_deg), sensor.width, sensor.height,
                                float(sensor.range_m), sensor.yaw_bins, float(sensor.pitch_deg), _ptr(mask), _ptr(yaw),
                                _ptr(E), int(n_threads))
    if rc != 0:
        raise OracleError(f"oracle_exact_yaw failed: {rc}")
    return yaw, E


def exact_dfs(parent, offsets, ids, nvox, node_mask=None):
    parent = _c(parent, np.int32)
    n = parent.shape[0]
    E = np.full(n, -1, np.int32)
    mask = None if node_mask is None else _c(node_mask, np.uint8)
    rc = lib().oracle_exact_dfs(n, _ptr(parent), _ptr(_c(offsets, np.int64)), _ptr(_c(ids, np.int32)), int(nvox),
                                _ptr(mask), _ptr(E))
    if rc != 0:
        raise OracleError("oracle_exact_dfs failed")
    return E


from oracle.exact import exact_hash_merge, exact_sorted_merge, gap_report  # noqa: E402,F401
