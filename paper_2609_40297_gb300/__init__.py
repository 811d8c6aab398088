"""Python binding of libmig.so: path-dependent marginal information gain on one GB300.

Argument marshalling only: every step of the path runs in the library's CUDA kernels. PyTorch
provides device memory (the caching allocator plugs into the library's allocator hook) and
streams. There is no CPU fallback: if libmig.so is missing or cannot load, importing the
binding's entry points raises.

Names follow the C ABI in include/mig.h (mig_ctx_create -> Context, mig_map_create -> Map,
mig_tree_eval -> tree_eval, ...).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmig.so")

MIG_OK, MIG_EINVAL, MIG_ENOMEM, MIG_ECUDA, MIG_ETIMEOUT, MIG_EBUSY, MIG_ENOTFOUND = range(7)
COUNT_AUTO, COUNT_RAYS, COUNT_PAIRS, COUNT_NODES = 0, 1, 2, 3
MODE_MARGINAL, MODE_SINGLE_PARENT, MODE_ABSOLUTE, MODE_INTERVAL, MODE_PANORAMIC = 0, 1, 2, 3, 4
BUILD_CHECKED = 1  # mig_build_flags(): the bounds-checked build
STATUS_NAMES = {0: "MIG_OK", 1: "MIG_EINVAL", 2: "MIG_ENOMEM", 3: "MIG_ECUDA", 4: "MIG_ETIMEOUT", 5: "MIG_EBUSY",
                6: "MIG_ENOTFOUND"}

# every symbol declared in include/mig.h
EXPORTS = [
    "mig_ctx_create", "mig_ctx_destroy", "mig_ctx_set_stream", "mig_ctx_sync",
    "mig_map_create", "mig_map_update", "mig_map_read", "mig_map_destroy",
    "mig_default_resolution", "mig_tree_check",
    "mig_tree_eval", "mig_tree_eval_ex", "mig_tree_eval_device", "mig_tree_eval_device_noalloc",
    "mig_tree_score", "mig_tree_score_device",
    "mig_tree_eval_batch", "mig_batch_set_tiles", "mig_batch_get_tiles", "mig_batch_set_timeout",
    "mig_batch_graph_stats", "mig_batch_trace", "mig_batch_trace_read", "mig_autotune",
    "mig_server_create", "mig_server_submit", "mig_server_poll", "mig_server_map_update", "mig_server_timing",
    "mig_server_destroy", "mig_ctx_profile", "mig_ctx_profile_read", "mig_tree_eval_stats", "mig_last_error",
    "mig_build_flags", "mig_probe_gather", "mig_ctx_set_count_kernel", "mig_server_memory",
]


class MigError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Sensor(C.Structure):
    _fields_ = [("hfov_deg", C.c_float), ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("range_m", C.c_float), ("yaw_bins", C.c_int32), ("pitch_deg", C.c_float)]

    @classmethod
    def of(cls, s):
        if isinstance(s, cls):
            return s
        return cls(float(s.hfov_deg), float(s.vfov_deg), int(s.width), int(s.height), float(s.range_m),
                   int(s.yaw_bins), float(s.pitch_deg))


class EvalOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("counts_abs", C.c_void_p), ("counts_marg", C.c_void_p),
                ("depth_buffers", C.c_void_p)]


class TreeDesc(C.Structure):
    _fields_ = [("map", C.c_void_p), ("n_nodes", C.c_int32), ("parent", C.c_void_p), ("pos_m", C.c_void_p),
                ("sensor", Sensor), ("mode", C.c_int32), ("abs_gain", C.c_void_p), ("marg_gain", C.c_void_p),
                ("best_yaw", C.c_void_p)]


class KernelTimes(C.Structure):
    _fields_ = [("count_ms", C.c_double), ("select_ms", C.c_double), ("render_ms", C.c_double),
                ("plan_ms", C.c_double), ("batch_ms", C.c_double), ("count_launches", C.c_uint64),
                ("select_launches", C.c_uint64), ("render_launches", C.c_uint64), ("plan_launches", C.c_uint64),
                ("batch_launches", C.c_uint64), ("cast_ms", C.c_double), ("voxel_ms", C.c_double),
                ("cast_launches", C.c_uint64), ("voxel_launches", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EvalStats(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("rays", "dda_steps", "unknown_visits", "samples", "ancestor_tests",
                                          "depth_reads", "render_rays", "render_steps", "count_launches",
                                          "render_launches", "cast_rays", "cast_steps", "cast_jumps",
                                          "voxel_candidates", "voxel_unknown", "visit_tests", "owned_samples",
                                          "voxel_ancestor_tests", "voxel_depth_reads", "voxel_pass")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class TraceRec(C.Structure):
    _fields_ = [("tree", C.c_int32), ("level", C.c_int32), ("phase", C.c_int32), ("items", C.c_int32),
                ("activated_us", C.c_double), ("done_us", C.c_double)]


class TileConfig(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("ctas_per_sm", C.c_int32), ("engine", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libmig.so (built in-tree by __graft_entry__.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            p, i, f = C.c_void_p, C.c_int, C.c_float
            st = C.c_int
            sig = {
                "mig_ctx_create": (st, [i, p, p, p]),
                "mig_ctx_destroy": (None, [p]),
                "mig_ctx_set_stream": (st, [p, p]),
                "mig_ctx_sync": (st, [p]),
                "mig_map_create": (st, [p, i, i, i, f, p, p, p]),
                "mig_map_update": (st, [p, i, i, i, i, i, i, p]),
                "mig_map_read": (st, [p, p]),
                "mig_map_destroy": (None, [p]),
                "mig_default_resolution": (st, [p, f, p, p]),
                "mig_tree_check": (st, [i, p, p, p]),
                "mig_tree_eval": (st, [p, i, p, p, p, p, p, p]),
                "mig_tree_eval_ex": (st, [p, i, p, p, p, p, p, p, p]),
                "mig_tree_eval_device": (st, [p, i, p, p, p, i, p, p, p]),
                "mig_tree_eval_device_noalloc": (st, [p, i, p, p, p, i, p, p, p]),
                "mig_tree_score": (st, [p, i, p, p, p, C.c_double, C.c_double, p, p, p]),
                "mig_tree_score_device": (st, [p, i, p, p, p, C.c_double, C.c_double, p, p, p]),
                "mig_tree_eval_batch": (st, [p, i, p]),
                "mig_batch_set_tiles": (st, [p, p]),
                "mig_batch_get_tiles": (st, [p, p]),
                "mig_batch_set_timeout": (st, [p, C.c_int64, i]),
                "mig_batch_graph_stats": (st, [p, p, p]),
                "mig_batch_trace": (st, [p, i]),
                "mig_autotune": (st, [p, i, p, i, p, i, p, p]),
                "mig_batch_trace_read": (st, [p, p, i, p]),
                "mig_server_create": (st, [p, C.c_size_t, i, p]),
                "mig_server_submit": (st, [p, p, p]),
                "mig_server_poll": (st, [p, C.c_uint64, C.c_int64]),
                "mig_server_map_update": (st, [p, p, i, i, i, i, i, i, p]),
                "mig_server_timing": (st, [p, C.c_uint64, p, p, p]),
                "mig_server_destroy": (None, [p]),
                "mig_ctx_profile": (st, [p, i]),
                "mig_ctx_profile_read": (st, [p, p]),
                "mig_tree_eval_stats": (st, [p, i, p, p, p, p, p, p, p]),
                "mig_last_error": (C.c_char_p, []),
                "mig_build_flags": (i, []),
                "mig_probe_gather": (st, [p, C.c_uint64, i, p]),
                "mig_ctx_set_count_kernel": (st, [p, i, C.c_uint64]),
                "mig_server_memory": (st, [p, p, p, p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().mig_last_error().decode()


def check(status):
    if status != MIG_OK:
        raise MigError(status, last_error())


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _torch_allocator(device):
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:  # out of memory -> NULL -> MIG_ENOMEM
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return Allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)


class Context:
    """mig_ctx: one GPU, one stream (default: torch's current stream), torch's allocator."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = True):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._alloc = _torch_allocator(device) if torch_allocator else None
        out = C.c_void_p()
        check(lib().mig_ctx_create(device, C.c_void_p(handle),
                                   C.byref(self._alloc) if self._alloc is not None else None, C.byref(out)))
        self.h = out

    def sync(self):
        check(lib().mig_ctx_sync(self.h))

    def set_tiles(self, tile_w, tile_h, ctas_per_sm=4, engine=None):
        if engine is None:
            engine = self.get_tiles()[3]
        check(lib().mig_batch_set_tiles(self.h, C.byref(TileConfig(tile_w, tile_h, ctas_per_sm, engine))))

    def set_batch_timeout(self, timeout_us, debug_stall=False):
        check(lib().mig_batch_set_timeout(self.h, int(timeout_us), 1 if debug_stall else 0))

    def graph_stats(self):
        a, b = C.c_uint64(), C.c_uint64()
        check(lib().mig_batch_graph_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def batch_trace(self, enable=True):
        check(lib().mig_batch_trace(self.h, 1 if enable else 0))

    def batch_trace_read(self):
        n = C.c_int()
        check(lib().mig_batch_trace_read(self.h, None, 0, C.byref(n)))
        recs = (TraceRec * max(1, n.value))()
        check(lib().mig_batch_trace_read(self.h, recs, n.value, C.byref(n)))
        return [{f: getattr(r, f) for f, _ in TraceRec._fields_} for r in recs[:n.value]]

    def get_tiles(self):
        t = TileConfig()
        check(lib().mig_batch_get_tiles(self.h, C.byref(t)))
        return (t.tile_w, t.tile_h, t.ctas_per_sm, t.engine)

    def set_count_kernel(self, kernel=0, steps_budget_bytes=0):
        """mig_ctx_set_count_kernel: COUNT_AUTO (0, default), COUNT_RAYS (1, also True), COUNT_PAIRS (2) or
        COUNT_NODES (3); steps_budget_bytes bounds the owned-voxel step-count buffer (0 = the default)."""
        check(lib().mig_ctx_set_count_kernel(self.h, int(kernel), int(steps_budget_bytes)))

    def profile(self, enable=True):
        check(lib().mig_ctx_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        t = KernelTimes()
        check(lib().mig_ctx_profile_read(self.h, C.byref(t)))
        return t.as_dict()

    def close(self):
        if getattr(self, "h", None):
            lib().mig_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Map:
    """mig_map: a device-resident voxel grid (codes 0 unknown, 1 free, 2 occupied)."""

    def __init__(self, ctx: Context, grid, voxel_size, origin=(0.0, 0.0, 0.0)):
        g = None if grid is None else _host(grid, np.uint8)
        if g is None:
            raise ValueError("grid is required (shape nz, ny, nx)")
        nz, ny, nx = g.shape
        org = (C.c_float * 3)(*[float(x) for x in origin])
        out = C.c_void_p()
        check(lib().mig_map_create(ctx.h, nx, ny, nz, float(voxel_size), org, _ptr(g), C.byref(out)))
        self.h = out
        self.ctx = ctx
        self.shape = (nz, ny, nx)
        self.voxel_size = float(voxel_size)
        self.origin = tuple(float(x) for x in origin)

    def update(self, x0, y0, z0, box):
        b = _host(box, np.uint8)
        dz, dy, dx = b.shape
        check(lib().mig_map_update(self.h, x0, y0, z0, dx, dy, dz, _ptr(b)))

    def read(self):
        out = np.empty(self.shape, np.uint8)
        check(lib().mig_map_read(self.h, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().mig_map_destroy(self.h)
            self.h = None


def default_resolution(sensor, voxel_size):
    w, h = C.c_int32(), C.c_int32()
    s = Sensor.of(sensor)
    check(lib().mig_default_resolution(C.byref(s), float(voxel_size), C.byref(w), C.byref(h)))
    return w.value, h.value


def tree_check(parent):
    parent = _host(parent, np.int32)
    depth = np.zeros(parent.shape[0], np.int32)
    md = C.c_int32()
    check(lib().mig_tree_check(parent.shape[0], _ptr(parent), _ptr(depth), C.byref(md)))
    return depth, md.value


def tree_eval(m: Map, parent, pos, sensor, mode=MODE_MARGINAL, want_counts=False, want_depth=False):
    """mig_tree_eval(_ex) on host arrays; returns dict(abs, marg, yaw[, cnt_abs, cnt_marg, depth])."""
    parent = _host(parent, np.int32)
    pos = _host(pos, np.float32).reshape(-1, 3)
    n = parent.shape[0]
    s = Sensor.of(sensor)
    out = {k: np.zeros(n, np.int32) for k in ("abs", "marg", "yaw")}
    opts = EvalOpts(int(mode), None, None, None)
    if want_counts:
        out["cnt_abs"] = np.zeros((n, s.yaw_bins), np.int32)
        out["cnt_marg"] = np.zeros((n, s.yaw_bins), np.int32)
        opts.counts_abs = out["cnt_abs"].ctypes.data
        opts.counts_marg = out["cnt_marg"].ctypes.data
    if want_depth:
        out["depth"] = np.zeros((n, s.height, s.width), np.uint32)
        opts.depth_buffers = out["depth"].ctypes.data
    check(lib().mig_tree_eval_ex(m.h, n, _ptr(parent), _ptr(pos), C.byref(s), C.byref(opts), _ptr(out["abs"]),
                                 _ptr(out["marg"]), _ptr(out["yaw"])))
    return out


def probe_gather(ctx: Context, buffer_bytes: int, elem_bytes: int = 1) -> float:
    """mig_probe_gather: random independent loads per second from a buffer of buffer_bytes."""
    out = C.c_double()
    check(lib().mig_probe_gather(ctx.h, int(buffer_bytes), int(elem_bytes), C.byref(out)))
    return out.value


def tree_eval_stats(m: Map, parent, pos, sensor):
    """mig_tree_eval_stats: results plus the algorithmic work of the count and render passes."""
    parent = _host(parent, np.int32)
    pos = _host(pos, np.float32).reshape(-1, 3)
    n = parent.shape[0]
    s = Sensor.of(sensor)
    out = {k: np.zeros(n, np.int32) for k in ("abs", "marg", "yaw")}
    st = EvalStats()
    check(lib().mig_tree_eval_stats(m.h, n, _ptr(parent), _ptr(pos), C.byref(s), C.byref(st), _ptr(out["abs"]),
                                    _ptr(out["marg"]), _ptr(out["yaw"])))
    return out, st.as_dict()


def tree_eval_device(m: Map, parent_dev, pos_dev, sensor, max_depth, abs_dev, marg_dev, yaw_dev):
    """mig_tree_eval_device: torch CUDA tensors in and out; enqueued on the context stream."""
    n = int(parent_dev.shape[0])
    s = Sensor.of(sensor)
    check(lib().mig_tree_eval_device(m.h, n, C.c_void_p(parent_dev.data_ptr()), C.c_void_p(pos_dev.data_ptr()),
                                     C.byref(s), int(max_depth), C.c_void_p(abs_dev.data_ptr()),
                                     C.c_void_p(marg_dev.data_ptr()), C.c_void_p(yaw_dev.data_ptr())))


def tree_eval_device_noalloc(m: Map, parent_dev, pos_dev, sensor, max_depth, abs_dev, marg_dev, yaw_dev):
    """mig_tree_eval_device_noalloc: as tree_eval_device, with all scratch in the library's static
    device array (nothing is allocated); calls that overlap on the GPU race."""
    n = int(parent_dev.shape[0])
    s = Sensor.of(sensor)
    check(lib().mig_tree_eval_device_noalloc(m.h, n, C.c_void_p(parent_dev.data_ptr()),
                                             C.c_void_p(pos_dev.data_ptr()), C.byref(s), int(max_depth),
                                             C.c_void_p(abs_dev.data_ptr()), C.c_void_p(marg_dev.data_ptr()),
                                             C.c_void_p(yaw_dev.data_ptr())))


def tree_score(ctx: Context, parent, pos, gain_counts, voxel_size, lam=0.5):
    """mig_tree_score: (cost, objective, best node) of Eq. 3 and Eq. 4 on host arrays."""
    parent = _host(parent, np.int32)
    pos = _host(pos, np.float32).reshape(-1, 3)
    gain = _host(gain_counts, np.int32)
    n = parent.shape[0]
    cost = np.zeros(n, np.float64)
    obj = np.zeros(n, np.float64)
    best = C.c_int32(-1)
    check(lib().mig_tree_score(ctx.h, n, _ptr(parent), _ptr(pos), _ptr(gain), float(voxel_size), float(lam),
                               _ptr(cost), _ptr(obj), C.byref(best)))
    return cost, obj, best.value


def tree_eval_batch(ctx: Context, problems, maps, mode=MODE_MARGINAL):
    """mig_tree_eval_batch over (parent, pos, sensor) problems on the given maps."""
    descs = (TreeDesc * len(problems))()
    keep, outs = [], []
    for i, ((parent, pos, sensor), m) in enumerate(zip(problems, maps)):
        parent = _host(parent, np.int32)
        pos = _host(pos, np.float32).reshape(-1, 3)
        n = parent.shape[0]
        o = {k: np.zeros(n, np.int32) for k in ("abs", "marg", "yaw")}
        keep += [parent, pos]
        outs.append(o)
        descs[i] = TreeDesc(m.h.value, n, parent.ctypes.data, pos.ctypes.data, Sensor.of(sensor), int(mode),
                            o["abs"].ctypes.data, o["marg"].ctypes.data, o["yaw"].ctypes.data)
    check(lib().mig_tree_eval_batch(ctx.h, len(problems), descs))
    return outs


class Server:
    """mig_server: continuous batching of replanning requests (worker thread in the library).

    max_inflight caps the requests evaluated together. Trees that each fill the GPU gain nothing
    from wide interleaving and wait longer, so the default is small (4); raise it for many small
    trees."""

    def __init__(self, ctx: Context, arena_budget_bytes: int, max_inflight: int = 4):
        out = C.c_void_p()
        check(lib().mig_server_create(ctx.h, int(arena_budget_bytes), int(max_inflight), C.byref(out)))
        self.h = out
        self.ctx = ctx
        self._keep = {}

    def submit(self, m: Map, parent, pos, sensor, mode=MODE_MARGINAL):
        """Returns (ticket, outputs dict); the outputs are filled when poll() returns True."""
        parent = _host(parent, np.int32)
        pos = _host(pos, np.float32).reshape(-1, 3)
        n = parent.shape[0]
        out = {k: np.zeros(n, np.int32) for k in ("abs", "marg", "yaw")}
        d = TreeDesc(m.h.value, n, parent.ctypes.data, pos.ctypes.data, Sensor.of(sensor), int(mode),
                     out["abs"].ctypes.data, out["marg"].ctypes.data, out["yaw"].ctypes.data)
        t = C.c_uint64()
        check(lib().mig_server_submit(self.h, C.byref(d), C.byref(t)))
        self._keep[t.value] = out
        return t.value, out

    def map_update(self, m: Map, x0, y0, z0, box):
        b = _host(box, np.uint8)
        dz, dy, dx = b.shape
        check(lib().mig_server_map_update(self.h, m.h, x0, y0, z0, dx, dy, dz, _ptr(b)))

    def poll(self, ticket, timeout_us=0):
        st = lib().mig_server_poll(self.h, C.c_uint64(ticket), int(timeout_us))
        if st == MIG_OK:
            return True
        if st in (MIG_EBUSY, MIG_ETIMEOUT):
            return False
        check(st)

    def memory(self):
        """mig_server_memory: device bytes of requests in flight, of map snapshots, and the peak sum."""
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        check(lib().mig_server_memory(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return {"in_use": a.value, "snapshots": b.value, "peak": c.value}

    def timing(self, ticket):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        check(lib().mig_server_timing(self.h, C.c_uint64(ticket), C.byref(a), C.byref(b), C.byref(c)))
        return {"admit_us": a.value, "start_us": b.value, "done_us": c.value}

    def close(self):
        if getattr(self, "h", None):
            lib().mig_server_destroy(self.h)
            self.h = None


DEFAULT_CANDIDATES = [(4, 16, 4, 1), (8, 8, 4, 1), (4, 8, 4, 1), (8, 16, 4, 1), (16, 16, 4, 1), (4, 16, 3, 1),
                      (4, 16, 4, 0), (8, 8, 4, 0)]


def autotune(ctx: Context, problems, maps, candidates=None, reps=2, cache_path=None):
    """mig_autotune over (tile_w, tile_h, ctas_per_sm, engine) candidates on a sample batch of
    (parent, pos, sensor) problems; the choice is cached in a JSON file keyed by GPU name and the
    sample's ray-grid/yaw signature. Returns (best, {candidate: ms})."""
    import json
    cands = [tuple(c) for c in (candidates or DEFAULT_CANDIDATES)]
    key = None
    if cache_path:
        import torch
        sig = sorted({(int(Sensor.of(s).width), int(Sensor.of(s).height), int(Sensor.of(s).yaw_bins))
                      for (_, _, s) in problems})
        key = f"{torch.cuda.get_device_name(ctx.device)}|{sig}"
        try:
            with open(cache_path) as f:
                hit = json.load(f).get(key)
            if hit:
                ctx.set_tiles(*hit["best"])
                return tuple(hit["best"]), {tuple(map(int, k.split(","))): v for k, v in hit["ms"].items()}
        except (OSError, ValueError):
            pass
    descs = (TreeDesc * len(problems))()
    keep = []
    for i, ((parent, pos, sensor), m) in enumerate(zip(problems, maps)):
        parent = _host(parent, np.int32)
        pos = _host(pos, np.float32).reshape(-1, 3)
        keep += [parent, pos]
        descs[i] = TreeDesc(m.h.value, parent.shape[0], parent.ctypes.data, pos.ctypes.data, Sensor.of(sensor), 0,
                            None, None, None)
    arr = (TileConfig * len(cands))(*[TileConfig(*c) for c in cands])
    ms = (C.c_double * len(cands))()
    best = TileConfig()
    check(lib().mig_autotune(ctx.h, len(problems), descs, len(cands), arr, int(reps), C.byref(best), ms))
    res = (best.tile_w, best.tile_h, best.ctas_per_sm, best.engine)
    times = {c: ms[i] for i, c in enumerate(cands)}
    if cache_path and key:
        try:
            with open(cache_path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
        data[key] = {"best": list(res), "ms": {",".join(map(str, c)): v for c, v in times.items()}}
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1)
    return res, times
