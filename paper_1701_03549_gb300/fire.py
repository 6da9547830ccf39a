"""Thin Python binding of libfire's C ABI (include/fire.h).

Argument marshalling only: every step of the simulation path runs in the
CUDA library.  Functions keep the C names (``fire_create``,
``fire_maps_upload``, ``fire_simulate_batch`` ...).  Host arrays are numpy
arrays; device arrays are CUDA ``torch.Tensor`` objects, passed with
``device=True`` (FIRE_DEVICE_PTRS).  PyTorch supplies device memory and the
stream only.

Loading fails loudly when libfire.so has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfire.so")

FIRE_OK = 0
FIRE_EINVAL = -1
FIRE_ENOMEM = -2
FIRE_ECUDA = -3
FIRE_EIGNITION = -4
FIRE_ETIMEOUT = -5
FIRE_ESTEPS = -6

FIRE_DEVICE_PTRS = 1
FIRE_WANT_STEPS = 2
FIRE_SYNC = 4
FIRE_GRAPH = 8
FIRE_CELL_UNIFORM = 16
FIRE_TC_A_MN = 32
FIRE_LONGEST_FIRST = 128
FIRE_TC_B_MN = 64

STATUS_BORDER = 1
STATUS_STEP_CAP = 2
STATUS_BAD_IGNITION = 4
STATUS_TIMEOUT = 8
STATUS_BAD_MAP = 16

STATE_AUTO = 0
STATE_SHARED = 1
STATE_GLOBAL = 2

# cudaStreamLegacy: the legacy default stream of the current context
CUDA_STREAM_LEGACY = 1

FITNESS_PAPER_DELTA = 0
FITNESS_JACCARD = 1

RESULT_FIELDS = ("burnt", "inter", "target", "steps", "status", "trials")
RESULT_DTYPE = np.dtype([(f, "<u4") for f in RESULT_FIELDS])

EXPORTED = (
    "fire_create", "fire_destroy", "fire_last_error", "fire_sync",
    "fire_set_launch", "fire_debug_fail_alloc",
    "fire_maps_upload", "fire_map_free", "fire_map_shape",
    "fire_target_upload", "fire_simulate_batch", "fire_fitness",
    "fire_thresholds", "fire_probabilities", "fire_map_features",
    "fire_screen_selftest", "fire_philox_blocks",
    "fire_simulate_batch_noalloc", "fire_simulate_multi", "fire_autotune",
    "ga_step", "fire_group_mean", "ignition_search", "fire_snap_ignitions",
    "fire_tc_gemm",
    "fire_net_param_count", "fire_net_create", "fire_net_free",
    "fire_net_set_params", "fire_net_get", "fire_net_forward",
    "fire_net_backward", "fire_net_adam", "fire_net_buffer",
    "fire_net_planes", "fire_net_inputs", "fire_net_labels",
    "fire_net_target_frac", "fire_net_screen", "fire_simulate_burnout",
    "fire_wait_selftest",
)


class FireError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfire error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libfire.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with __graft_entry__.build() "
            "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(path)
    vp, i32, u32, u64 = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64
    sig = {
        "fire_create": (i32, [C.POINTER(vp), i32, vp]),
        "fire_destroy": (None, [vp]),
        "fire_last_error": (C.c_char_p, [vp]),
        "fire_sync": (i32, [vp]),
        "fire_set_launch": (i32, [vp, i32, i32, i32, i32]),
        "fire_debug_fail_alloc": (i32, [vp, i32]),
        "fire_maps_upload": (i32, [vp, i32, i32, C.c_float, vp, vp, vp, vp, vp,
                                   u32, C.POINTER(vp)]),
        "fire_map_free": (None, [vp]),
        "fire_map_shape": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
        "fire_target_upload": (i32, [vp, vp, vp, u32]),
        "fire_simulate_batch": (i32, [vp, vp, i32, vp, vp, vp, u32, u32, vp,
                                      vp]),
        "fire_fitness": (i32, [vp, vp, i32, i32, u32, vp]),
        "fire_thresholds": (i32, [vp, vp, vp, u32, vp]),
        "fire_probabilities": (i32, [vp, vp, vp, u32, vp, vp]),
        "fire_map_features": (i32, [vp, vp, u32, vp, vp, vp, vp, vp]),
        "fire_screen_selftest": (i32, [vp, u64, u64, vp, vp]),
        "fire_philox_blocks": (i32, [vp, u64, vp, vp, u32, vp]),
        "fire_simulate_batch_noalloc": (i32, [vp, vp, i32, vp, vp, vp, u32,
                                              u32, vp, vp]),
        "fire_simulate_multi": (i32, [vp, i32, vp, vp, i32, vp, vp, vp, u32,
                                      u32, vp]),
        "fire_autotune": (i32, [vp, i32, vp, vp, i32, vp, vp, vp, u32, vp]),
        "ga_step": (i32, [vp, i32, i32, vp, vp, i32, i32, u64, vp, vp, u32,
                          vp]),
        "fire_group_mean": (i32, [vp, vp, i32, i32, u32, vp]),
        "fire_snap_ignitions": (i32, [vp, vp, i32, i32, i32, i32, vp, i32,
                                      u32, vp]),
        "ignition_search": (i32, [vp, vp, vp, i32, i32, i32, u64, i32,
                                  C.c_double, u32, vp, vp, vp]),
        "fire_tc_gemm": (i32, [vp, i32, i32, i32, vp, vp, i32, u32, vp]),
        "fire_wait_selftest": (i32, [vp]),
        "fire_simulate_burnout": (i32, [vp, vp, i32, vp, vp, vp, vp, u32,
                                        u32, vp, vp]),
        "fire_net_param_count": (C.c_int64, []),
        "fire_net_create": (i32, [vp, i32, i32, C.POINTER(vp)]),
        "fire_net_free": (None, [vp]),
        "fire_net_set_params": (i32, [vp, vp, vp, u32]),
        "fire_net_get": (i32, [vp, vp, i32, u32, vp]),
        "fire_net_forward": (i32, [vp, vp, i32, vp, u32, vp]),
        "fire_net_backward": (i32, [vp, vp, i32, vp, vp, u32, vp]),
        "fire_net_adam": (i32, [vp, vp, C.c_float, u32]),
        "fire_net_buffer": (i32, [vp, vp, i32, i32, i32, u32, vp]),
        "fire_net_planes": (i32, [vp, i32, i32, i32, vp, vp, vp, vp, u32,
                                  vp]),
        "fire_net_inputs": (i32, [vp, i32, i32, i32, i32, vp, vp, vp, u32,
                                  vp]),
        "fire_net_labels": (i32, [vp, vp, i32, i32, i32, vp, vp, u64, u32,
                                  u32, vp, vp]),
        "fire_net_target_frac": (i32, [vp, vp, i32, u32, vp]),
        "fire_net_screen": (i32, [vp, i32, i32, vp, vp, C.c_double, i32,
                                  i32, u32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers

def _is_tensor(a) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(a, torch.Tensor)


def _ptr(a):
    """Address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if _is_tensor(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# torch dtype names accepted for each device-buffer type of fire.h
_F64, _F32, _I32, _U8 = ("float64",), ("float32",), ("int32",), ("uint8",)
_RES = ("int32", "uint32")       # fire_result words (bit patterns)
_SEED = ("int64", "uint64")      # uint64 seeds (bit patterns)
_BF16 = ("bfloat16",)


def _dev(ctx, t, name, dtypes, numel, allow_none=False):
    """Pointer of a device-mode argument, after the checks the library cannot
    make through a plain pointer: a contiguous CUDA tensor on the context's
    device, of one of `dtypes` (torch dtype names), holding exactly `numel`
    elements, the count the call reads or writes.  Any other tensor would be
    accessed past its end; it raises FireError(FIRE_EINVAL) instead."""
    def bad(msg):
        return FireError(FIRE_EINVAL, f"{name}: {msg}")
    if t is None:
        if allow_none:
            return None
        raise bad("a CUDA tensor is required")
    if not _is_tensor(t) or not t.is_cuda:
        raise bad("expected a CUDA tensor")
    if t.device.index != ctx.device:
        raise bad(f"on cuda:{t.device.index}, the context is on "
                  f"cuda:{ctx.device}")
    dt = str(t.dtype).rpartition(".")[2]
    if dt not in dtypes:
        raise bad(f"dtype {dt}, expected {' or '.join(dtypes)}")
    if t.numel() != numel:
        raise bad(f"{t.numel()} elements, expected {numel}")
    if not t.is_contiguous():
        raise bad("tensor must be contiguous")
    return t.data_ptr()


def _rows(ctx, t, name, width):
    """Leading dimension n of a device tensor of n rows of `width` values."""
    if not _is_tensor(t) or t.dim() < 1:
        raise FireError(FIRE_EINVAL, f"{name}: expected a CUDA tensor")
    n = int(t.shape[0])
    if t.numel() != n * width:
        raise FireError(FIRE_EINVAL, f"{name}: expected {width} values per "
                        f"row, got shape {tuple(t.shape)}")
    return n


def _host_plane(a, dtype, H, W, name):
    """A host raster as a C-contiguous (H, W) array of `dtype`."""
    a = _host(a, dtype)
    if a.shape != (H, W):
        raise FireError(FIRE_EINVAL, f"{name}: shape {a.shape}, expected "
                        f"{(H, W)}")
    return a


class Context:
    """A libfire context (fire_create) bound to one device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(
                stream)
            if s == 0:
                # torch's default stream is the legacy default stream; NULL
                # would ask the library for a stream of its own
                s = CUDA_STREAM_LEGACY
        rc = self.lib.fire_create(C.byref(h), int(device), s)
        if rc != FIRE_OK:
            raise FireError(rc, "fire_create failed")
        self.h = h
        self.device = device
        # maps and networks of this context: the library requires them freed
        # before the context, so close() frees the ones still alive
        self._owned = weakref.WeakSet()

    # -- errors
    def check(self, rc):
        if rc != FIRE_OK:
            msg = self.lib.fire_last_error(self.h)
            raise FireError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if self.h:
            for obj in list(self._owned):
                obj.free()
            self.lib.fire_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        return self.check(self.lib.fire_sync(self.h))

    def debug_fail_alloc(self, after: int = 0):
        """fire_debug_fail_alloc: make the buffer growth `after` growths from
        now fail with FIRE_ENOMEM (-1: off)."""
        return self.check(self.lib.fire_debug_fail_alloc(self.h, int(after)))

    def set_launch(self, warps_per_block: int = 0, blocks_per_sm: int = 0,
                   queue_entries: int = 0, state_mode: int = 0):
        return self.check(self.lib.fire_set_launch(
            self.h, warps_per_block, blocks_per_sm, queue_entries, state_mode))

    # -- maps
    def maps_upload(self, veg, elev, slope, aspect, wind, cell_m=30.0,
                    device=False):
        names = ("veg", "elev", "slope", "aspect", "wind")
        if device:
            H, W = veg.shape
            ptrs = [_dev(self, a, nm, _U8 if nm == "veg" else _F32, H * W)
                    for nm, a in zip(names, (veg, elev, slope, aspect, wind))]
            flags = FIRE_DEVICE_PTRS
        else:
            H, W = np.shape(veg)
            arrs = [_host_plane(a, np.uint8 if nm == "veg" else np.float32,
                                H, W, nm)
                    for nm, a in zip(names, (veg, elev, slope, aspect, wind))]
            ptrs = [_ptr(a) for a in arrs]
            flags = 0
        h = C.c_void_p()
        self.check(self.lib.fire_maps_upload(
            self.h, H, W, float(cell_m), *ptrs, flags, C.byref(h)))
        return Map(self, h, H, W)

    def landscape_upload(self, land):
        return self.maps_upload(land.veg, land.elev, land.slope, land.aspect,
                                land.wind, cell_m=land.cell_m)


class Map:
    """A device-resident landscape (fire_maps_upload)."""

    def __init__(self, ctx: Context, h, H: int, W: int):
        self.ctx, self.h, self.H, self.W = ctx, h, H, W
        ctx._owned.add(self)

    def free(self):
        # after the context's close() the map is already freed (h is None)
        if self.h:
            self.ctx.lib.fire_map_free(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.free()
        except Exception:
            pass

    def _sim_args(self, params, ignitions, seeds, out, burn_step, want_steps):
        """Checked device pointers of a batch of n = params rows: params (n,
        5) float64, ignitions (n, 2) int32, seeds (n,) int64 or uint64, out
        (n, 6) int32 or uint32, burn_step (n, H, W) int32 (required with
        want_steps)."""
        ctx = self.ctx
        n = _rows(ctx, params, "params", 5)
        return n, (_dev(ctx, params, "params", _F64, 5 * n),
                   _dev(ctx, ignitions, "ignitions", _I32, 2 * n),
                   _dev(ctx, seeds, "seeds", _SEED, n),
                   _dev(ctx, out, "out", _RES, 6 * n),
                   _dev(ctx, burn_step, "burn_step", _I32,
                        n * self.H * self.W, allow_none=not want_steps))

    def target_upload(self, burnt, device=False):
        if device:
            self.ctx.check(self.ctx.lib.fire_target_upload(
                self.ctx.h, self.h,
                _dev(self.ctx, burnt, "burnt", ("uint8", "bool"),
                     self.H * self.W), FIRE_DEVICE_PTRS))
        else:
            b = _host_plane(np.asarray(burnt) != 0, np.uint8, self.H, self.W,
                            "burnt")
            self.ctx.check(self.ctx.lib.fire_target_upload(
                self.ctx.h, self.h, _ptr(b), 0))

    def simulate_batch(self, params, ignitions, seeds, want_steps=False,
                       max_steps=0, device=False, out=None, burn_step=None,
                       sync=False, cell_uniform=False, longest_first=False):
        """fire_simulate_batch.

        Host mode: params (n, 5) float64, ignitions (n, 2) int32 (row, col),
        seeds (n,) uint64; returns (results structured array, burn_step or
        None).  Device mode: torch CUDA tensors params (n, 5) float64,
        ignitions (n, 2) int32, seeds (n,) int64 (bit pattern of the uint64
        seeds), out (n, 6) int32 (bit pattern of the uint32 results), optional
        burn_step (n, H, W) int32; returns (out, burn_step).
        """
        lib = self.ctx.lib
        flags = FIRE_WANT_STEPS if want_steps else 0
        flags |= FIRE_CELL_UNIFORM if cell_uniform else 0
        flags |= FIRE_LONGEST_FIRST if longest_first else 0
        if device:
            n, (pp, pg, ps, po, pb) = self._sim_args(
                params, ignitions, seeds, out, burn_step, want_steps)
            flags |= FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0)
            self.ctx.check(lib.fire_simulate_batch(
                self.ctx.h, self.h, n, pp, pg, ps, int(max_steps), flags, po,
                pb))
            return out, burn_step
        p = _host(params, np.float64).reshape(-1, 5)
        n = p.shape[0]
        g = _host(ignitions, np.int32).reshape(n, 2)
        s = _host(seeds, np.uint64).reshape(n)
        res = np.zeros(n, RESULT_DTYPE)
        bs = np.zeros((n, self.H, self.W), np.int32) if want_steps else None
        self.ctx.check(lib.fire_simulate_batch(
            self.ctx.h, self.h, n, _ptr(p), _ptr(g), _ptr(s), int(max_steps),
            flags, _ptr(res), _ptr(bs)))
        return res, bs

    def simulate_burnout(self, params, ignitions, seeds, burn_time,
                         want_steps=False, max_steps=0, device=False, out=None,
                         burn_step=None, sync=False):
        """fire_simulate_burnout: as simulate_batch with per-cell burn times
        burn_time (uint8 (H, W); a torch CUDA uint8 tensor in device mode)."""
        lib = self.ctx.lib
        flags = FIRE_WANT_STEPS if want_steps else 0
        if device:
            n, (pp, pg, ps, po, pb) = self._sim_args(
                params, ignitions, seeds, out, burn_step, want_steps)
            pt = _dev(self.ctx, burn_time, "burn_time", _U8, self.H * self.W)
            flags |= FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0)
            self.ctx.check(lib.fire_simulate_burnout(
                self.ctx.h, self.h, n, pp, pg, ps, pt, int(max_steps), flags,
                po, pb))
            return out, burn_step
        p = _host(params, np.float64).reshape(-1, 5)
        n = p.shape[0]
        g = _host(ignitions, np.int32).reshape(n, 2)
        s = _host(seeds, np.uint64).reshape(n)
        bt = _host(burn_time, np.uint8).reshape(self.H, self.W)
        res = np.zeros(n, RESULT_DTYPE)
        bs = np.zeros((n, self.H, self.W), np.int32) if want_steps else None
        self.ctx.check(lib.fire_simulate_burnout(
            self.ctx.h, self.h, n, _ptr(p), _ptr(g), _ptr(s), _ptr(bt),
            int(max_steps), flags, _ptr(res), _ptr(bs)))
        return res, bs

    def simulate_batch_noalloc(self, params, ignitions, seeds, out,
                               burn_step=None, want_steps=False, max_steps=0,
                               sync=True):
        """fire_simulate_batch_noalloc: device tensors only (as the device
        mode of simulate_batch); the library allocates nothing."""
        flags = (FIRE_WANT_STEPS if want_steps else 0) | FIRE_DEVICE_PTRS
        flags |= FIRE_SYNC if sync else 0
        n, (pp, pg, ps, po, pb) = self._sim_args(
            params, ignitions, seeds, out, burn_step, want_steps)
        self.ctx.check(self.ctx.lib.fire_simulate_batch_noalloc(
            self.ctx.h, self.h, n, pp, pg, ps, int(max_steps), flags, po, pb))
        return out, burn_step

    def thresholds(self, beta):
        b = _host(beta, np.float64).reshape(5)
        out = np.zeros((8, self.H, self.W), np.int64)
        self.ctx.check(self.ctx.lib.fire_thresholds(
            self.ctx.h, self.h, _ptr(b), 0, _ptr(out)))
        return out

    def probabilities(self, beta):
        b = _host(beta, np.float64).reshape(5)
        p32 = np.zeros((8, self.H, self.W), np.float32)
        p64 = np.zeros((8, self.H, self.W), np.float64)
        self.ctx.check(self.ctx.lib.fire_probabilities(
            self.ctx.h, self.h, _ptr(b), 0, _ptr(p32), _ptr(p64)))
        return p32, p64

    def features(self):
        H, W = self.H, self.W
        psi = np.zeros((H, W), np.float32)
        sig = np.zeros((H, W), np.float32)
        cw = np.zeros((H, W), np.float32)
        sw = np.zeros((H, W), np.float32)
        fl = np.zeros((H, W), np.uint16)
        self.ctx.check(self.ctx.lib.fire_map_features(
            self.ctx.h, self.h, 0, _ptr(psi), _ptr(sig), _ptr(cw), _ptr(sw),
            _ptr(fl)))
        return dict(psi=psi, sig=sig, cw=cw, sw=sw, flags=fl)


# ---------------------------------------------------------------------------
# functions with the C names

def fire_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def fire_maps_upload(ctx: Context, veg, elev, slope, aspect, wind,
                     cell_m=30.0, device=False) -> Map:
    return ctx.maps_upload(veg, elev, slope, aspect, wind, cell_m, device)


def fire_target_upload(ctx: Context, m: Map, burnt, device=False):
    return m.target_upload(burnt, device)


def fire_simulate_batch(ctx: Context, m: Map, params, ignitions, seeds,
                        **kw):
    return m.simulate_batch(params, ignitions, seeds, **kw)


class FireLaunch(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("queue_entries", C.c_int32), ("state_mode", C.c_int32),
                ("ms", C.c_float)]


def _map_handles(maps):
    arr = (C.c_void_p * len(maps))(*[m.h.value if hasattr(m.h, "value")
                                     else m.h for m in maps])
    return arr


def fire_simulate_multi(ctx: Context, maps, map_of_sim, params, ignitions,
                        seeds, max_steps=0, device=False, out=None,
                        graph=False, sync=False, cell_uniform=False):
    """Uneven batch over several maps (see fire_simulate_multi in fire.h).

    Host mode: numpy inputs, returns the structured results.  Device mode:
    torch CUDA tensors (map_of_sim int32, others as in simulate_batch) and a
    preallocated `out` (n, 6) int32; returns `out`."""
    lib = ctx.lib
    handles = _map_handles(maps)
    if device:
        n = _rows(ctx, params, "params", 5)
        ptrs = (_dev(ctx, map_of_sim, "map_of_sim", _I32, n),
                _dev(ctx, params, "params", _F64, 5 * n),
                _dev(ctx, ignitions, "ignitions", _I32, 2 * n),
                _dev(ctx, seeds, "seeds", _SEED, n),
                _dev(ctx, out, "out", _RES, 6 * n))
        flags = FIRE_DEVICE_PTRS | (FIRE_GRAPH if graph else 0)
        flags |= FIRE_SYNC if sync else 0
        flags |= FIRE_CELL_UNIFORM if cell_uniform else 0
        ctx.check(lib.fire_simulate_multi(
            ctx.h, len(maps), handles, ptrs[0], n, *ptrs[1:4],
            int(max_steps), flags, ptrs[4]))
        return out
    p = _host(params, np.float64).reshape(-1, 5)
    n = p.shape[0]
    mi = _host(map_of_sim, np.int32).reshape(n)
    g = _host(ignitions, np.int32).reshape(n, 2)
    s = _host(seeds, np.uint64).reshape(n)
    res = np.zeros(n, RESULT_DTYPE)
    ctx.check(lib.fire_simulate_multi(
        ctx.h, len(maps), handles, _ptr(mi), n, _ptr(p), _ptr(g), _ptr(s),
        int(max_steps), FIRE_CELL_UNIFORM if cell_uniform else 0, _ptr(res)))
    return res


def fire_autotune(ctx: Context, maps, map_of_sim, params, ignitions, seeds,
                  device=False, longest_first=False):
    """Pick and record the fastest launch shape for this batch (timed in
    longest-first order with longest_first, one map only); returns it as a
    dict (warps_per_block, blocks_per_sm, queue_entries, state_mode, ms)."""
    lib = ctx.lib
    handles = _map_handles(maps)
    best = FireLaunch()
    lpt = FIRE_LONGEST_FIRST if longest_first else 0
    if device:
        n = _rows(ctx, params, "params", 5)
        ctx.check(lib.fire_autotune(
            ctx.h, len(maps), handles,
            _dev(ctx, map_of_sim, "map_of_sim", _I32, n, allow_none=True), n,
            _dev(ctx, params, "params", _F64, 5 * n),
            _dev(ctx, ignitions, "ignitions", _I32, 2 * n),
            _dev(ctx, seeds, "seeds", _SEED, n), FIRE_DEVICE_PTRS | lpt,
            C.byref(best)))
    else:
        p = _host(params, np.float64).reshape(-1, 5)
        n = p.shape[0]
        mi = (None if map_of_sim is None
              else _host(map_of_sim, np.int32).reshape(n))
        g = _host(ignitions, np.int32).reshape(n, 2)
        s = _host(seeds, np.uint64).reshape(n)
        ctx.check(lib.fire_autotune(
            ctx.h, len(maps), handles, _ptr(mi), n, _ptr(p), _ptr(g), _ptr(s),
            lpt, C.byref(best)))
    return {f: getattr(best, f) for f, _ in FireLaunch._fields_}


def ga_step(ctx: Context, genes, fitness, generation, total_gens, ga_seed,
            lo, hi, device=False, out=None):
    """One GA generation (Appendix B).  Host mode: numpy in/out.  Device mode:
    torch CUDA float64 tensors (genes (P, G), fitness (P,), lo, hi (G,)) and a
    preallocated `out` like genes."""
    lib = ctx.lib
    if device:
        if not _is_tensor(genes) or genes.dim() != 2:
            raise FireError(FIRE_EINVAL, "genes: expected a (P, G) tensor")
        P, G = int(genes.shape[0]), int(genes.shape[1])
        ctx.check(lib.ga_step(ctx.h, P, G,
                              _dev(ctx, genes, "genes", _F64, P * G),
                              _dev(ctx, fitness, "fitness", _F64, P),
                              int(generation), int(total_gens), int(ga_seed),
                              _dev(ctx, lo, "lo", _F64, G),
                              _dev(ctx, hi, "hi", _F64, G), FIRE_DEVICE_PTRS,
                              _dev(ctx, out, "out", _F64, P * G)))
        return out
    g = _host(genes, np.float64)
    P, G = g.shape
    f = _host(fitness, np.float64).reshape(P)
    l = _host(lo, np.float64).reshape(G)
    h = _host(hi, np.float64).reshape(G)
    o = np.zeros_like(g)
    ctx.check(lib.ga_step(ctx.h, P, G, _ptr(g), _ptr(f), int(generation),
                          int(total_gens), int(ga_seed), _ptr(l), _ptr(h), 0,
                          _ptr(o)))
    return o


def ignition_search(ctx: Context, m: Map, beta, lat_h, lat_w, reps, seed,
                    kind=FITNESS_PAPER_DELTA, cutoff=1.5):
    """Lattice ignition search on the map's target (see fire.h); returns
    (fitness map (lat_h, lat_w), cells (lat_h, lat_w, 2), [x mean, x sd,
    y mean, y sd])."""
    b = _host(beta, np.float64).reshape(5)
    fm = np.zeros((lat_h, lat_w), np.float64)
    cells = np.zeros((lat_h, lat_w, 2), np.int32)
    xy = np.zeros(4, np.float64)
    ctx.check(ctx.lib.ignition_search(ctx.h, m.h, _ptr(b), int(lat_h),
                                      int(lat_w), int(reps), int(seed),
                                      int(kind), float(cutoff), 0, _ptr(fm),
                                      _ptr(cells), _ptr(xy)))
    return fm, cells, xy


def fire_snap_ignitions(ctx: Context, m: Map, genes, gx: int, gy: int,
                        reps: int = 1, device=False, out=None):
    """Ignition cells of a population whose genes gx (x = column) and gy
    (y = row) hold the ignition point: the burnable target cell nearest to
    each clamped, rounded point, repeated `reps` times per individual.
    Host mode: numpy genes (n, G); returns (n * reps, 2) int32 (row, col).
    Device mode: torch CUDA float64 genes (n, G) and a preallocated int32
    `out` (n * reps, 2); returns `out`."""
    lib = ctx.lib
    if device:
        n = int(genes.shape[0])
        G = int(genes.shape[1]) if genes.dim() == 2 else 0
        ctx.check(lib.fire_snap_ignitions(
            ctx.h, m.h, n, G, int(gx), int(gy),
            _dev(ctx, genes, "genes", _F64, n * G), int(reps),
            FIRE_DEVICE_PTRS, _dev(ctx, out, "out", _I32, 2 * n * int(reps))))
        return out
    g = _host(genes, np.float64)
    if g.ndim != 2:
        raise FireError(FIRE_EINVAL, "genes: expected (n, G)")
    n, G = g.shape
    o = np.zeros((n * int(reps), 2), np.int32)
    ctx.check(lib.fire_snap_ignitions(ctx.h, m.h, n, G, int(gx), int(gy),
                                      _ptr(g), int(reps), 0, _ptr(o)))
    return o


def fire_group_mean(ctx: Context, values, per_group, device=False, out=None):
    lib = ctx.lib
    if device:
        nv = int(values.numel()) if _is_tensor(values) else -1
        if per_group <= 0 or nv % int(per_group):
            raise FireError(FIRE_EINVAL, f"values: {nv} values are not whole "
                            f"groups of {per_group}")
        groups = nv // int(per_group)
        ctx.check(lib.fire_group_mean(ctx.h,
                                      _dev(ctx, values, "values", _F64, nv),
                                      groups, int(per_group), FIRE_DEVICE_PTRS,
                                      _dev(ctx, out, "out", _F64, groups)))
        return out
    v = _host(values, np.float64).ravel()
    groups = v.size // int(per_group)
    o = np.zeros(groups, np.float64)
    ctx.check(lib.fire_group_mean(ctx.h, _ptr(v), groups, int(per_group), 0,
                                  _ptr(o)))
    return o


def fire_fitness(ctx: Context, results, kind=FITNESS_PAPER_DELTA,
                 device=False, out=None):
    lib = ctx.lib
    if device:
        n = _rows(ctx, results, "results", 6)
        ctx.check(lib.fire_fitness(ctx.h,
                                   _dev(ctx, results, "results", _RES, 6 * n),
                                   n, int(kind), FIRE_DEVICE_PTRS,
                                   _dev(ctx, out, "out", _F64, n)))
        return out
    r = np.ascontiguousarray(results, RESULT_DTYPE)
    o = np.zeros(r.shape[0], np.float64)
    ctx.check(lib.fire_fitness(ctx.h, _ptr(r), r.shape[0], int(kind), 0,
                               _ptr(o)))
    return o


def fire_thresholds(ctx: Context, m: Map, beta):
    return m.thresholds(beta)


def fire_probabilities(ctx: Context, m: Map, beta):
    return m.probabilities(beta)


def fire_map_features(ctx: Context, m: Map):
    return m.features()


def fire_screen_selftest(ctx: Context, n: int, seed: int):
    counts = np.zeros(3, np.uint64)
    mx = np.zeros(1, np.float64)
    ctx.check(ctx.lib.fire_screen_selftest(ctx.h, int(n), int(seed),
                                           _ptr(counts), _ptr(mx)))
    return dict(cases=int(counts[0]), fallbacks=int(counts[1]),
                flips=int(counts[2]), max_err_ratio=float(mx[0]))


def fire_philox_blocks(ctx: Context, n: int, ctr, key):
    c = _host(ctr, np.uint32).reshape(4)
    k = _host(key, np.uint32).reshape(2)
    out = np.zeros((n, 4), np.uint32)
    ctx.check(ctx.lib.fire_philox_blocks(ctx.h, int(n), _ptr(c), _ptr(k), 0,
                                         _ptr(out)))
    return out


def results_view(out_tensor) -> np.ndarray:
    """Device results tensor (n, 6) int32 -> host structured array."""
    a = out_tensor.detach().cpu().numpy().astype(np.int32, copy=False)
    return a.view(np.uint32).reshape(-1, 6).copy().view(RESULT_DTYPE).reshape(-1)


def fire_tc_gemm(ctx: Context, A, B, M: int, N: int, K: int, out,
                 a_mn: bool = False, b_mn: bool = False, ksplit: int = 1,
                 sync: bool = True):
    """fire_tc_gemm on device tensors: A, B bfloat16 (A[M, K] or, a_mn,
    A[K, M]; B[N, K] or, b_mn, B[K, N]); out float32 [M, N]."""
    flags = FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0)
    flags |= (FIRE_TC_A_MN if a_mn else 0) | (FIRE_TC_B_MN if b_mn else 0)
    M, N, K = int(M), int(N), int(K)
    ctx.check(ctx.lib.fire_tc_gemm(ctx.h, M, N, K,
                                   _dev(ctx, A, "A", _BF16, M * K),
                                   _dev(ctx, B, "B", _BF16, N * K),
                                   int(ksplit), flags,
                                   _dev(ctx, out, "out", _F32, M * N)))
    return out


def fire_wait_selftest(ctx: Context) -> int:
    """Run the device-side timeout self-check; returns the library's code
    (FIRE_ETIMEOUT when the timeout path works) instead of raising it."""
    return int(ctx.lib.fire_wait_selftest(ctx.h))


# ---------------------------------------------------------------------------
# learned surrogate (fire_net_*); device tensors throughout

NET_CIN = 16
NET_C = 128
NET_LAYERS = 8
NET_PARAMS, NET_GRAD, NET_ADAM_M, NET_ADAM_V = 0, 1, 2, 3
BUF_ACT, BUF_DZ, BUF_PROB = 0, 1, 2


def fire_net_param_count() -> int:
    return int(load().fire_net_param_count())


class Net:
    """fire_net: the surrogate network of one context (S x S inputs,
    batches of up to max_batch samples)."""

    def __init__(self, ctx: Context, S: int, max_batch: int):
        self.ctx, self.S, self.max_batch = ctx, int(S), int(max_batch)
        h = C.c_void_p()
        ctx.check(ctx.lib.fire_net_create(ctx.h, self.S, self.max_batch,
                                          C.byref(h)))
        self.h = h
        self.P = fire_net_param_count()
        ctx._owned.add(self)

    def free(self):
        if self.h:
            self.ctx.lib.fire_net_free(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.free()
        except Exception:
            pass

    def set_params(self, theta):
        """theta: float32 numpy array or CUDA tensor of param_count."""
        if _is_tensor(theta):
            self.ctx.check(self.ctx.lib.fire_net_set_params(
                self.ctx.h, self.h, _dev(self.ctx, theta, "theta", _F32,
                                         self.P), FIRE_DEVICE_PTRS))
        else:
            t = _host(theta, np.float32).ravel()
            if t.size != self.P:
                raise FireError(FIRE_EINVAL, f"theta: {t.size} values, "
                                f"expected {self.P}")
            self.ctx.check(self.ctx.lib.fire_net_set_params(
                self.ctx.h, self.h, _ptr(t), 0))

    def get(self, which=NET_PARAMS) -> np.ndarray:
        out = np.zeros(self.P, np.float32)
        self.ctx.check(self.ctx.lib.fire_net_get(self.ctx.h, self.h,
                                                 int(which), 0, _ptr(out)))
        return out

    def _x(self, x):
        """Sample count and pointer of inputs x (n, S, S, 16) bfloat16."""
        n = _rows(self.ctx, x, "x", self.S * self.S * NET_CIN)
        return n, _dev(self.ctx, x, "x", _BF16, n * self.S * self.S * NET_CIN)

    def forward(self, x, prob, sync=False):
        n, px = self._x(x)
        self.ctx.check(self.ctx.lib.fire_net_forward(
            self.ctx.h, self.h, n, px,
            FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0),
            _dev(self.ctx, prob, "prob", _F32, n * self.S * self.S)))
        return prob

    def backward(self, x, target, loss=None, sync=False):
        n, px = self._x(x)
        self.ctx.check(self.ctx.lib.fire_net_backward(
            self.ctx.h, self.h, n, px,
            _dev(self.ctx, target, "target", _F32, n * self.S * self.S),
            FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0),
            _dev(self.ctx, loss, "loss", _F64, 1, allow_none=True)))
        return loss

    def adam(self, lr: float, sync=False):
        self.ctx.check(self.ctx.lib.fire_net_adam(
            self.ctx.h, self.h, float(lr), FIRE_SYNC if sync else 0))

    def buffer(self, which, layer, n, out):
        px = int(n) * self.S * self.S
        if which == BUF_PROB:
            po = _dev(self.ctx, out, "out", _F32, px)
        else:
            po = _dev(self.ctx, out, "out", _BF16, px * NET_C)
        self.ctx.check(self.ctx.lib.fire_net_buffer(
            self.ctx.h, self.h, int(which), int(layer), int(n),
            FIRE_DEVICE_PTRS, po))
        return out


def fire_net_planes(ctx: Context, S: int, veg, slope, aspect, wind, out,
                    sync=False):
    H, W = int(veg.shape[0]), int(veg.shape[1])
    S = int(S)
    ctx.check(ctx.lib.fire_net_planes(
        ctx.h, H, W, S, _dev(ctx, veg, "veg", _U8, H * W),
        _dev(ctx, slope, "slope", _F32, H * W),
        _dev(ctx, aspect, "aspect", _F32, H * W),
        _dev(ctx, wind, "wind", _F32, H * W),
        FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0),
        _dev(ctx, out, "out", _F32, S * S * 10)))
    return out


def fire_net_inputs(ctx: Context, S: int, H: int, W: int, planes, params,
                    ign, out, sync=False):
    n = _rows(ctx, params, "params", 5)
    S = int(S)
    ctx.check(ctx.lib.fire_net_inputs(
        ctx.h, S, int(H), int(W), n,
        _dev(ctx, planes, "planes", _F32, S * S * 10),
        _dev(ctx, params, "params", _F64, 5 * n),
        _dev(ctx, ign, "ign", _I32, 2 * n),
        FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0),
        _dev(ctx, out, "out", _BF16, n * S * S * NET_CIN)))
    return out


def fire_net_labels(ctx: Context, m: Map, S: int, params, ign, reps: int,
                    seed: int, labels, results=None, max_steps=0,
                    cell_uniform=False, sync=False):
    groups = _rows(ctx, params, "params", 5)
    S, reps = int(S), int(reps)
    flags = FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0)
    flags |= FIRE_CELL_UNIFORM if cell_uniform else 0
    ctx.check(ctx.lib.fire_net_labels(
        ctx.h, m.h, S, groups, reps,
        _dev(ctx, params, "params", _F64, 5 * groups),
        _dev(ctx, ign, "ign", _I32, 2 * groups),
        int(seed), int(max_steps), flags,
        _dev(ctx, labels, "labels", _F32, groups * S * S),
        _dev(ctx, results, "results", _RES, 6 * groups * max(reps, 0),
             allow_none=True)))
    return labels


def fire_net_target_frac(ctx: Context, m: Map, S: int, out, sync=False):
    S = int(S)
    ctx.check(ctx.lib.fire_net_target_frac(
        ctx.h, m.h, S, FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0),
        _dev(ctx, out, "out", _F32, S * S)))
    return out


def fire_net_screen(ctx: Context, S: int, prob, target_frac, cells: float,
                    kind: int, keep: int, pred, keep_idx=None, sync=False):
    S = int(S)
    n = _rows(ctx, prob, "prob", S * S)
    ctx.check(ctx.lib.fire_net_screen(
        ctx.h, S, n, _dev(ctx, prob, "prob", _F32, n * S * S),
        _dev(ctx, target_frac, "target_frac", _F32, S * S), float(cells),
        int(kind), int(keep), FIRE_DEVICE_PTRS | (FIRE_SYNC if sync else 0),
        _dev(ctx, pred, "pred", _F64, n),
        _dev(ctx, keep_idx, "keep_idx", _I32, max(int(keep), 0),
             allow_none=True)))
    return pred, keep_idx
