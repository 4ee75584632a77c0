"""GB300 (sm_103a) contour-guided demons registration (CG-DIR, arXiv:1301.0970).

Thin ctypes binding of ``libcgdir.so`` (the C ABI in ``include/cgdir.h``).
Every step of the registration runs in the library's CUDA kernels; this
module only marshals arguments.  PyTorch supplies device memory and the
stream.  There is no CPU fallback: if the library has not been built (see
``paper_1301_0970_gb300.build``) importing the binding's functions raises.

The functions ``cgdir_*`` mirror the C entry points one to one and take raw
pointers; ``Context`` wraps them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_int8, c_longlong, c_size_t, c_uint, c_void_p
from typing import List, Optional, Sequence

from . import build as _build

# ---- constants (include/cgdir.h) ------------------------------------------
CGDIR_OK, CGDIR_EINVAL, CGDIR_ENOMEM, CGDIR_ECUDA, CGDIR_ETIMEDOUT, CGDIR_ECANCELED, CGDIR_EBUSY = range(7)
CGDIR_F32, CGDIR_F16, CGDIR_BF16 = 0, 1, 2
CGDIR_STORAGE_AUTO = -1
CGDIR_HOST, CGDIR_DEVICE = 0, 1
CGDIR_STOP_FIXED, CGDIR_STOP_WINDOW10, CGDIR_STOP_PAPER_LITERAL = 0, 1, 2
CGDIR_COMPOSE, CGDIR_ADDITIVE = 0, 1
CGDIR_REASON_CAP, CGDIR_REASON_CONVERGED, CGDIR_REASON_SKIPPED = 0, 1, 2
CGDIR_MAX_MASKS, CGDIR_MAX_LEVELS = 8, 8


class cgdir_config(ctypes.Structure):
    _fields_ = [("device", c_int), ("stream", c_void_p), ("mem_budget_bytes", c_size_t)]


class cgdir_volume(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("dtype", c_int),
                ("where", c_int), ("data", c_void_p)]


class cgdir_masks(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("where", c_int),
                ("data", POINTER(c_void_p)), ("count", c_int)]


class cgdir_params(ctypes.Structure):
    _fields_ = [("levels", c_int), ("iters", POINTER(c_int)), ("sigma_fluid", c_float),
                ("sigma_diff", c_float), ("lambda_", POINTER(c_float)), ("sign", POINTER(c_int8)),
                ("contour_level_mask", c_uint), ("stop_mode", c_int), ("eps", c_double),
                ("spacing_mm", c_double * 3), ("margin_mm", c_double),
                ("intensity_offset", c_float), ("compose_mode", c_int),
                ("init_dvf", c_void_p), ("init_dvf_where", c_int), ("storage_dtype", c_int)]


class cgdir_level_stats(ctypes.Structure):
    _fields_ = [("level", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("iters_run", c_int), ("stop_reason", c_int), ("hist_len", c_int),
                ("rms_id", POINTER(c_double))]


class cgdir_tuning(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("contour", c_int), ("storage_dtype", c_int),
                ("smooth_variant", c_int), ("smooth_zchunk", c_int), ("force_zchunk", c_int),
                ("smooth_ms", c_float), ("force_ms", c_float), ("default_smooth_ms", c_float),
                ("default_force_ms", c_float), ("force_width", c_int)]


CGDIR_SMOOTH_MARCH, CGDIR_SMOOTH_TILE, CGDIR_SMOOTH_SPLIT, CGDIR_SMOOTH_FUSED, CGDIR_SMOOTH_MARCH32 = 1, 2, 3, 4, 5


class cgdir_kernel_time(ctypes.Structure):
    _fields_ = [("kernel", c_int), ("level", c_int), ("launches", c_longlong), ("total_ms", c_double)]


CGDIR_K_FORCE, CGDIR_K_SMOOTH_DU, CGDIR_K_COMPOSE, CGDIR_K_SMOOTH_U, CGDIR_K_FINALIZE, \
    CGDIR_K_METRIC, CGDIR_K_SETUP, CGDIR_K_LEVEL = range(8)
KERNEL_NAMES = ["force", "smooth_du", "compose", "smooth_u", "finalize", "metric", "setup", "level"]

_SIGNATURES = {
    "cgdir_launch_count": (ctypes.c_ulonglong, []),
    "cgdir_profile": (c_int, [c_void_p, c_uint]),
    "cgdir_profile_read": (c_int, [c_void_p, POINTER(cgdir_kernel_time), c_int]),
    "cgdir_profile_levels": (c_int, [c_void_p, c_uint]),
    "cgdir_default_params": (None, [POINTER(cgdir_params)]),
    "cgdir_create": (c_int, [POINTER(c_void_p), POINTER(cgdir_config)]),
    "cgdir_destroy": (None, [c_void_p]),
    "cgdir_strerror": (ctypes.c_char_p, [c_int]),
    "cgdir_last_error": (ctypes.c_char_p, [c_void_p]),
    "cgdir_mem_in_use": (c_size_t, [c_void_p]),
    "cgdir_sync": (c_int, [c_void_p]),
    "cgdir_register": (c_int, [c_void_p, POINTER(cgdir_volume), POINTER(cgdir_volume),
                               POINTER(cgdir_masks), POINTER(cgdir_masks), POINTER(cgdir_params),
                               c_void_p, c_int, POINTER(cgdir_level_stats)]),
    "cgdir_autotune": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_uint, c_int, c_float]),
    "cgdir_set_autotune": (c_int, [c_void_p, c_int]),
    "cgdir_tuning_read": (c_int, [c_void_p, POINTER(cgdir_tuning), c_int]),
    "cgdir_tuning_load": (c_int, [c_void_p, POINTER(cgdir_tuning), c_int]),
    "cgdir_selftest_wait_timeout": (c_int, [c_void_p, c_int]),
    "cgdir_register_batch": (c_int, [c_void_p, c_int, POINTER(cgdir_volume), POINTER(cgdir_volume),
                                     POINTER(cgdir_masks), POINTER(cgdir_masks), POINTER(cgdir_params),
                                     POINTER(c_void_p), c_int, POINTER(cgdir_level_stats)]),
    "cgdir_set_max_inflight": (c_int, [c_void_p, c_int]),
    "cgdir_submit": (c_int, [c_void_p, POINTER(cgdir_volume), POINTER(cgdir_volume),
                             POINTER(cgdir_masks), POINTER(cgdir_masks), POINTER(cgdir_params),
                             c_void_p, c_int, POINTER(c_longlong)]),
    "cgdir_poll": (c_int, [c_void_p, c_longlong]),
    "cgdir_wait": (c_int, [c_void_p, c_longlong, c_int]),
    "cgdir_release": (c_int, [c_void_p, c_longlong, POINTER(cgdir_level_stats)]),
    "cgdir_cancel": (c_int, [c_void_p, c_longlong]),
    "cgdir_pack_masks": (c_int, [c_void_p, POINTER(c_void_p), c_int, c_size_t, c_void_p]),
    "cgdir_warp": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "cgdir_force": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                            POINTER(c_float), POINTER(c_int8), c_float, c_int, c_void_p, c_int,
                            c_int, c_int, c_void_p, c_void_p, POINTER(c_double)]),
    "cgdir_smooth": (c_int, [c_void_p, c_void_p, c_int, c_float, c_int, c_int, c_int, c_void_p]),
    "cgdir_compose": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_float, c_int, c_int, c_int,
                              c_void_p]),
    "cgdir_smooth_compose": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_float, c_int, c_int, c_int,
                                     c_void_p]),
    "cgdir_iterate": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                              POINTER(c_float), POINTER(c_int8), c_float, c_int, c_float, c_float,
                              c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                              POINTER(c_double)]),
    "cgdir_restrict_image": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "cgdir_restrict_bits": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "cgdir_prolong": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_int,
                              c_void_p]),
    "cgdir_uroi": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, POINTER(c_double),
                           c_double, c_void_p]),
    "cgdir_auto_sign": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                POINTER(c_int8)]),
    "cgdir_rms_id": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int,
                             c_int, POINTER(c_double), POINTER(c_longlong)]),
    "cgdir_rms_id_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                     c_void_p, POINTER(c_double), POINTER(c_longlong)]),
}

_lib = None


def launch_count() -> int:
    """Kernels launched by the CUDA library in this process so far."""
    return int(load().cgdir_launch_count())


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libcgdir.so (building it with nvcc if it is missing or stale).
    Raises if it cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CG-DIR CUDA library missing at {path}; build it with "
                           "`python -m paper_1301_0970_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class CgdirError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [{status}]")
        self.status = status


def _lib_fn(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    return call


# the C entry points, same names, raw arguments
for _name in _SIGNATURES:
    globals()[_name] = _lib_fn(_name)


# --------------------------------------------------------------------------- #
# torch-facing wrapper
# --------------------------------------------------------------------------- #
def _torch():
    import torch
    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _dims(t):
    nz, ny, nx = t.shape[-3:]
    return int(nx), int(ny), int(nz)


def _dtype_code(t) -> int:
    torch = _torch()
    return {torch.float32: CGDIR_F32, torch.float16: CGDIR_F16, torch.bfloat16: CGDIR_BF16}[t.dtype]


def _stats_list(stats, first: int, n: int):
    out = []
    for i in range(first, first + n):
        s = stats[i]
        hist = [s.rms_id[j] for j in range(s.hist_len)] if s.hist_len else []
        out.append({"level": s.level, "shape": (s.nz, s.ny, s.nx), "iters_run": s.iters_run,
                    "stop_reason": s.stop_reason, "rms_id": hist})
    return out


class Request:
    """The C arguments of one registration (Algorithm A), kept alive while it
    runs.  Images are [nz,ny,nx] tensors (CUDA or CPU; float32/16/bf16),
    masks k-long lists (or [k,nz,ny,nx] tensors) of uint8 tensors."""

    def __init__(self, static, moving, static_masks=None, moving_masks=None, *,
                 levels: int = 2, iters: Sequence[int] = (100, 50), sigma_fluid: float = 1.0,
                 sigma_diff: float = 1.0, lam: Optional[Sequence[float]] = None,
                 sign: Optional[Sequence[int]] = None, contour_level_mask: Optional[int] = None,
                 stop_mode: int = CGDIR_STOP_WINDOW10, eps: float = 1e-4,
                 spacing_mm=(1.97, 1.97, 2.5), margin_mm: float = 10.0,
                 intensity_offset: float = 1000.0, compose_mode: int = CGDIR_COMPOSE,
                 init_dvf=None, dvf_out=None, storage_dtype: int = CGDIR_STORAGE_AUTO):
        torch = _torch()
        nx, ny, nz = _dims(static)
        sm = list(static_masks) if static_masks is not None else []
        mm = list(moving_masks) if moving_masks is not None else []
        k = len(sm)
        for m in sm + mm:
            if m.dtype != torch.uint8 or not m.is_contiguous():
                raise ValueError("masks must be contiguous uint8 tensors")
        self.levels = int(levels)
        self.ticket = -1
        self.S = cgdir_volume(nx, ny, nz, _dtype_code(static),
                              CGDIR_DEVICE if static.is_cuda else CGDIR_HOST, c_void_p(_ptr(static)))
        self.M = cgdir_volume(*_dims(moving), _dtype_code(moving),
                              CGDIR_DEVICE if moving.is_cuda else CGDIR_HOST, c_void_p(_ptr(moving)))
        sptr = (c_void_p * max(k, 1))(*[c_void_p(_ptr(m)) for m in sm])
        mptr = (c_void_p * max(len(mm), 1))(*[c_void_p(_ptr(m)) for m in mm])
        self.SM = cgdir_masks(nx, ny, nz, CGDIR_DEVICE if (k and sm[0].is_cuda) else CGDIR_HOST,
                              ctypes.cast(sptr, POINTER(c_void_p)), k)
        self.MM = cgdir_masks(nx, ny, nz, CGDIR_DEVICE if (mm and mm[0].is_cuda) else CGDIR_HOST,
                              ctypes.cast(mptr, POINTER(c_void_p)), len(mm))
        it = (c_int * max(self.levels, 1))(*[int(v) for v in iters])
        p = cgdir_params()
        load().cgdir_default_params(ctypes.byref(p))
        p.levels = self.levels
        p.iters = ctypes.cast(it, POINTER(c_int))
        p.sigma_fluid, p.sigma_diff = sigma_fluid, sigma_diff
        lam_a = (c_float * max(k, 1))(*([float(v) for v in lam] if lam is not None else [1e-3] * k))
        p.lambda_ = ctypes.cast(lam_a, POINTER(c_float))
        sg_a = (c_int8 * max(k, 1))(*([int(v) for v in sign] if sign is not None else [0] * k))
        p.sign = ctypes.cast(sg_a, POINTER(c_int8))
        p.contour_level_mask = (1 << (self.levels - 1)) if contour_level_mask is None else contour_level_mask
        p.stop_mode, p.eps = stop_mode, eps
        p.spacing_mm = (c_double * 3)(*spacing_mm)
        p.margin_mm = margin_mm
        p.intensity_offset = intensity_offset
        p.compose_mode = compose_mode
        p.storage_dtype = storage_dtype
        if init_dvf is not None:
            p.init_dvf = c_void_p(_ptr(init_dvf))
            p.init_dvf_where = CGDIR_DEVICE if init_dvf.is_cuda else CGDIR_HOST
        if dvf_out is None:
            dvf_out = torch.empty((3, nz, ny, nx), dtype=torch.float32,
                                  device=static.device if static.is_cuda else "cpu")
        self.p = p
        self.dvf = dvf_out
        self.dvf_where = CGDIR_DEVICE if dvf_out.is_cuda else CGDIR_HOST
        # everything the C structures point into
        self._keep = (static, moving, sm, mm, sptr, mptr, it, lam_a, sg_a, init_dvf)


class Context:
    """One device + one stream (default: torch's current stream on `device`)."""

    def __init__(self, device: int = 0, stream=None, mem_budget_bytes: int = 0):
        torch = _torch()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        # torch's default stream has handle 0; NULL asks the library for a
        # stream of its own, so name the legacy default stream explicitly
        handle = int(stream.cuda_stream) or 1      # cudaStreamLegacy
        cfg = cgdir_config(device, c_void_p(handle), mem_budget_bytes)
        h = c_void_p()
        st = load().cgdir_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != CGDIR_OK:
            raise CgdirError(st, f"cgdir_create: {load().cgdir_strerror(st).decode()}")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().cgdir_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int, what: str):
        if st != CGDIR_OK:
            lib = load()
            raise CgdirError(st, f"{what}: {lib.cgdir_strerror(st).decode()}: "
                                 f"{lib.cgdir_last_error(self._h).decode()}")

    def sync(self):
        self._check(load().cgdir_sync(self._h), "cgdir_sync")

    def mem_in_use(self) -> int:
        return int(load().cgdir_mem_in_use(self._h))

    def profile(self, kernels: Sequence[int] = (), levels: Optional[Sequence[int]] = None):
        """Time the given kernel classes (CGDIR_K_*) in later registrations,
        at the given pyramid levels (default: all)."""
        mask = 0
        for k in kernels:
            mask |= 1 << int(k)
        self._check(load().cgdir_profile(self._h, mask), "cgdir_profile")
        if levels is not None:
            lm = 0
            for l in levels:
                lm |= 1 << int(l)
            self._check(load().cgdir_profile_levels(self._h, lm), "cgdir_profile_levels")

    def profile_read(self):
        buf = (cgdir_kernel_time * 256)()
        n = load().cgdir_profile_read(self._h, buf, 256)
        if n < 0:
            raise CgdirError(-n, "cgdir_profile_read")
        return [{"kernel": KERNEL_NAMES[buf[i].kernel], "level": buf[i].level,
                 "launches": int(buf[i].launches), "total_ms": float(buf[i].total_ms)}
                for i in range(n)]

    # ---- autotuner -------------------------------------------------------------
    def autotune(self, shape, k: int, levels: int, contour_level_mask: Optional[int] = None,
                 storage_dtype: int = CGDIR_F32, sigma: float = 1.0):
        """Time the kernel configurations of every level shape of a pyramid
        whose finest level is `shape` = (nz, ny, nx) and keep the fastest."""
        nz, ny, nx = shape
        mask = (1 << (levels - 1)) if contour_level_mask is None else contour_level_mask
        self._check(load().cgdir_autotune(self._h, nx, ny, nz, k, levels, mask, storage_dtype, sigma),
                    "cgdir_autotune")
        return self.tuning()

    def set_autotune(self, on: bool = True):
        self._check(load().cgdir_set_autotune(self._h, int(bool(on))), "cgdir_set_autotune")

    def tuning(self):
        n = load().cgdir_tuning_read(self._h, None, 0)
        buf = (cgdir_tuning * max(n, 1))()
        n = load().cgdir_tuning_read(self._h, buf, n)
        names = {CGDIR_SMOOTH_MARCH: "march", CGDIR_SMOOTH_TILE: "tile", CGDIR_SMOOTH_SPLIT: "split",
                 CGDIR_SMOOTH_FUSED: "fused", CGDIR_SMOOTH_MARCH32: "march32"}
        return [{"shape": (b.nz, b.ny, b.nx), "contour": bool(b.contour), "storage_dtype": b.storage_dtype,
                 "smooth": names.get(b.smooth_variant, str(b.smooth_variant)), "smooth_zchunk": b.smooth_zchunk,
                 "force_zchunk": b.force_zchunk, "force_width": b.force_width,
                 "smooth_ms": b.smooth_ms, "force_ms": b.force_ms,
                 "default_smooth_ms": b.default_smooth_ms, "default_force_ms": b.default_force_ms}
                for b in buf[:n]]

    def selftest_wait_timeout(self, limit_us: int = 20000) -> int:
        """Run a kernel whose bounded wait runs out; returns the status
        (CGDIR_ETIMEDOUT when the timeout path works) without raising."""
        return load().cgdir_selftest_wait_timeout(self._h, int(limit_us))

    def load_tuning(self, table):
        """Install a tuning table as tuning() returns it (e.g. saved as JSON by
        an earlier process); registrations of those shapes then use it."""
        codes = {"march": CGDIR_SMOOTH_MARCH, "tile": CGDIR_SMOOTH_TILE, "split": CGDIR_SMOOTH_SPLIT,
                 "fused": CGDIR_SMOOTH_FUSED, "march32": CGDIR_SMOOTH_MARCH32}
        buf = (cgdir_tuning * max(len(table), 1))()
        for b, t in zip(buf, table):
            b.nz, b.ny, b.nx = t["shape"]
            b.contour, b.storage_dtype = int(bool(t["contour"])), int(t["storage_dtype"])
            b.smooth_variant, b.smooth_zchunk = codes[t["smooth"]], int(t["smooth_zchunk"])
            b.force_zchunk = int(t["force_zchunk"])
            b.force_width = int(t.get("force_width", 0))
            b.smooth_ms, b.force_ms = t["smooth_ms"], t["force_ms"]
            b.default_smooth_ms, b.default_force_ms = t["default_smooth_ms"], t["default_force_ms"]
        self._check(load().cgdir_tuning_load(self._h, buf, len(table)), "cgdir_tuning_load")

    # ---- whole registration ------------------------------------------------
    def register(self, static, moving, static_masks=None, moving_masks=None, **kw):
        """Algorithm A on (static, moving) [nz,ny,nx] tensors (CUDA or CPU;
        float32/16/bf16) with k-long lists (or [k,nz,ny,nx] tensors) of uint8
        masks.  Keyword arguments: see `Request`.  Returns (dvf [3,nz,ny,nx]
        float32, stats list coarse->fine)."""
        r = Request(static, moving, static_masks, moving_masks, **kw)
        stats = (cgdir_level_stats * r.levels)()
        st = load().cgdir_register(self._h, ctypes.byref(r.S), ctypes.byref(r.M), ctypes.byref(r.SM),
                                   ctypes.byref(r.MM), ctypes.byref(r.p), c_void_p(_ptr(r.dvf)),
                                   r.dvf_where, stats)
        self._check(st, "cgdir_register")
        return r.dvf, _stats_list(stats, 0, r.levels)

    def register_batch(self, cases):
        """Register every case of `cases` (dicts with static, moving,
        static_masks, moving_masks and any `Request` keyword) in one call: one
        CUDA graph with a concurrent branch per case.  All dvf outputs must be
        on the same side (all CUDA or all host).  Returns a list of
        (dvf, stats) per case."""
        reqs = [Request(c["static"], c["moving"], c.get("static_masks"), c.get("moving_masks"),
                        **{k: v for k, v in c.items()
                           if k not in ("static", "moving", "static_masks", "moving_masks")})
                for c in cases]
        n = len(reqs)
        if n == 0:
            return []
        where = {r.dvf_where for r in reqs}
        if len(where) != 1:
            raise ValueError("register_batch: dvf outputs must all be on the device or all on the host")
        Sa = (cgdir_volume * n)(*[r.S for r in reqs])
        Ma = (cgdir_volume * n)(*[r.M for r in reqs])
        SMa = (cgdir_masks * n)(*[r.SM for r in reqs])
        MMa = (cgdir_masks * n)(*[r.MM for r in reqs])
        Pa = (cgdir_params * n)(*[r.p for r in reqs])
        outs = (c_void_p * n)(*[c_void_p(_ptr(r.dvf)) for r in reqs])
        total = sum(r.levels for r in reqs)
        stats = (cgdir_level_stats * total)()
        st = load().cgdir_register_batch(self._h, n, Sa, Ma, SMa, MMa, Pa, outs, where.pop(), stats)
        self._check(st, "cgdir_register_batch")
        res, o = [], 0
        for r in reqs:
            res.append((r.dvf, _stats_list(stats, o, r.levels)))
            o += r.levels
        return res

    # ---- serving ---------------------------------------------------------------
    def set_max_inflight(self, n: int):
        self._check(load().cgdir_set_max_inflight(self._h, int(n)), "cgdir_set_max_inflight")

    def submit(self, static, moving, static_masks=None, moving_masks=None, **kw) -> "Request":
        """Queue one registration; returns its `Request` at once.  Raises
        CgdirError with code CGDIR_EBUSY when no slot or budget is free."""
        r = Request(static, moving, static_masks, moving_masks, **kw)
        t = c_longlong()
        st = load().cgdir_submit(self._h, ctypes.byref(r.S), ctypes.byref(r.M), ctypes.byref(r.SM),
                                 ctypes.byref(r.MM), ctypes.byref(r.p), c_void_p(_ptr(r.dvf)),
                                 r.dvf_where, ctypes.byref(t))
        self._check(st, "cgdir_submit")
        r.ticket = int(t.value)
        return r

    def poll(self, req: "Request") -> bool:
        st = load().cgdir_poll(self._h, req.ticket)
        if st == CGDIR_EBUSY:
            return False
        self._check(st, "cgdir_poll")
        return True

    def wait(self, req: "Request", timeout_ms: int = -1):
        """Wait for `req`, free its slot and return (dvf, stats).  On timeout
        raises CgdirError(CGDIR_ETIMEDOUT) and the request stays in flight."""
        self._check(load().cgdir_wait(self._h, req.ticket, int(timeout_ms)), "cgdir_wait")
        stats = (cgdir_level_stats * req.levels)()
        self._check(load().cgdir_release(self._h, req.ticket, stats), "cgdir_release")
        req.ticket = -1
        return req.dvf, _stats_list(stats, 0, req.levels)

    def cancel(self, req: "Request"):
        self._check(load().cgdir_cancel(self._h, req.ticket), "cgdir_cancel")
        req.ticket = -1

    # ---- primitives ------------------------------------------------------------
    def pack_masks(self, masks, out=None):
        torch = _torch()
        masks = list(masks)
        n = masks[0].numel() if masks else 0
        if out is None:
            out = torch.empty(masks[0].shape, dtype=torch.uint8, device=masks[0].device)
        ptrs = (c_void_p * max(len(masks), 1))(*[c_void_p(_ptr(m)) for m in masks])
        self._check(load().cgdir_pack_masks(self._h, ptrs, len(masks), n, c_void_p(_ptr(out))),
                    "cgdir_pack_masks")
        return out

    def warp(self, f, u, out=None):
        out = _torch().empty_like(f) if out is None else out
        self._check(load().cgdir_warp(self._h, _ptr(f), _ptr(u), *_dims(f), _ptr(out)), "cgdir_warp")
        return out

    def force(self, I0, T0, mbits, sbits, lam, sign, u, *, offset=1000.0, contour=True, uroi=None,
              du=None, warped=None, want_stats=False):
        torch = _torch()
        k = len(lam)
        du = torch.empty((3,) + tuple(I0.shape), dtype=torch.float32, device=I0.device) if du is None else du
        lam_a = (c_float * max(k, 1))(*[float(v) for v in lam])
        sg_a = (c_int8 * max(k, 1))(*[int(v) for v in sign])
        stats = (c_double * 3)() if want_stats else None
        st = load().cgdir_force(self._h, _ptr(I0), _ptr(T0), _ptr(mbits), _ptr(sbits), _ptr(uroi), k,
                                lam_a, sg_a, offset, int(bool(contour)), _ptr(u), *_dims(I0), _ptr(du),
                                _ptr(warped), stats)
        self._check(st, "cgdir_force")
        return (du, list(stats)) if want_stats else du

    def smooth(self, f, sigma, out=None):
        ncomp = 1 if f.dim() == 3 else int(f.shape[0])
        out = _torch().empty_like(f) if out is None else out
        self._check(load().cgdir_smooth(self._h, _ptr(f), ncomp, sigma, *_dims(f), _ptr(out)), "cgdir_smooth")
        return out

    def compose(self, u, du, mode=CGDIR_COMPOSE, sigma=0.0, out=None):
        out = _torch().empty_like(u) if out is None else out
        self._check(load().cgdir_compose(self._h, _ptr(u), _ptr(du), mode, sigma, *_dims(u), _ptr(out)),
                    "cgdir_compose")
        return out

    def smooth_compose(self, du, u, mode=CGDIR_COMPOSE, sigma=1.0, out=None):
        """Algorithm A steps 2-3: G(du) + u(x + G(du)) (or u + G(du))."""
        out = _torch().empty_like(u) if out is None else out
        self._check(load().cgdir_smooth_compose(self._h, _ptr(du), _ptr(u), mode, sigma, *_dims(u), _ptr(out)),
                    "cgdir_smooth_compose")
        return out

    def iterate(self, I0, T0, mbits, sbits, lam, sign, u, *, offset=1000.0, contour=True, uroi=None,
                sigma_fluid=1.0, sigma_diff=1.0, compose_mode=CGDIR_COMPOSE, out=None, du_out=None,
                want_stats=False):
        k = len(lam)
        out = _torch().empty_like(u) if out is None else out
        lam_a = (c_float * max(k, 1))(*[float(v) for v in lam])
        sg_a = (c_int8 * max(k, 1))(*[int(v) for v in sign])
        stats = (c_double * 3)() if want_stats else None
        st = load().cgdir_iterate(self._h, _ptr(I0), _ptr(T0), _ptr(mbits), _ptr(sbits), _ptr(uroi), k,
                                  lam_a, sg_a, offset, int(bool(contour)), sigma_fluid, sigma_diff,
                                  compose_mode, _ptr(u), *_dims(I0), _ptr(out), _ptr(du_out), stats)
        self._check(st, "cgdir_iterate")
        return (out, list(stats)) if want_stats else out

    def restrict_image(self, f):
        nx, ny, nz = _dims(f)
        out = _torch().empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2), dtype=f.dtype, device=f.device)
        self._check(load().cgdir_restrict_image(self._h, _ptr(f), nx, ny, nz, _ptr(out)), "cgdir_restrict_image")
        return out

    def restrict_bits(self, b):
        nx, ny, nz = _dims(b)
        out = _torch().empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2), dtype=b.dtype, device=b.device)
        self._check(load().cgdir_restrict_bits(self._h, _ptr(b), nx, ny, nz, _ptr(out)), "cgdir_restrict_bits")
        return out

    def prolong(self, uc, fine_shape):
        cx, cy, cz = _dims(uc)
        nz, ny, nx = fine_shape
        out = _torch().empty((3, nz, ny, nx), dtype=uc.dtype, device=uc.device)
        self._check(load().cgdir_prolong(self._h, _ptr(uc), cx, cy, cz, nx, ny, nz, _ptr(out)), "cgdir_prolong")
        return out

    def uroi(self, sbits, k, spacing=(1.97, 1.97, 2.5), margin=10.0):
        nx, ny, nz = _dims(sbits)
        out = _torch().empty_like(sbits)
        sp = (c_double * 3)(*spacing)
        self._check(load().cgdir_uroi(self._h, _ptr(sbits), k, nx, ny, nz, sp, margin, _ptr(out)), "cgdir_uroi")
        return out

    def auto_sign(self, T0, sbits, k) -> List[int]:
        out = (c_int8 * max(k, 1))()
        self._check(load().cgdir_auto_sign(self._h, _ptr(T0), _ptr(sbits), k, *_dims(T0), out),
                    "cgdir_auto_sign")
        return [int(out[i]) for i in range(k)]

    def rms_id(self, I0, T0, u, uroi=None):
        r = c_double()
        c = c_longlong()
        self._check(load().cgdir_rms_id(self._h, _ptr(I0), _ptr(T0), _ptr(u), _ptr(uroi), *_dims(I0),
                                        ctypes.byref(r), ctypes.byref(c)), "cgdir_rms_id")
        return float(r.value), int(c.value)
