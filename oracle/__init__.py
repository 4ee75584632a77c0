"""FP64 CPU oracle of contour-guided demons registration (CG-DIR).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It is the plain, slow restatement of the paper's method that the
CUDA library is checked against; the library never calls it and shares no
code with it.  The arithmetic lives in ``cgdir_oracle.c`` (plain C, FP64,
one loop nest per step of Algorithm A, Sec. 2.2); this module only compiles
it with gcc and marshals NumPy arrays.

Pins (tests/test_oracle_*.py) tie each function to the paper and to
mathematics rather than to itself: closed forms, brute force on tiny inputs,
a library distance transform for the UROI, a direct minimisation of Eq. 6 for
the force, recovery of a known deformation for the whole registration.
Parity is unpinned only for the paper's clinical accuracy tables (their data
is not available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgdir_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcgdir_oracle.so")
_lock = threading.Lock()
_lib = None

STOP_FIXED, STOP_WINDOW10, STOP_PAPER_LITERAL = 0, 1, 2
COMPOSE, ADDITIVE = 0, 1
REASON_CAP, REASON_CONVERGED, REASON_SKIPPED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fno-fast-math",
            "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB)
            _lib.oracle_rms_id.restype = ctypes.c_double
            _lib.oracle_gauss_radius.restype = ctypes.c_int
            _lib.oracle_gauss_radius.argtypes = [ctypes.c_double]
            _lib.oracle_gauss_taps.argtypes = [ctypes.c_double, ctypes.c_void_p]
        return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a) != 0, dtype=np.uint8)


def _p(a) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _dims(vol):
    nz, ny, nx = vol.shape[-3:]
    return int(nx), int(ny), int(nz)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------------- #
# primitives
# --------------------------------------------------------------------------- #
def warp(f, u) -> np.ndarray:
    """f(x + u(x)), trilinear, clamped (kernel 4)."""
    f, u = _d(f), _d(u)
    out = np.empty_like(f)
    _load().oracle_warp(_p(f), _p(u), *_dims(f), _p(out))
    return out


def gradient(f) -> np.ndarray:
    """Central differences with clamped indices, [3][...] (kernel 2)."""
    f = _d(f)
    g = np.empty((3,) + f.shape)
    _load().oracle_gradient(_p(f), *_dims(f), _p(g))
    return g


def gauss_radius(sigma: float) -> int:
    return int(_load().oracle_gauss_radius(float(sigma)))


def gauss_taps(sigma: float) -> np.ndarray:
    r = gauss_radius(sigma)
    t = np.empty(2 * r + 1)
    _load().oracle_gauss_taps(ctypes.c_double(sigma), _p(t))
    return t


def gauss(f, sigma: float) -> np.ndarray:
    """Separable Gaussian, x then y then z, clamp-to-edge (kernel 1)."""
    f = _d(f)
    out = np.empty_like(f)
    _load().oracle_gauss(_p(f), *_dims(f), ctypes.c_double(sigma), _p(out))
    return out


def gauss_field(u, sigma: float) -> np.ndarray:
    u = _d(u)
    out = np.empty_like(u)
    _load().oracle_gauss_field(_p(u), *_dims(u), ctypes.c_double(sigma), _p(out))
    return out


def compose(u, du, mode: int = COMPOSE) -> np.ndarray:
    """u o (Id + du) (Algorithm A step 3); mode ADDITIVE gives u + du."""
    u, du = _d(u), _d(du)
    out = np.empty_like(u)
    _load().oracle_compose(_p(u), _p(du), *_dims(u), ctypes.c_int(mode), _p(out))
    return out


def _masks(masks, shape):
    if masks is None or len(masks) == 0:
        return np.zeros((0,) + tuple(shape), np.uint8), 0
    m = _u8(masks)
    return m, int(m.shape[0])


def force(I0, T0, moving_masks, static_masks, lam: Sequence[float], sign: Sequence[int],
          u=None, offset: float = 1000.0, contour: bool = True, return_warped=False):
    """du = v n with v from Eq. 7 (kernels 2 and 3)."""
    I0, T0 = _d(I0), _d(T0)
    mm, k = _masks(moving_masks, I0.shape)
    sm, _ = _masks(static_masks, I0.shape)
    u = np.zeros((3,) + I0.shape) if u is None else _d(u)
    lam_a = _d(list(lam) if k else [0.0])
    sg = np.ascontiguousarray(list(sign) if k else [1], dtype=np.int32)
    du = np.empty((3,) + I0.shape)
    warped = np.empty_like(I0) if return_warped else None
    _load().oracle_force(_p(I0), _p(T0), _p(mm), _p(sm), ctypes.c_int(k), _p(lam_a), _p(sg),
                         ctypes.c_double(offset), ctypes.c_int(int(bool(contour))), _p(u),
                         *_dims(I0), _p(du), _p(warped))
    return (du, warped) if return_warped else du


def restrict_image(f) -> np.ndarray:
    f = _d(f)
    nx, ny, nz = _dims(f)
    out = np.empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2))
    _load().oracle_restrict_image(_p(f), nx, ny, nz, _p(out))
    return out


def restrict_mask(m) -> np.ndarray:
    m = _u8(m)
    nx, ny, nz = _dims(m)
    out = np.empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2), np.uint8)
    _load().oracle_restrict_mask(_p(m), nx, ny, nz, _p(out))
    return out


def prolong(uc, fine_shape) -> np.ndarray:
    uc = _d(uc)
    cx, cy, cz = _dims(uc)
    nz, ny, nx = fine_shape
    out = np.empty((3, nz, ny, nx))
    _load().oracle_prolong(_p(uc), cx, cy, cz, nx, ny, nz, _p(out))
    return out


def uroi(static_masks, shape, spacing=(1.97, 1.97, 2.5), margin: float = 10.0) -> np.ndarray:
    sm, k = _masks(static_masks, shape)
    nz, ny, nx = shape
    out = np.empty(shape, np.uint8)
    sp = _d(spacing)
    _load().oracle_uroi(_p(sm), ctypes.c_int(k), nx, ny, nz, _p(sp), ctypes.c_double(margin), _p(out))
    return out


def auto_sign(T0, static_masks) -> list:
    T0 = _d(T0)
    sm, k = _masks(static_masks, T0.shape)
    out = np.zeros(max(k, 1), np.int32)
    if k:
        _load().oracle_auto_sign(_p(T0), _p(sm), ctypes.c_int(k), *_dims(T0), _p(out))
    return [int(s) for s in out[:k]]


def rms_id(warped, T0, uroi_map):
    warped, T0 = _d(warped), _d(T0)
    ur = _u8(uroi_map)
    cnt = ctypes.c_long(0)
    v = _load().oracle_rms_id(_p(warped), _p(T0), _p(ur), *_dims(T0), ctypes.byref(cnt))
    return float(v), int(cnt.value)


def stop_test(history: Sequence[float], n: int, mode: int, eps: float = 1e-4) -> bool:
    h = _d(history)
    return bool(_load().oracle_stop_test(_p(h), ctypes.c_int(n), ctypes.c_int(mode),
                                         ctypes.c_double(eps)))


def step(I0, T0, moving_masks, static_masks, lam, sign, u, offset=1000.0, contour=True,
         sigma_fluid=1.0, sigma_diff=1.0, compose_mode=COMPOSE, return_du=False):
    """One iteration, Algorithm A steps 1-4."""
    I0, T0, u = _d(I0), _d(T0), _d(u)
    mm, k = _masks(moving_masks, I0.shape)
    sm, _ = _masks(static_masks, I0.shape)
    lam_a = _d(list(lam) if k else [0.0])
    sg = np.ascontiguousarray(list(sign) if k else [1], dtype=np.int32)
    out = np.empty_like(u)
    du = np.empty_like(u) if return_du else None
    _load().oracle_step(_p(I0), _p(T0), _p(mm), _p(sm), ctypes.c_int(k), _p(lam_a), _p(sg),
                        ctypes.c_double(offset), ctypes.c_int(int(bool(contour))),
                        ctypes.c_double(sigma_fluid), ctypes.c_double(sigma_diff),
                        ctypes.c_int(compose_mode), _p(u), *_dims(I0), _p(out), _p(du))
    return (out, du) if return_du else out


def register(static, moving, static_masks, moving_masks, levels: int = 2,
             iters: Sequence[int] = (100, 50), sigma_fluid: float = 1.0,
             sigma_diff: float = 1.0, lam: Optional[Sequence[float]] = None,
             sign: Optional[Sequence[int]] = None, contour_mask: Optional[int] = None,
             stop_mode: int = STOP_FIXED, eps: float = 1e-4,
             spacing=(1.97, 1.97, 2.5), margin: float = 10.0, offset: float = 1000.0,
             compose_mode: int = COMPOSE, init_dvf=None):
    """Algorithm A over a coarse-to-fine pyramid.  Returns (dvf, stats) where
    stats is a list (coarse -> fine) of dicts: iters_run, stop_reason, rms_id."""
    S, M = _d(static), _d(moving)
    sm, k = _masks(static_masks, S.shape)
    mm, _ = _masks(moving_masks, S.shape)
    lam_a = _d(list(lam) if lam is not None else [1e-3] * max(k, 1))
    if lam is not None and len(lam) == 0:
        lam_a = _d([0.0])
    sg = np.ascontiguousarray(list(sign) if sign is not None and len(sign) else [0] * max(k, 1),
                              dtype=np.int32)
    it = np.ascontiguousarray(list(iters), dtype=np.int32)
    if contour_mask is None:
        contour_mask = 1 << (levels - 1)
    stride = int(max(it)) + 2
    dvf = np.empty((3,) + S.shape)
    ir = np.zeros(levels, np.int32)
    sr = np.zeros(levels, np.int32)
    hl = np.zeros(levels, np.int32)
    hist = np.zeros(levels * stride)
    sp = _d(spacing)
    init = _d(init_dvf) if init_dvf is not None else None
    rc = _load().oracle_register(
        _p(S), _p(M), _p(sm), _p(mm), ctypes.c_int(k), *_dims(S), ctypes.c_int(levels), _p(it),
        ctypes.c_double(sigma_fluid), ctypes.c_double(sigma_diff), _p(lam_a), _p(sg),
        ctypes.c_uint(contour_mask), ctypes.c_int(stop_mode), ctypes.c_double(eps), _p(sp),
        ctypes.c_double(margin), ctypes.c_double(offset), ctypes.c_int(compose_mode), _p(init),
        _p(dvf), _p(ir), _p(sr), _p(hl), _p(hist), ctypes.c_int(stride))
    if rc != 0:
        raise ValueError(f"oracle_register rejected its arguments (status {rc})")
    stats = []
    for l in range(levels):
        stats.append({"iters_run": int(ir[l]), "stop_reason": int(sr[l]),
                      "rms_id": hist[l * stride: l * stride + int(hl[l])].copy()})
    return dvf, stats
