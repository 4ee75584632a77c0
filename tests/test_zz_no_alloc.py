"""The allocation-free RMS-ID entry point (cgdir_rms_id_noalloc), for callers
that cannot allocate device memory (hosts whose own pool owns every byte of
it, loops where allocation is forbidden), against the context-based
cgdir_rms_id and against the FP64 oracle.

This file sorts last so that a run stopping at the first failure has already
run every other test; it must also pass on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1301_0970_gb300 as cg  # noqa: E402

MAX_VOXELS = 67_108_864          # the entry point's documented limit


def _noalloc(I0, T0, u, ur, stream):
    nz, ny, nx = I0.shape
    r = ctypes.c_double(-1.0)
    n = ctypes.c_longlong(-1)
    st = cg.load().cgdir_rms_id_noalloc(I0.data_ptr(), T0.data_ptr(), u.data_ptr(),
                                        None if ur is None else ur.data_ptr(), nx, ny, nz,
                                        ctypes.c_void_p(stream), ctypes.byref(r), ctypes.byref(n))
    assert st == cg.CGDIR_OK, cg.load().cgdir_strerror(st)
    return r.value, n.value


def _oracle_rms(I0, T0, u, ur):
    """RMS-ID in FP64 from the oracle's warp (Sec. 2.2, stopping criterion)."""
    warped = oracle.warp(I0, u)
    m = np.ones(I0.shape, np.uint8) if ur is None else ur
    return oracle.rms_id(warped, T0, m)


def _check(I0h, T0h, uh, urh):
    dev = torch.device("cuda:0")
    I0, T0, u = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (I0h, T0h, uh))
    ur = None if urh is None else torch.from_numpy(np.ascontiguousarray(urh)).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with cg.Context(0) as ctx:
        ref, ref_n = ctx.rms_id(I0, T0, u, ur)
    want, want_n = _oracle_rms(I0h, T0h, uh, urh)
    assert ref_n == want_n
    for _ in range(2):      # the shared scratch keeps the last call's contents
        got, n = _noalloc(I0, T0, u, ur, stream)
        assert n == ref_n
        assert abs(got - ref) <= 1e-5 * max(ref, 1e-12)
        assert abs(got - want) <= 1e-5 * max(want, 1e-12)


@pytest.mark.parametrize("shape,use_uroi", [((12, 36, 40), True), ((17, 33, 70), False),
                                            ((40, 96, 96), True)])
def test_noalloc_rms_matches_context_entry_point_and_oracle_twice(shape, use_uroi):
    c = phantom.make_case("headneck256", shape=shape)
    ur = oracle.uroi(c.static_masks, shape).astype(np.uint8) if use_uroi else None
    _check(c.moving, c.static, (0.5 * c.u_gt).astype(np.float32), ur)


def test_noalloc_at_its_voxel_limit():
    """64 x 1024 x 1024 voxels, the largest volume accepted: 64 voxels per
    thread, every one of the 4096 partial slots in use."""
    shape = (64, 1024, 1024)
    assert int(np.prod(shape)) == MAX_VOXELS
    rng = np.random.default_rng(77)
    I0 = (rng.standard_normal(shape, dtype=np.float32) * 300.0).astype(np.float32)
    T0 = (rng.standard_normal(shape, dtype=np.float32) * 300.0).astype(np.float32)
    u = rng.uniform(-3.0, 3.0, size=(3,) + shape).astype(np.float32)
    ur = (rng.random(shape, dtype=np.float32) < 0.6).astype(np.uint8)
    _check(I0, T0, u, ur)


def test_noalloc_rejects_volumes_beyond_its_scratch():
    dev = torch.device("cuda:0")
    t = torch.zeros(8, dtype=torch.float32, device=dev)
    r = ctypes.c_double()
    st = cg.load().cgdir_rms_id_noalloc(t.data_ptr(), t.data_ptr(), t.data_ptr(), None, 4096, 4096, 8,
                                        None, ctypes.byref(r), None)
    assert st == cg.CGDIR_EINVAL
    st = cg.load().cgdir_rms_id_noalloc(t.data_ptr(), t.data_ptr(), t.data_ptr(), None, 1025, 1024, 64,
                                        None, ctypes.byref(r), None)
    assert st == cg.CGDIR_EINVAL
