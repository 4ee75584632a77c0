"""The allocation-free RMS-ID entry point (cgdir_rms_id_noalloc), for callers
that cannot allocate device memory, against the context-based cgdir_rms_id.

This file sorts last so that a run stopping at the first failure has already
run every other test; it must also pass on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1301_0970_gb300 as cg  # noqa: E402


def _noalloc(I0, T0, u, ur, stream):
    nz, ny, nx = I0.shape
    r = ctypes.c_double(-1.0)
    n = ctypes.c_longlong(-1)
    st = cg.load().cgdir_rms_id_noalloc(I0.data_ptr(), T0.data_ptr(), u.data_ptr(),
                                        None if ur is None else ur.data_ptr(), nx, ny, nz,
                                        ctypes.c_void_p(stream), ctypes.byref(r), ctypes.byref(n))
    assert st == cg.CGDIR_OK, cg.load().cgdir_strerror(st)
    return r.value, n.value


@pytest.mark.parametrize("shape,use_uroi", [((12, 36, 40), True), ((17, 33, 70), False),
                                            ((40, 96, 96), True)])
def test_noalloc_rms_matches_context_entry_point_twice(shape, use_uroi):
    c = phantom.make_case("headneck256", shape=shape)
    dev = torch.device("cuda:0")
    I0 = torch.from_numpy(c.moving).to(dev)
    T0 = torch.from_numpy(c.static).to(dev)
    u = torch.from_numpy(np.ascontiguousarray(0.5 * c.u_gt)).to(dev)
    ur = None
    if use_uroi:
        with cg.Context(0) as ctx:
            bits = ctx.pack_masks([torch.from_numpy(m).to(dev) for m in c.static_masks])
            ur = ctx.uroi(bits, c.k)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with cg.Context(0) as ctx:
        ref, ref_n = ctx.rms_id(I0, T0, u, ur)
    for _ in range(2):      # the shared scratch keeps the last call's contents
        got, n = _noalloc(I0, T0, u, ur, stream)
        assert n == ref_n
        assert abs(got - ref) <= 1e-5 * max(ref, 1e-12)


def test_noalloc_rejects_volumes_beyond_its_scratch():
    dev = torch.device("cuda:0")
    t = torch.zeros(8, dtype=torch.float32, device=dev)
    r = ctypes.c_double()
    st = cg.load().cgdir_rms_id_noalloc(t.data_ptr(), t.data_ptr(), t.data_ptr(), None, 4096, 4096, 8,
                                        None, ctypes.byref(r), None)
    assert st == cg.CGDIR_EINVAL
