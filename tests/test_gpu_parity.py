"""GPU parity: every step of the CUDA path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances.  The kernels compute in FP32 and the oracle in FP64, so a value
of magnitude |f| carries a rounding error of a few ulp(|f|) ~ 1e-7 |f| per
operation.  Element-wise checks use 1e-5 of the field's scale (10 to 100
ulps of headroom for the few dozen operations of a step).  The per-iteration
DVF bar is the one the method's contract states: ||u_gpu - u_ref|| <= 1e-5
||u_ref|| (plus an absolute floor of 1e-7 voxel per element for fields that
are ~0), and the final DVF of a registration must be within 0.05 voxel RMS.
Integer and mask work (bit packing, mask restriction, the UROI, the signs,
iteration counts) must be bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1301_0970_gb300 as cg  # noqa: E402

DEV = torch.device("cuda:0")
RNG = np.random.default_rng(2024)
# nx % 4 == 0 shapes take the TMA kernels, the others the plain-load kernels
SHAPES = [(9, 21, 45), (1, 1, 1), (3, 8, 32), (17, 33, 70), (5, 1, 7), (9, 21, 44), (17, 33, 68),
          (6, 17, 36)]


def make_context(kernels: str):
    """A context with the default kernels ("tma": two-pass force, TMA
    smoothing where eligible), the one-pass TMA force kernel ("fused") or the
    plain-load kernels everywhere ("plain")."""
    import os
    old = os.environ.get("CGDIR_KERNELS")
    os.environ["CGDIR_KERNELS"] = kernels
    try:
        return cg.Context(0)
    finally:
        if old is None:
            del os.environ["CGDIR_KERNELS"]
        else:
            os.environ["CGDIR_KERNELS"] = old


@pytest.fixture(scope="module", params=["tma", "fused", "plain"])
def ctx(request):
    c = make_context(request.param)
    yield c
    c.close()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def pack(masks):
    b = np.zeros(masks.shape[1:], np.uint8)
    for j in range(masks.shape[0]):
        b |= (masks[j].astype(bool).astype(np.uint8) << j)
    return b


def close_elementwise(got, ref, rel=1e-5, floor=1e-6):
    scale = max(float(np.abs(ref).max()), 1.0)
    err = float(np.abs(got - ref).max())
    assert err <= rel * scale + floor, f"max err {err:.3e} vs scale {scale:.3e}"


def close_normwise(got, ref, rel=1e-5, floor=1e-7):
    num = float(np.linalg.norm((got - ref).ravel()))
    den = float(np.linalg.norm(ref.ravel()))
    assert num <= rel * den + floor * math.sqrt(ref.size), f"{num:.3e} vs {rel:.0e} * {den:.3e}"


def rand_field(shape, amp=2.5):
    return RNG.uniform(-amp, amp, size=(3,) + shape).astype(np.float32)


# ---------------------------------------------------------------- primitives
@pytest.mark.parametrize("k", [0, 1, 5, 8])
def test_pack_masks_bit_exact(ctx, k):
    shape = (7, 13, 37)
    m = (RNG.random((k,) + shape) < 0.3).astype(np.uint8) * RNG.integers(1, 255, size=(k,) + shape,
                                                                           dtype=np.uint8)
    out = ctx.pack_masks([dev(m[j]) for j in range(k)]) if k else None
    if k:
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), pack(m))


@pytest.mark.parametrize("shape", SHAPES)
def test_warp(ctx, shape):
    f = (RNG.normal(size=shape) * 300).astype(np.float32)
    u = rand_field(shape, 3.0)
    got = host(ctx.warp(dev(f), dev(u)))
    close_elementwise(got, oracle.warp(f, u))


@pytest.mark.parametrize("shape", SHAPES + [(8, 16, 64)])
def test_restrict_image_and_bits(ctx, shape):
    f = (RNG.normal(size=shape) * 300).astype(np.float32)
    close_elementwise(host(ctx.restrict_image(dev(f))), oracle.restrict_image(f))
    m = (RNG.random((8,) + shape) < 0.5).astype(np.uint8)
    got = ctx.restrict_bits(dev(pack(m)))
    torch.cuda.synchronize()
    ref = pack(np.stack([oracle.restrict_mask(m[j]) for j in range(8)]))
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("shape", [(5, 11, 23), (1, 1, 1), (4, 4, 4), (9, 13, 70), (12, 20, 33)])
def test_prolong(ctx, shape):
    """Several 64 x 8 x 8 fine tiles with ragged tails in x, y and z, odd and
    even fine sizes."""
    fine = tuple(2 * s - (i % 2) for i, s in enumerate(shape))   # odd and even fine sizes
    uc = rand_field(shape)
    close_elementwise(host(ctx.prolong(dev(uc), fine)), oracle.prolong(uc, fine))


@pytest.mark.parametrize("spacing,margin", [((1.97, 1.97, 2.5), 10.0), ((3.94, 3.94, 5.0), 10.0),
                                            ((1.0, 1.0, 1.0), 10.0),    # 21 z offsets: 32-bit z masks
                                            ((1.0, 1.0, 1.0), 3.0), ((2.0, 1.5, 1.0), 0.0)])
def test_uroi_bit_exact(ctx, spacing, margin):
    shape = (19, 27, 41)
    m = np.zeros((3,) + shape, np.uint8)
    m[0, 5:8, 10:14, 3:9] = 1
    m[1, 15, 25, 39] = 1
    m[2, 0:2, 0:3, 30:41] = 1
    got = ctx.uroi(dev(pack(m)), 3, spacing, margin)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.uroi(m, shape, spacing, margin))
    allv = ctx.uroi(dev(pack(m)), 0, spacing, margin)
    torch.cuda.synchronize()
    assert int(allv.sum()) == int(np.prod(shape))


def test_auto_sign_matches_oracle(ctx):
    c = phantom.make_case("headneck256", shape=(24, 64, 64))
    got = ctx.auto_sign(dev(c.static), dev(pack(c.static_masks)), c.k)
    assert got == oracle.auto_sign(c.static, c.static_masks)


@pytest.mark.parametrize("flip, sign", [(False, -1), (True, 1)])
def test_auto_sign_shell_fixture(ctx, flip, sign):
    """The layered fixture whose sign flips with any other shell (distance 1,
    distance 3, Euclidean radius 2): the device takes the oracle's reading."""
    n = 16
    idx = np.indices((n, n, n))
    d = np.max(np.maximum(np.maximum(6 - idx, idx - 9), 0), axis=0)
    T = np.select([d == 0, d == 1, d == 2], [0.0, -100.0, 110.0], default=-1000.0)
    T = -T if flip else T
    m = (d == 0).astype(np.uint8)[None]
    assert oracle.auto_sign(T, m) == [sign]
    assert ctx.auto_sign(dev(T.astype(np.float32)), dev(pack(m)), 1) == [sign]


@pytest.mark.parametrize("sigma", [1.0, 0.6, 2.0, 0.0])
@pytest.mark.parametrize("shape", [(9, 21, 45), (17, 33, 70), (1, 1, 1), (2, 3, 1), (9, 21, 44),
                                   (17, 33, 72), (30, 8, 4), (3, 5, 8)])
def test_smooth(ctx, sigma, shape):
    u = rand_field(shape)
    got = host(ctx.smooth(dev(u), sigma))
    close_elementwise(got, oracle.gauss_field(u, sigma))
    one = host(ctx.smooth(dev(u[0]), sigma))
    close_elementwise(one, oracle.gauss(u[0], sigma))


@pytest.mark.parametrize("variant", ["tile", "march", "split"])
@pytest.mark.parametrize("shape", [(40, 256, 256), (9, 21, 44), (17, 33, 68), (13, 37, 70)])
def test_smooth_variants(variant, shape):
    """The smoothing kernels (3-D tile, TMA z-march, split xy + z) on the
    same field, one size past the point where the automatic choice
    switches, one with ragged 32-wide tiles."""
    import os
    old = os.environ.get("CGDIR_SMOOTH")
    os.environ["CGDIR_SMOOTH"] = variant
    try:
        c = cg.Context(0)
    finally:
        if old is None:
            del os.environ["CGDIR_SMOOTH"]
        else:
            os.environ["CGDIR_SMOOTH"] = old
    try:
        f = rand_field(shape)
        got = host(c.smooth(dev(f), 1.0))
    finally:
        c.close()
    close_elementwise(got, oracle.gauss_field(f, 1.0))


@pytest.mark.parametrize("mode", [cg.CGDIR_COMPOSE, cg.CGDIR_ADDITIVE])
@pytest.mark.parametrize("sigma", [0.0, 1.0])
@pytest.mark.parametrize("shape,amp", [((9, 21, 45), 1.0), ((9, 21, 44), 1.0), ((20, 37, 64), 3.0),
                                       ((3, 5, 8), 2.5)])
def test_compose(ctx, mode, sigma, shape, amp):
    """The composite update (and, with sigma > 0, G of it) on ragged shapes,
    |du| up to 3 voxels."""
    u, du = rand_field(shape, 4.0), rand_field(shape, amp)
    got = host(ctx.compose(dev(u), dev(du), mode, sigma))
    ref = oracle.compose(u, du, mode)
    if sigma > 0:
        ref = oracle.gauss_field(ref, sigma)
    close_elementwise(got, ref)


def variant_ctx(variant):
    import os
    old = os.environ.get("CGDIR_SMOOTH")
    os.environ["CGDIR_SMOOTH"] = variant
    try:
        return cg.Context(0)
    finally:
        if old is None:
            del os.environ["CGDIR_SMOOTH"]
        else:
            os.environ["CGDIR_SMOOTH"] = old


@pytest.mark.parametrize("sigma", [0.3, 0.6, 1.0, 1.2])
@pytest.mark.parametrize("shape", [(40, 256, 256), (9, 21, 48), (17, 33, 72), (5, 19, 8), (30, 70, 136)])
def test_wide_march_equals_narrow_march_bitwise(shape, sigma):
    """The wide-tile z-march (64 x 16 tiles, nx % 8 == 0, radii 1-4) and the
    32 x 16 one give the same bits (same order of operations) and match the
    oracle; ragged tiles in x, y and z, volumes thinner than the filter, and
    one 8-wide volume whose only x task takes both border clamps."""
    f = rand_field(shape)
    outs = []
    for variant in ("march", "march32"):
        c = variant_ctx(variant)
        try:
            outs.append(host(c.smooth(dev(f), sigma)))
            outs.append(host(c.smooth(dev(f[1]), sigma)))
        finally:
            c.close()
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])
    close_elementwise(outs[0], oracle.gauss_field(f, sigma))
    close_elementwise(outs[1], oracle.gauss(f[1], sigma))


def smooth_wave(shape, amp):
    """A smooth displacement-like field of amplitude amp plus a little noise."""
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    f = np.stack([np.sin(0.31 * x + 0.17 * y + 0.5), np.cos(0.23 * y - 0.29 * z), np.sin(0.19 * z + 0.13 * x)])
    return (amp * f + RNG.uniform(-0.3, 0.3, size=f.shape)).astype(np.float32)


@pytest.mark.parametrize("mode", [cg.CGDIR_COMPOSE, cg.CGDIR_ADDITIVE])
@pytest.mark.parametrize("shape", [(9, 21, 45), (16, 24, 40), (13, 30, 36), (8, 8, 8)])
def test_smooth_compose_all_variants(shape, mode):
    """Algorithm A steps 2-3 (G(du) then the update) with every smoothing
    variant: against the oracle, and the fused 3-D tile kernel equal to the
    tile kernel + update kernel bit for bit.  |G(du)| reaches 3.5 voxels,
    so the update's corners fall both inside the fused kernel's
    shared-memory copy of u (2-voxel halo) and outside it (global loads);
    nx % 4 != 0 takes the fused kernel's plain-load path."""
    u, du = rand_field(shape, 4.0), smooth_wave(shape, 3.5)
    ref = oracle.compose(u, oracle.gauss_field(du, 1.0), mode)
    outs = {}
    for variant in ("tile", "march", "split", "fused"):
        c = variant_ctx(variant)
        try:
            outs[variant] = host(c.smooth_compose(dev(du), dev(u), mode, 1.0))
        finally:
            c.close()
        close_elementwise(outs[variant], ref)
    assert np.array_equal(outs["fused"], outs["tile"])
    assert np.array_equal(outs["split"], outs["tile"])


def case_inputs(shape=(12, 36, 40), masks=None, name="phantom64"):
    c = phantom.make_case(name, shape=shape, masks=masks)
    return c


@pytest.mark.parametrize("k", [0, 1, 2, 5, 8])
@pytest.mark.parametrize("contour", [True, False])
@pytest.mark.parametrize("shape", [(11, 37, 45), (11, 37, 48), (5, 9, 16), (13, 20, 64)])
def test_force(ctx, k, contour, shape):
    c = case_inputs(shape=shape, name="headneck256")
    sm = np.concatenate([c.static_masks] * 2)[:k]
    mm = np.concatenate([c.moving_masks] * 2)[:k]
    lam = list(RNG.uniform(1e-3, 1.0, size=k))
    sign = [1 if j % 2 == 0 else -1 for j in range(k)]
    u = (0.5 * c.u_gt).astype(np.float32)
    ur = oracle.uroi(sm, c.shape) if k else np.ones(c.shape, np.uint8)
    du, stats = ctx.force(dev(c.moving), dev(c.static), dev(pack(mm)), dev(pack(sm)), lam, sign,
                          dev(u), contour=contour, uroi=dev(ur), want_stats=True)
    ref, warped = oracle.force(c.moving, c.static, mm, sm, lam, sign, u=u, contour=contour,
                               return_warped=True)
    got = host(du)
    close_normwise(got, ref)
    sel = ur.astype(bool)
    ssd = float(((warped - c.static)[sel] ** 2).sum())
    assert stats[1] == sel.sum()
    assert abs(stats[0] - ssd) <= 1e-5 * ssd + 1e-6
    assert abs(stats[2] - float(np.sqrt((ref ** 2).sum(0)).max())) <= 1e-4


@pytest.mark.parametrize("kernels", ["tma", "fused"])
def test_force_uniform_mask_fast_path_matches_general_path(kernels):
    """The shortcut where all corners share their mask bits (two-pass and
    one-pass TMA force) must agree with the plain kernel's per-corner
    accumulation."""
    c = phantom.make_case("headneck256", shape=(16, 64, 64))
    u = (0.5 * c.u_gt).astype(np.float32)
    args = (dev(c.moving), dev(c.static), dev(pack(c.moving_masks)), dev(pack(c.static_masks)),
            [0.5] * c.k, c.signs, dev(u))
    a = make_context(kernels)
    b = make_context("plain")
    try:
        da = host(a.force(*args))
        db = host(b.force(*args))
    finally:
        a.close()
        b.close()
    close_normwise(da, db, rel=2e-6)


def test_force_identical_images_is_exactly_zero(ctx):
    c = case_inputs()
    du = ctx.force(dev(c.static), dev(c.static), dev(pack(c.static_masks)), dev(pack(c.static_masks)),
                   c.lam, c.signs, dev(np.zeros((3,) + c.shape, np.float32)))
    torch.cuda.synchronize()
    assert float(du.abs().max()) == 0.0


@pytest.mark.parametrize("name,shape", [("phantom64", (12, 36, 40)), ("headneck256", (13, 45, 50)),
                                        ("pelvis512", (10, 48, 40)), ("headneck256", (24, 64, 64))])
def test_single_iteration_meets_1e5(ctx, name, shape):
    """One iteration (Algorithm A steps 1-4) from a nonzero DVF: relative
    norm-wise difference <= 1e-5."""
    c = phantom.make_case(name, shape=shape)
    u = (0.7 * c.u_gt).astype(np.float32)
    got = host(ctx.iterate(dev(c.moving), dev(c.static), dev(pack(c.moving_masks)),
                           dev(pack(c.static_masks)), c.lam, c.signs, dev(u)))
    ref = oracle.step(c.moving, c.static, c.moving_masks, c.static_masks, c.lam, c.signs, u)
    close_normwise(got, ref, rel=1e-5)


@pytest.fixture(scope="module")
def fused_ctx():
    import os
    old = os.environ.get("CGDIR_SMOOTH")
    os.environ["CGDIR_SMOOTH"] = "fused"
    try:
        c = cg.Context(0)
    finally:
        if old is None:
            del os.environ["CGDIR_SMOOTH"]
        else:
            os.environ["CGDIR_SMOOTH"] = old
    yield c
    c.close()


@pytest.mark.parametrize("mode", [cg.CGDIR_COMPOSE, cg.CGDIR_ADDITIVE])
@pytest.mark.parametrize("name,shape", [("phantom64", (12, 36, 40)), ("headneck256", (13, 45, 50)),
                                        ("pelvis512", (10, 48, 41)), ("headneck256", (5, 3, 7))])
def test_single_iteration_fused_tile_update(fused_ctx, name, shape, mode):
    """One iteration with G(du) and the update in one 3-D tile kernel (8^3
    tiles of all three components, ragged in x, y and z): relative
    norm-wise difference <= 1e-5 from the oracle."""
    c = phantom.make_case(name, shape=shape)
    u = (0.7 * c.u_gt).astype(np.float32)
    got = host(fused_ctx.iterate(dev(c.moving), dev(c.static), dev(pack(c.moving_masks)),
                                 dev(pack(c.static_masks)), c.lam, c.signs, dev(u), compose_mode=mode))
    ref = oracle.step(c.moving, c.static, c.moving_masks, c.static_masks, c.lam, c.signs, u,
                      compose_mode=mode)
    close_normwise(got, ref, rel=1e-5)


def test_rms_id(ctx):
    c = case_inputs()
    ur = oracle.uroi(c.static_masks, c.shape)
    u = c.u_gt.astype(np.float32)
    r, n = ctx.rms_id(dev(c.moving), dev(c.static), dev(u), dev(ur))
    w = oracle.warp(c.moving, u)
    ref, cnt = oracle.rms_id(w, c.static, ur)
    assert n == cnt
    assert abs(r - ref) <= 1e-5 * ref


# --------------------------------------------------------- whole registration
def run_both(c, levels, iters, **kw):
    lam = kw.pop("lam", c.lam)
    sign = kw.pop("sign", c.signs)
    cmask = kw.pop("contour_level_mask", 1 << (levels - 1))
    stop = kw.pop("stop_mode", cg.CGDIR_STOP_FIXED)
    eps = kw.pop("eps", 1e-4)
    with cg.Context(0) as ctx:
        dvf, st = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                               [dev(m) for m in c.moving_masks], levels=levels, iters=iters, lam=lam,
                               sign=sign, contour_level_mask=cmask, stop_mode=stop, eps=eps, **kw)
        got = host(dvf)
    ref, rst = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=levels,
                               iters=iters, lam=lam, sign=sign if sign is not None else None,
                               contour_mask=cmask, stop_mode=stop, eps=eps)
    return got, st, ref, rst


def dvf_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum(axis=0).mean()))


def test_register_two_levels_matches_oracle():
    c = phantom.make_case("phantom64", shape=(20, 48, 44))
    got, st, ref, rst = run_both(c, 2, [40, 30], contour_level_mask=3)
    assert [s["iters_run"] for s in st] == [40, 30]
    assert dvf_rms(got, ref) <= 0.05
    for s, r in zip(st, rst):
        np.testing.assert_allclose(s["rms_id"], r["rms_id"], rtol=1e-3)


def test_register_c1_full_config_matches_oracle():
    """64x64x32, 2 masks, one level of 100 iterations, contour weight 1."""
    c = phantom.make_case("phantom64")
    got, st, ref, rst = run_both(c, 1, [100])
    assert st[0]["iters_run"] == 100
    assert dvf_rms(got, ref) <= 0.05


def test_register_identical_images_give_zero_dvf():
    c = phantom.make_case("phantom64", shape=(10, 30, 34))
    c.moving = c.static.copy()
    c.moving_masks = c.static_masks.copy()
    got, st, _, _ = run_both(c, 2, [5, 5], contour_level_mask=3)
    assert np.all(got == 0)
    assert all(all(v == 0 for v in s["rms_id"]) for s in st)


def test_register_without_masks_is_plain_demons_over_whole_volume():
    c = phantom.make_case("phantom64", shape=(10, 30, 34))
    c.static_masks = c.static_masks[:0]
    c.moving_masks = c.moving_masks[:0]
    got, st, ref, rst = run_both(c, 2, [10, 10], lam=[], sign=[])
    assert dvf_rms(got, ref) <= 0.05


def test_register_odd_sizes_three_levels_and_additive():
    c = phantom.make_case("headneck256", shape=(13, 23, 37))
    got, st, ref, rst = run_both(c, 3, [6, 4, 3], compose_mode=cg.CGDIR_ADDITIVE)
    assert dvf_rms(got, ref) <= 0.05
    assert [s["shape"] for s in st] == [(4, 6, 10), (7, 12, 19), (13, 23, 37)]


def test_register_window10_stops_where_the_oracle_stops():
    c = phantom.make_case("phantom64", shape=(12, 36, 40))
    got, st, ref, rst = run_both(c, 1, [300], stop_mode=cg.CGDIR_STOP_WINDOW10, eps=5e-2)
    assert st[0]["stop_reason"] == rst[0]["stop_reason"] == cg.CGDIR_REASON_CONVERGED
    assert st[0]["iters_run"] == rst[0]["iters_run"]
    assert dvf_rms(got, ref) <= 0.05


def test_register_paper_literal_stops_at_eleven():
    c = phantom.make_case("phantom64", shape=(12, 36, 40))
    got, st, ref, rst = run_both(c, 1, [50], stop_mode=cg.CGDIR_STOP_PAPER_LITERAL)
    assert st[0]["iters_run"] == rst[0]["iters_run"]


def test_register_host_and_device_inputs_agree_bitwise():
    c = phantom.make_case("phantom64", shape=(10, 30, 34))
    kw = dict(levels=2, iters=[5, 5], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as ctx:
        a, _ = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                            [dev(m) for m in c.moving_masks], **kw)
        a = a.cpu()
        b, _ = ctx.register(torch.from_numpy(c.static), torch.from_numpy(c.moving),
                            [torch.from_numpy(m) for m in c.static_masks],
                            [torch.from_numpy(m) for m in c.moving_masks], **kw)
    assert torch.equal(a, b)


def test_register_auto_sign_equals_explicit_sign():
    c = phantom.make_case("headneck256", shape=(16, 48, 48))
    kw = dict(levels=1, iters=[5], lam=c.lam, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as ctx:
        a, _ = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                            [dev(m) for m in c.moving_masks], sign=None, **kw)
        b, _ = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                            [dev(m) for m in c.moving_masks], sign=c.signs, **kw)
        assert torch.equal(a, b)


def test_register_init_dvf_skips_coarse_levels():
    c = phantom.make_case("phantom64", shape=(12, 36, 40))
    with cg.Context(0) as ctx:
        dvf, st = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                               [dev(m) for m in c.moving_masks], levels=2, iters=[30, 4], lam=c.lam,
                               sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED, init_dvf=dev(c.u_gt))
        got = host(dvf)
    assert st[0]["stop_reason"] == cg.CGDIR_REASON_SKIPPED and st[1]["iters_run"] == 4
    ref, _ = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2, iters=[30, 4],
                             lam=c.lam, sign=c.signs, init_dvf=c.u_gt)
    assert dvf_rms(got, ref) <= 0.05


def test_invalid_arguments_are_rejected(ctx):
    c = phantom.make_case("phantom64", shape=(6, 10, 12))
    with pytest.raises(cg.CgdirError) as e:
        ctx.register(dev(c.static), dev(c.moving[:, :, :-1].copy()), levels=1, iters=[1])
    assert e.value.status == cg.CGDIR_EINVAL
    with pytest.raises(cg.CgdirError) as e:
        ctx.register(dev(c.static), dev(c.moving), levels=1, iters=[1], sigma_fluid=3.0)
    assert e.value.status == cg.CGDIR_EINVAL
    masks = [dev(c.static_masks[0])] * 9
    with pytest.raises(cg.CgdirError) as e:
        ctx.register(dev(c.static), dev(c.moving), masks, masks, levels=1, iters=[1])
    assert e.value.status == cg.CGDIR_EINVAL
    with pytest.raises(cg.CgdirError) as e:
        ctx.register(dev(c.static), dev(c.moving), levels=9, iters=[1] * 9)
    assert e.value.status == cg.CGDIR_EINVAL


def _register_with_env(c, env, repeat=1, **kw):
    import os
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        ctx = cg.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    outs = []
    try:
        for _ in range(repeat):
            dvf, st = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                                   [dev(m) for m in c.moving_masks], **kw)
            outs.append((dvf.cpu(), st))
    finally:
        ctx.close()
    return outs


def test_graph_replay_equals_eager_launches_bitwise():
    """The captured CUDA graph runs the same kernels in the same order as the
    eager launch sequence: identical results, also on a second replay."""
    c = phantom.make_case("headneck256", shape=(24, 64, 64))
    kw = dict(levels=2, iters=[6, 4], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_WINDOW10, eps=1e-3)
    g = _register_with_env(c, {"CGDIR_GRAPHS": "1"}, repeat=2, **kw)
    e = _register_with_env(c, {"CGDIR_GRAPHS": "0"}, repeat=1, **kw)
    assert torch.equal(g[0][0], g[1][0]) and torch.equal(g[0][0], e[0][0])
    assert g[0][1] == g[1][1] == e[0][1]


def test_one_context_serves_changing_shapes():
    """Workspace growth drops cached graphs; each call must still match a
    fresh context."""
    shapes = [(12, 32, 32), (20, 48, 64), (12, 32, 32), (8, 16, 16)]
    with cg.Context(0) as ctx:
        for shp in shapes:
            c = phantom.make_case("phantom64", shape=shp)
            kw = dict(levels=2, iters=[4, 3], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
            a, _ = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                                [dev(m) for m in c.moving_masks], **kw)
            b = _register_with_env(c, {}, **kw)[0][0]
            assert torch.equal(a.cpu(), b)


def test_profile_reports_every_kernel_class():
    c = phantom.make_case("phantom64", shape=(12, 32, 32))
    with cg.Context(0) as ctx:
        ctx.profile(list(range(8)))
        ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                     [dev(m) for m in c.moving_masks], levels=2, iters=[3, 2], lam=c.lam, sign=c.signs,
                     stop_mode=cg.CGDIR_STOP_FIXED)
        prof = ctx.profile_read()
    kinds = {p["kernel"] for p in prof}
    # the composite update runs fused into the du smoothing (steps 2 + 3) and
    # the RMS-ID reduction inside the force / metric kernels
    assert {"force", "smooth_du", "smooth_u", "metric", "setup"} <= kinds
    force = {p["level"]: p["launches"] for p in prof if p["kernel"] == "force"}
    assert force == {0: 3, 1: 2}
    assert all(p["total_ms"] > 0 for p in prof)


# ------------------------------------------------- 16-bit image storage (FP32 math)
@pytest.mark.parametrize("storage", [cg.CGDIR_F16, cg.CGDIR_BF16])
@pytest.mark.parametrize("kernels", ["tma", "fused", "plain"])
@pytest.mark.parametrize("shape", [(20, 48, 48), (13, 30, 37)])
def test_half_storage_registration_within_a_tenth_of_a_voxel(storage, kernels, shape):
    """Images stored in FP16 / BF16, all arithmetic FP32: with FP16 storage the
    final DVF stays within 0.1 voxel RMS of the FP64 oracle run on the FP32
    images.  BF16 keeps 8 mantissa bits, a 4 HU step at -1000 HU next to
    15-20 HU contrasts, so its bound is 0.25 voxel."""
    c = phantom.make_case("phantom64", shape=shape)
    ctx = make_context(kernels)
    try:
        dvf, st = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                               [dev(m) for m in c.moving_masks], levels=2, iters=[30, 20], lam=c.lam,
                               sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED, storage_dtype=storage)
        got = host(dvf)
    finally:
        ctx.close()
    ref, _ = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2,
                             iters=[30, 20], lam=c.lam, sign=c.signs)
    assert dvf_rms(got, ref) <= (0.1 if storage == cg.CGDIR_F16 else 0.25)
    assert [s["iters_run"] for s in st] == [30, 20]


@pytest.mark.parametrize("dtype,code", [(torch.float16, cg.CGDIR_F16), (torch.bfloat16, cg.CGDIR_BF16)])
def test_half_inputs_equal_on_device_conversion(dtype, code):
    c = phantom.make_case("phantom64", shape=(16, 40, 48))
    kw = dict(levels=2, iters=[5, 5], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as ctx:
        a, _ = ctx.register(dev(c.static).to(dtype), dev(c.moving).to(dtype),
                            [dev(m) for m in c.static_masks], [dev(m) for m in c.moving_masks], **kw)
        a = a.cpu()
        b, _ = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                            [dev(m) for m in c.moving_masks], storage_dtype=code, **kw)
        b = b.cpu()
        f, _ = ctx.register(dev(c.static), dev(c.moving), [dev(m) for m in c.static_masks],
                            [dev(m) for m in c.moving_masks], storage_dtype=cg.CGDIR_F32, **kw)
    assert torch.equal(a, b)
    assert float((a - f.cpu()).abs().max()) > 0       # the storage type is really in effect
