"""Pins of the oracle's whole registration (Algorithm A, Sec. 2.2) against
invariants, an independently written loop built on SciPy's interpolation and
filtering, recovery of a known deformation, and the paper's qualitative
claim that the contour term improves ROI overlap (Table 2)."""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
import phantom

OFF = 1000.0


# ---------------------------------------------------------------------------
# an independently written Algorithm A (SciPy interpolation and filtering)
# ---------------------------------------------------------------------------
def lib_warp(f, u):
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in f.shape], indexing="ij")
    c = np.stack([np.clip(z + u[2], 0, f.shape[0] - 1), np.clip(y + u[1], 0, f.shape[1] - 1),
                  np.clip(x + u[0], 0, f.shape[2] - 1)])
    return ndimage.map_coordinates(f, c, order=1, mode="nearest")


def lib_grad(f):
    out = []
    for axis in (2, 1, 0):
        n = f.shape[axis]
        i = np.arange(n)
        out.append(0.5 * (np.take(f, np.minimum(i + 1, n - 1), axis=axis)
                          - np.take(f, np.maximum(i - 1, 0), axis=axis)))
    return np.stack(out)


def lib_smooth(u, sigma=1.0):
    r = math.ceil(3 * sigma - 1e-9)
    t = np.exp(-np.arange(-r, r + 1) ** 2 / (2 * sigma * sigma))
    t /= t.sum()
    out = np.empty_like(u)
    for c in range(3):
        v = u[c]
        for axis in (2, 1, 0):
            v = ndimage.correlate1d(v, t, axis=axis, mode="nearest")
        out[c] = v
    return out


def lib_iteration(I0, T0, mm, sm, lam, sign, u):
    w0 = lib_warp(I0, u)
    g0 = lib_grad(w0)
    gn = np.sqrt((g0 * g0).sum(0))
    safe = np.where(gn > 0, gn, 1.0)
    n = g0 / safe
    r0 = T0 - w0
    num = gn * r0
    den = gn * gn
    for i in range(len(lam)):
        Ii = (1 + sign[i] * mm[i] / 2.0) * (I0 + OFF)
        Ti = (1 + sign[i] * sm[i] / 2.0) * (T0 + OFF)
        wi = lib_warp(Ii, u)
        ai = (lib_grad(wi) * n).sum(0)
        num = num + lam[i] * ai * (Ti - wi)
        den = den + lam[i] * ai * ai
    v = np.where(gn > 0, num / (den + r0 * r0), 0.0)
    du = lib_smooth(v * n)
    return lib_smooth(np.stack([du[c] + lib_warp(u[c], du) for c in range(3)]))


def small_case(shape=(12, 20, 18), masks=None):
    return phantom.make_case("phantom64", shape=shape, masks=masks)


# ---------------------------------------------------------------------------
def test_one_iteration_matches_library_built_loop():
    c = small_case()
    u0 = 0.3 * c.u_gt.astype(float)
    ref = lib_iteration(c.moving.astype(float), c.static.astype(float), c.moving_masks,
                        c.static_masks, c.lam, c.signs, u0)
    out = oracle.step(c.moving, c.static, c.moving_masks, c.static_masks, c.lam, c.signs, u0)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("lam", [None, 0.0])
def test_whole_level_matches_library_built_loop(lam):
    c = small_case()
    lam_v = c.lam if lam is None else [lam] * c.k
    dvf, stats = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=1,
                                 iters=[12], lam=lam_v, sign=c.signs)
    u = np.zeros((3,) + c.shape)
    for _ in range(12):
        u = lib_iteration(c.moving.astype(float), c.static.astype(float), c.moving_masks,
                          c.static_masks, lam_v, c.signs, u)
    np.testing.assert_allclose(dvf, u, rtol=0, atol=1e-9)
    assert stats[0]["iters_run"] == 12 and len(stats[0]["rms_id"]) == 13


def test_identical_images_give_zero_dvf_at_every_level():
    c = small_case()
    dvf, stats = oracle.register(c.static, c.static.copy(), c.static_masks, c.static_masks.copy(),
                                 levels=2, iters=[5, 5], lam=[1.0] * c.k, sign=c.signs,
                                 contour_mask=3)
    assert np.all(dvf == 0)
    for s in stats:
        assert np.all(s["rms_id"] == 0)


def test_lambda_zero_equals_contour_switched_off():
    c = small_case()
    a, _ = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2,
                           iters=[4, 4], lam=[0.0] * c.k, sign=c.signs, contour_mask=3)
    b, _ = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2,
                           iters=[4, 4], lam=c.lam, sign=c.signs, contour_mask=0)
    np.testing.assert_array_equal(a, b)


def test_pyramid_prolongs_coarse_result_into_the_fine_level():
    """With zero fine iterations the result is the prolongated coarse field."""
    c = small_case()
    coarse, _ = oracle.register(oracle.restrict_image(c.static), oracle.restrict_image(c.moving),
                                [oracle.restrict_mask(m) for m in c.static_masks],
                                [oracle.restrict_mask(m) for m in c.moving_masks], levels=1,
                                iters=[6], lam=c.lam, sign=c.signs, contour_mask=0,
                                spacing=(2 * 1.97, 2 * 1.97, 5.0))
    dvf, stats = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2,
                                 iters=[6, 0], lam=c.lam, sign=c.signs)
    np.testing.assert_allclose(dvf, oracle.prolong(coarse, c.shape), atol=1e-13)
    assert stats[1]["iters_run"] == 0 and len(stats[1]["rms_id"]) == 1


def test_rms_history_is_the_uroi_rms_of_the_warped_moving_image():
    c = small_case()
    dvf, stats = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=1,
                                 iters=[3], lam=c.lam, sign=c.signs)
    ur = oracle.uroi(c.static_masks, c.shape)
    w = lib_warp(c.moving.astype(float), dvf)
    sel = ur.astype(bool)
    expect = math.sqrt(((w - c.static)[sel] ** 2).mean())
    assert abs(stats[0]["rms_id"][-1] - expect) < 1e-9
    w0 = c.moving.astype(float)
    assert abs(stats[0]["rms_id"][0] - math.sqrt(((w0 - c.static)[sel] ** 2).mean())) < 1e-9


def test_window10_stops_early_on_a_converging_case_and_fixed_runs_the_cap():
    c = small_case()
    _, st_fixed = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=1,
                                  iters=[60], lam=c.lam, sign=c.signs)
    assert st_fixed[0]["iters_run"] == 60 and st_fixed[0]["stop_reason"] == oracle.REASON_CAP
    _, st = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=1,
                            iters=[400], lam=c.lam, sign=c.signs, stop_mode=oracle.STOP_WINDOW10,
                            eps=1e-2)
    n = st[0]["iters_run"]
    d = st[0]["rms_id"]
    assert st[0]["stop_reason"] == oracle.REASON_CONVERGED and 10 <= n < 400
    assert d[n - 10] - d[n] <= 1e-2
    assert all(d[m - 10] - d[m] > 1e-2 for m in range(10, n))


def test_init_dvf_skips_the_coarse_levels():
    c = small_case()
    dvf, st = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2,
                              iters=[50, 3], lam=c.lam, sign=c.signs, init_dvf=c.u_gt)
    assert st[0]["stop_reason"] == oracle.REASON_SKIPPED and st[0]["iters_run"] == 0
    assert st[1]["iters_run"] == 3
    ref, _ = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=1,
                             iters=[3], lam=c.lam, sign=c.signs, init_dvf=c.u_gt)
    np.testing.assert_array_equal(dvf, ref)


def test_odd_sizes_and_three_levels_run():
    c = phantom.make_case("headneck256", shape=(13, 23, 21))
    dvf, st = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=3,
                              iters=[3, 2, 1], lam=c.lam, sign=c.signs)
    assert dvf.shape == (3, 13, 23, 21)
    assert [s["iters_run"] for s in st] == [3, 2, 1]
    assert np.isfinite(dvf).all()


def test_auto_sign_matches_the_phantom_contrast():
    c = phantom.make_case("headneck256", shape=(24, 64, 64))
    assert oracle.auto_sign(c.static, c.static_masks) == c.signs


# ---------------------------------------------------------------------------
# method-level pins on the synthetic phantom (known ground truth)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1_results():
    c = phantom.make_case("phantom64")
    out = {}
    for name, lam in (("cgdir", c.lam), ("demons", [0.0] * c.k)):
        dvf, st = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2,
                                  iters=[100, 100], lam=lam, sign=c.signs, contour_mask=3)
        out[name] = (dvf, st)
    return c, out


def test_recovers_known_smooth_deformation(c1_results):
    """Two-scale registration (Sec. 2.2) of the phantom pair recovers the
    ground-truth DVF: RMS error over the body <= 0.5 RMS(u_gt)."""
    c, out = c1_results
    body = c.body.astype(bool)
    gt = np.sqrt((c.u_gt.astype(float) ** 2).sum(0))[body]
    for name in ("cgdir", "demons"):
        err = np.sqrt(((out[name][0] - c.u_gt) ** 2).sum(0))[body]
        assert np.sqrt((err ** 2).mean()) <= 0.5 * np.sqrt((gt ** 2).mean()), name


def test_contour_term_improves_roi_overlap(c1_results):
    """Table 2's qualitative claim: CG-DIR's deformed ROI overlaps the target
    ROI at least as well as demons', and both beat no registration."""
    c, out = c1_results

    def dsc(a, b):
        return 2.0 * (a & b).sum() / (a.sum() + b.sum())
    for i in range(c.k):
        target = c.static_masks[i].astype(bool)
        before = dsc(c.moving_masks[i].astype(bool), target)
        d = {n: dsc(lib_warp(c.moving_masks[i].astype(float), out[n][0]) >= 0.5, target)
             for n in ("cgdir", "demons")}
        assert d["cgdir"] >= d["demons"] > before


def test_rms_id_decreases_to_the_noise_floor(c1_results):
    """Each level lowers the UROI RMS-ID; at the end it is below the RMS of
    the difference of two independent noise fields (sqrt(2) * 20 HU)."""
    _, out = c1_results
    for name in ("cgdir", "demons"):
        for s in out[name][1]:
            h = s["rms_id"]
            assert h[-1] < h[0]
        assert out[name][1][-1]["rms_id"][-1] < math.sqrt(2) * 20.0
        assert out[name][1][0]["rms_id"][0] > 3 * math.sqrt(2) * 20.0
