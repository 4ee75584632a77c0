"""Pins of the oracle's moving-vector step (Eq. 5-7, Sec. 2.1; kernels 2-3)
against a direct numerical minimisation of Eq. 6, Thirion's closed form
(lambda = 0) and the special cases the method has."""
import numpy as np
import pytest
from scipy import optimize

import oracle

RNG = np.random.default_rng(77)
OFF = 1000.0


def clamped_central_difference(f):
    """(f[i+1] - f[i-1]) / 2 with clamped indices, per axis, [3][...]."""
    out = []
    for axis in (2, 1, 0):  # x, y, z
        n = f.shape[axis]
        i = np.arange(n)
        up = np.take(f, np.minimum(i + 1, n - 1), axis=axis)
        dn = np.take(f, np.maximum(i - 1, 0), axis=axis)
        out.append(0.5 * (up - dn))
    return np.stack(out)


def make_inputs(shape=(6, 7, 8), k=3, seed=0):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    I0 = 30 * np.sin(0.7 * x + 0.3 * y) + 20 * np.cos(0.5 * z - 0.4 * x) + 5 * y + rng.normal(0, 3, shape)
    T0 = I0 + rng.normal(0, 15, shape)
    mm = (rng.random((k,) + shape) < 0.4).astype(np.uint8)
    sm = (rng.random((k,) + shape) < 0.4).astype(np.uint8)
    lam = list(rng.uniform(0.2, 2.0, size=k))
    sign = list(rng.choice([-1, 1], size=k))
    return I0, T0, mm, sm, lam, sign


def eq6_terms(I0, T0, mm, sm, lam, sign, shift=(0, 0, 0)):
    """Warped images (an integer shift is an exact warp), their central
    differences, and the per-voxel coefficients of Eq. 6."""
    def shifted(f):
        g = f
        for axis, s in zip((2, 1, 0), shift):
            n = f.shape[axis]
            idx = np.clip(np.arange(n) + s, 0, n - 1)
            g = np.take(g, idx, axis=axis)
        return g
    w0 = shifted(I0)
    g0 = clamped_central_difference(w0)
    terms = []
    for i in range(len(lam)):
        Ii = (1 + sign[i] * mm[i] / 2.0) * (I0 + OFF)      # Sec. 2.1 modified image
        Ti = (1 + sign[i] * sm[i] / 2.0) * (T0 + OFF)
        wi = shifted(Ii)
        terms.append((lam[i], clamped_central_difference(wi), Ti - wi))
    return w0, g0, terms


def argmin_eq6(a0, r0, parts, beta):
    def E(v):
        e = 0.5 * (a0 * v - r0) ** 2 + 0.5 * beta * v * v
        for lam, ai, ri in parts:
            e += 0.5 * lam * (ai * v - ri) ** 2
        return e
    res = optimize.minimize_scalar(E, bounds=(-1e3, 1e3), method="bounded",
                                   options={"xatol": 1e-12, "maxiter": 10000})
    return res.x, E


@pytest.mark.parametrize("shift", [(0, 0, 0), (1, -2, 1)])
def test_eq7_is_the_minimiser_of_eq6(shift):
    I0, T0, mm, sm, lam, sign = make_inputs()
    u = np.zeros((3,) + I0.shape)
    for a in range(3):
        u[a] = shift[a]
    du = oracle.force(I0, T0, mm, sm, lam, sign, u=u, offset=OFF)
    w0, g0, terms = eq6_terms(I0, T0, mm, sm, lam, sign, shift)
    checked = 0
    for idx in np.ndindex(I0.shape):
        g = g0[(slice(None),) + idx]
        gn = np.linalg.norm(g)
        if gn == 0:
            assert np.all(du[(slice(None),) + idx] == 0)
            continue
        n = g / gn
        r0 = T0[idx] - w0[idx]
        parts = [(lam_i, float(gi[(slice(None),) + idx] @ n), float(ri[idx]))
                 for (lam_i, gi, ri) in terms]
        v_star, E = argmin_eq6(gn, r0, parts, beta=r0 * r0)
        d = du[(slice(None),) + idx]
        v = float(d @ n)
        # du is along n
        np.testing.assert_allclose(d, v * n, atol=1e-12 * (1 + abs(v)))
        assert abs(v - v_star) <= 1e-6 * (1 + abs(v_star))
        # and it is a local minimum of Eq. 6
        h = 1e-4 * (1 + abs(v))
        assert E(v) <= E(v + h) and E(v) <= E(v - h)
        checked += 1
    assert checked > 200


def test_lambda_zero_is_thirion_demons_with_moving_gradient():
    I0, T0, mm, sm, lam, sign = make_inputs(seed=3)
    du = oracle.force(I0, T0, mm, sm, [0.0] * len(lam), sign, offset=OFF)
    g = clamped_central_difference(I0)
    r0 = T0 - I0
    denom = (g * g).sum(0) + r0 * r0
    expect = np.where(denom > 0, r0 / np.where(denom > 0, denom, 1), 0) * g
    np.testing.assert_allclose(du, expect, rtol=1e-12, atol=1e-14)


def test_contour_switch_off_equals_lambda_zero():
    I0, T0, mm, sm, lam, sign = make_inputs(seed=4)
    a = oracle.force(I0, T0, mm, sm, lam, sign, contour=False)
    b = oracle.force(I0, T0, mm, sm, [0.0] * len(lam), sign)
    np.testing.assert_array_equal(a, b)


def test_identical_images_and_masks_give_zero_force():
    I0, _, mm, _, lam, sign = make_inputs(seed=5)
    du = oracle.force(I0, I0.copy(), mm, mm.copy(), lam, sign)
    assert np.all(du == 0)


def test_flat_image_has_zero_gradient_and_zero_force():
    I0 = np.full((4, 5, 6), 12.0)
    T0 = I0 + RNG.normal(size=I0.shape)
    m = (RNG.random((2,) + I0.shape) < 0.5).astype(np.uint8)
    du = oracle.force(I0, T0, m, m, [1.0, 1.0], [1, -1])
    assert np.all(du == 0)


def test_force_bounded_by_half_voxel_without_contour_term():
    """Thirion's force r g / (|g|^2 + r^2) never exceeds 1/2 in length."""
    I0, T0, mm, sm, lam, sign = make_inputs(seed=6)
    du = oracle.force(I0, T0 * 3, mm, sm, lam, sign, contour=False)
    assert np.sqrt((du ** 2).sum(0)).max() <= 0.5 + 1e-12


def test_contour_term_pulls_the_moving_roi_onto_the_static_roi_for_either_sign():
    """Identical images (r0 = 0), the static ROI one voxel to the right of the
    moving ROI.  At the voxel covered only by the static ROI the update must
    sample the moving image further left (du_x < 0, pull-back), towards the
    moving ROI, whatever the sign of M_i, N_i; the factors 1.5 / 0.5 inside
    the ROI (Sec. 2.1) set the magnitude."""
    shape = (5, 6, 9)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    I0 = 10.0 * x
    m = np.zeros((1,) + shape, np.uint8)
    m[0, :, :, 3:6] = 1
    sm = np.roll(m, 1, axis=3)
    for s, factor in ((1, 1.5), (-1, 0.5)):
        du = oracle.force(I0, I0.copy(), m, sm, [1.0], [s], offset=OFF)
        J = lambda xx: 10.0 * xx + OFF
        gi = 0.5 * (J(7) - factor * J(5))
        ri = factor * J(6) - J(6)
        v = gi * ri / (10.0 ** 2 + gi * gi)
        assert du[0][2, 3, 6] < 0
        assert abs(du[0][2, 3, 6] - v) < 1e-12
