"""Pins of the FP64 oracle's primitives against closed forms, brute force and
independent library routines (never against the oracle itself).

Sec. 2.2 (kernels 1, 2, 4; the multi-scale strategy; the UROI and the
stopping test)."""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle

RNG = np.random.default_rng(1234)
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "paper_parameters.json")))


def ramp(shape, coef=(0.7, -1.3, 2.1), c0=5.0):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return coef[0] * x + coef[1] * y + coef[2] * z + c0, (x, y, z)


# ------------------------------------------------------------------ warp ---
def test_warp_zero_field_is_identity_bit_exact():
    f = RNG.normal(size=(5, 7, 9)) * 100
    out = oracle.warp(f, np.zeros((3,) + f.shape))
    assert np.array_equal(out, f)


def test_warp_integer_shift_is_exact_in_interior():
    f = RNG.normal(size=(8, 9, 10))
    s = (2, -1, 3)  # x, y, z
    u = np.zeros((3,) + f.shape)
    for a in range(3):
        u[a] = s[a]
    out = oracle.warp(f, u)
    # out[z,y,x] = f[z+3, y-1, x+2] where in range
    assert np.array_equal(out[:-3, 1:, :-2], f[3:, :-1, 2:])


def test_warp_reproduces_affine_functions_for_in_domain_samples():
    shape = (6, 7, 8)
    f, (x, y, z) = ramp(shape)
    u = RNG.uniform(-1.5, 1.5, size=(3,) + shape)
    px, py, pz = x + u[0], y + u[1], z + u[2]
    inside = (px >= 0) & (px <= shape[2] - 1) & (py >= 0) & (py <= shape[1] - 1) & \
             (pz >= 0) & (pz <= shape[0] - 1)
    out = oracle.warp(f, u)
    expect = 0.7 * px - 1.3 * py + 2.1 * pz + 5.0
    assert inside.sum() > 100
    np.testing.assert_allclose(out[inside], expect[inside], rtol=0, atol=1e-12)


def test_warp_clamps_out_of_domain_samples_to_the_border():
    shape = (4, 5, 6)
    f, (x, y, z) = ramp(shape)
    u = RNG.uniform(-8, 8, size=(3,) + shape)
    px = np.clip(x + u[0], 0, shape[2] - 1)
    py = np.clip(y + u[1], 0, shape[1] - 1)
    pz = np.clip(z + u[2], 0, shape[0] - 1)
    np.testing.assert_allclose(oracle.warp(f, u), 0.7 * px - 1.3 * py + 2.1 * pz + 5.0,
                               atol=1e-12)


def test_warp_matches_library_linear_interpolation():
    """scipy.ndimage.map_coordinates(order=1, mode='nearest') is an independent
    trilinear interpolator with replicated borders."""
    f = RNG.normal(size=(7, 6, 9))
    u = RNG.uniform(-3, 3, size=(3,) + f.shape)
    z, y, x = np.meshgrid(*[np.arange(n) for n in f.shape], indexing="ij")
    coords = np.stack([np.clip(z + u[2], 0, f.shape[0] - 1), np.clip(y + u[1], 0, f.shape[1] - 1),
                       np.clip(x + u[0], 0, f.shape[2] - 1)])
    ref = ndimage.map_coordinates(f, coords, order=1, mode="nearest")
    np.testing.assert_allclose(oracle.warp(f, u), ref, atol=1e-12)


# -------------------------------------------------------------- gradient ---
def test_central_difference_is_exact_on_quadratics_in_interior():
    shape = (7, 8, 9)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    f = 0.3 * x * x - 0.2 * y * y + 0.5 * z * z + 0.7 * x * y - 0.4 * y * z + 1.1 * x - 3
    g = oracle.gradient(f)
    gx = 0.6 * x + 0.7 * y + 1.1
    gy = -0.4 * y + 0.7 * x - 0.4 * z
    gz = 1.0 * z - 0.4 * y
    sl = (slice(1, -1),) * 3
    np.testing.assert_allclose(g[0][sl], gx[sl], atol=1e-11)
    np.testing.assert_allclose(g[1][sl], gy[sl], atol=1e-11)
    np.testing.assert_allclose(g[2][sl], gz[sl], atol=1e-11)


def test_gradient_of_constant_is_zero_and_border_is_half_one_sided():
    assert np.all(oracle.gradient(np.full((3, 4, 5), 7.0)) == 0)
    f, _ = ramp((3, 4, 5))
    g = oracle.gradient(f)
    # clamped index at the border: (f[1] - f[0]) / 2 = slope / 2
    np.testing.assert_allclose(g[0][:, :, 0], 0.35, atol=1e-12)
    np.testing.assert_allclose(g[0][:, :, 2], 0.7, atol=1e-12)
    np.testing.assert_allclose(g[2][-1], 1.05, atol=1e-12)


def test_gradient_of_single_voxel_axis_is_zero():
    f = RNG.normal(size=(1, 4, 5))
    assert np.all(oracle.gradient(f)[2] == 0)


# -------------------------------------------------------------- gaussian ---
def closed_form_taps(sigma):
    r = math.ceil(3 * sigma - 1e-9)
    j = np.arange(-r, r + 1)
    t = np.exp(-j * j / (2 * sigma * sigma))
    return t / t.sum()


@pytest.mark.parametrize("sigma", [1.0, 0.6, 1.7])
def test_gauss_taps_closed_form(sigma):
    t = oracle.gauss_taps(sigma)
    np.testing.assert_allclose(t, closed_form_taps(sigma), rtol=1e-14)
    assert abs(t.sum() - 1) < 1e-14


def test_paper_sigma_gives_radius_three():
    assert oracle.gauss_radius(GOLDEN["gaussian_sigma_voxels"]["value"]) == 3


@pytest.mark.parametrize("sigma", [1.0, 0.6])
def test_gauss_equals_brute_force_3d_convolution(sigma):
    """Separable x->y->z filtering equals one 3-D convolution with the
    outer-product kernel (scipy, mode='nearest' == clamp-to-edge)."""
    f = RNG.normal(size=(9, 10, 11))
    t = closed_form_taps(sigma)
    k3 = t[:, None, None] * t[None, :, None] * t[None, None, :]
    ref = ndimage.correlate(f, k3, mode="nearest")
    np.testing.assert_allclose(oracle.gauss(f, sigma), ref, atol=1e-12)


def test_gauss_impulse_response_is_the_outer_product():
    f = np.zeros((9, 9, 9))
    f[4, 4, 4] = 1.0
    t = closed_form_taps(1.0)
    out = oracle.gauss(f, 1.0)
    np.testing.assert_allclose(out[1:8, 1:8, 1:8],
                               t[:, None, None] * t[None, :, None] * t[None, None, :], atol=1e-15)


def test_gauss_preserves_constants_and_interior_linear_fields():
    np.testing.assert_allclose(oracle.gauss(np.full((5, 6, 7), 3.25), 1.0), 3.25, atol=1e-13)
    f, _ = ramp((12, 12, 12))
    out = oracle.gauss(f, 1.0)
    sl = (slice(3, -3),) * 3
    np.testing.assert_allclose(out[sl], f[sl], atol=1e-11)


def test_gauss_sigma_zero_is_identity():
    f = RNG.normal(size=(3, 4, 5))
    assert np.array_equal(oracle.gauss(f, 0.0), f)


def test_gauss_field_smooths_each_component_independently():
    u = RNG.normal(size=(3, 5, 6, 7))
    out = oracle.gauss_field(u, 1.0)
    for c in range(3):
        np.testing.assert_array_equal(out[c], oracle.gauss(u[c], 1.0))


# --------------------------------------------------------------- compose ---
def test_compose_with_zero_field_returns_du():
    du = RNG.normal(size=(3, 4, 5, 6))
    np.testing.assert_array_equal(oracle.compose(np.zeros_like(du), du), du)


def test_compose_of_constant_shifts_adds():
    shape = (8, 8, 8)
    u = np.zeros((3,) + shape)
    du = np.zeros((3,) + shape)
    for a, (s, d) in enumerate([(1.25, 0.5), (-0.75, 1.0), (0.5, -0.25)]):
        u[a], du[a] = s, d
    out = oracle.compose(u, du)
    for a, tot in enumerate([1.75, 0.25, 0.25]):
        np.testing.assert_allclose(out[a], tot, atol=1e-14)


def test_compose_of_affine_field_is_exact_in_domain():
    """u(x) = A x + b, so u(x + d) = u(x) + A d exactly for trilinear."""
    shape = (10, 10, 10)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    A = RNG.uniform(-0.1, 0.1, size=(3, 3))
    b = RNG.uniform(-1, 1, size=3)
    pos = [x, y, z]
    u = np.stack([A[a, 0] * x + A[a, 1] * y + A[a, 2] * z + b[a] for a in range(3)])
    d = np.array([0.4, -0.7, 1.2])
    du = np.broadcast_to(d[:, None, None, None], u.shape).copy()
    out = oracle.compose(u, du)
    expect = np.stack([d[a] + u[a] + A[a] @ d for a in range(3)])
    sl = (slice(None), slice(1, -2), slice(1, -2), slice(1, -2))
    np.testing.assert_allclose(out[sl], expect[sl], atol=1e-12)
    assert pos  # silence linters


def test_additive_mode_is_sum():
    u = RNG.normal(size=(3, 3, 4, 5))
    du = RNG.normal(size=u.shape)
    np.testing.assert_allclose(oracle.compose(u, du, oracle.ADDITIVE), u + du, atol=0)


# --------------------------------------------------------- restrict/prolong ---
def test_restrict_constant_and_ramp():
    assert np.all(oracle.restrict_image(np.full((6, 8, 10), -3.5)) == -3.5)
    f, _ = ramp((8, 10, 12))
    c = oracle.restrict_image(f)
    assert c.shape == (4, 5, 6)
    Z, Y, X = np.meshgrid(*[np.arange(n, dtype=float) for n in c.shape], indexing="ij")
    np.testing.assert_allclose(c, 0.7 * (2 * X + 0.5) - 1.3 * (2 * Y + 0.5) + 2.1 * (2 * Z + 0.5) + 5,
                               atol=1e-12)


def test_restrict_odd_sizes_round_up_and_replicate():
    f = RNG.normal(size=(3, 5, 7))
    c = oracle.restrict_image(f)
    assert c.shape == (2, 3, 4)
    # last x cell of an odd row averages the border voxel with itself
    np.testing.assert_allclose(c[0, 0, 3], (2 * f[0, 0, 6] + 2 * f[0, 1, 6] + 2 * f[1, 0, 6]
                                            + 2 * f[1, 1, 6]) / 8, atol=1e-14)


def test_restrict_mask_majority_with_ties_inside():
    m = np.zeros((2, 2, 2), np.uint8)
    m[0] = 1                                   # exactly 4 of 8
    assert oracle.restrict_mask(m)[0, 0, 0] == 1
    m[0, 0, 0] = 0                             # 3 of 8
    assert oracle.restrict_mask(m)[0, 0, 0] == 0


def test_prolong_doubles_constants_and_maps_ramps_cell_centred():
    uc = np.zeros((3, 4, 5, 6))
    uc[0], uc[1], uc[2] = 1.5, -0.25, 2.0
    uf = oracle.prolong(uc, (8, 10, 12))
    for a, v in enumerate([3.0, -0.5, 4.0]):
        np.testing.assert_allclose(uf[a], v, atol=1e-14)
    c, _ = ramp((4, 5, 6))
    uc = np.stack([c, c, c])
    uf = oracle.prolong(uc, (8, 10, 12))
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in (8, 10, 12)], indexing="ij")
    X, Y, Z = (x + 0.5) / 2 - 0.5, (y + 0.5) / 2 - 0.5, (z + 0.5) / 2 - 0.5
    expect = 2 * (0.7 * X - 1.3 * Y + 2.1 * Z + 5)
    sl = (slice(1, -1),) * 3
    np.testing.assert_allclose(uf[0][sl], expect[sl], atol=1e-12)


def test_restrict_then_prolong_round_trip_of_a_ramp_field():
    """Restricting a voxel-unit field halves its units; prolongation doubles
    them back, so an affine displacement survives the round trip inside."""
    f, _ = ramp((12, 12, 12), coef=(0.05, 0.02, -0.03), c0=0.5)
    half = oracle.restrict_image(f) / 2.0
    back = oracle.prolong(np.stack([half] * 3), f.shape)[0]
    sl = (slice(2, -2),) * 3
    np.testing.assert_allclose(back[sl], f[sl], atol=1e-12)


# -------------------------------------------------------------------- UROI ---
@pytest.mark.parametrize("spacing,margin", [((1.97, 1.97, 2.5), 10.0), ((1.0, 1.0, 1.0), 2.0),
                                            ((3.0, 2.0, 1.5), 4.5)])
def test_uroi_equals_library_euclidean_distance_transform(spacing, margin):
    shape = (14, 17, 19)
    m = np.zeros((2,) + shape, np.uint8)
    m[0, 6:8, 4:7, 5:9] = 1
    m[1, 3, 12, 14] = 1
    union = m.any(axis=0)
    dist = ndimage.distance_transform_edt(~union, sampling=(spacing[2], spacing[1], spacing[0]))
    ref = (dist <= margin + 1e-9).astype(np.uint8)
    np.testing.assert_array_equal(oracle.uroi(m, shape, spacing, margin), ref)


def test_uroi_without_structures_is_whole_volume():
    assert np.all(oracle.uroi(None, (3, 4, 5)) == 1)


def test_uroi_paper_margin_radii():
    """1 cm at 1.97 x 1.97 x 2.5 mm reaches 5 voxels in x/y and 4 in z."""
    shape = (11, 13, 13)
    m = np.zeros((1,) + shape, np.uint8)
    m[0, 5, 6, 6] = 1
    u = oracle.uroi(m, shape, GOLDEN["voxel_spacing_mm"]["value"],
                    GOLDEN["uroi_margin_mm"]["value"])
    assert u[5, 6, 11] == 1 and u[5, 6, 12] == 0
    assert u[9, 6, 6] == 1 and u[10, 6, 6] == 0


# -------------------------------------------------------------------- sign ---
def test_auto_sign_follows_roi_contrast():
    T = np.full((12, 12, 12), 40.0)
    m = np.zeros((2, 12, 12, 12), np.uint8)
    m[0, 4:8, 4:8, 4:8] = 1
    m[1, 1:3, 8:11, 8:11] = 1
    T[4:8, 4:8, 4:8] = 55.0     # brighter
    T[1:3, 8:11, 8:11] = 25.0   # darker
    assert oracle.auto_sign(T, m) == [1, -1]


def shell_sign_fixture(flip=False):
    """A 4^3 ROI (value 0) wrapped in layers at Chebyshev distance 1 (-100),
    2 (+110) and 3 or more (-1000) from it, or all values negated.  The shell
    of the sign rule (distance 1 or 2) averages +38.75 (-38.75 flipped), but a
    shell of distance 1 alone averages -100, one of distance 3 about -503,
    and a Euclidean shell of radius 2 (the faces of layer 2 only) -18.7: each
    of those readings gives the other sign."""
    n = 16
    idx = np.indices((n, n, n))
    d = np.max(np.maximum(np.maximum(6 - idx, idx - 9), 0), axis=0)   # Chebyshev distance to [6, 9]^3
    T = np.select([d == 0, d == 1, d == 2], [0.0, -100.0, 110.0], default=-1000.0)
    if flip:
        T = -T
    m = (d == 0).astype(np.uint8)[None]
    return T, m


@pytest.mark.parametrize("flip, sign", [(False, -1), (True, 1)])
def test_auto_sign_shell_is_chebyshev_distance_two(flip, sign):
    T, m = shell_sign_fixture(flip)
    assert oracle.auto_sign(T, m) == [sign]


# ------------------------------------------------------------------ RMS-ID ---
def test_rms_id_brute_force_over_enumerated_uroi_voxels():
    w = RNG.normal(size=(4, 5, 6))
    T = RNG.normal(size=(4, 5, 6))
    ur = RNG.integers(0, 2, size=(4, 5, 6)).astype(np.uint8)
    s, c = 0.0, 0
    for (z, y, x) in np.argwhere(ur):
        s += (w[z, y, x] - T[z, y, x]) ** 2
        c += 1
    v, cnt = oracle.rms_id(w, T, ur)
    assert cnt == c
    assert abs(v - math.sqrt(s / c)) < 1e-13
    assert oracle.rms_id(w, T, np.zeros_like(ur)) == (0.0, 0)


# --------------------------------------------------------------- stop test ---
def test_window10_reading():
    eps = GOLDEN["stop_eps"]["value"]
    lin = [10 - 1e-3 * n for n in range(40)]
    assert not any(oracle.stop_test(lin, n, oracle.STOP_WINDOW10, eps) for n in range(40))
    flat = [10 - 0.5 * min(n, 5) for n in range(40)]
    first = next(n for n in range(40) if oracle.stop_test(flat, n, oracle.STOP_WINDOW10, eps))
    assert first == 15


def test_paper_literal_reading_fires_at_first_chance_on_decelerating_decay():
    """The printed criterion l^(k-10) - l^(k) <= eps is negative whenever the
    RMS-ID decreases and decelerates, so it stops at k = 11."""
    d = [100 * 0.9 ** n for n in range(40)]
    first = next(n for n in range(40) if oracle.stop_test(d, n, oracle.STOP_PAPER_LITERAL, 1e-4))
    assert first == 11
    assert not any(oracle.stop_test(d, n, oracle.STOP_FIXED, 1e-4) for n in range(40))
