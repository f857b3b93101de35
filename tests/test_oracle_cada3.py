"""Pins of the oracle's cada3 limiter (Cada & Torrilhon 2009, the compact
third-order limiter of the limiter table, two ghost cells) against facts that
its definition fixes, none retyping its formula:

* where the slope ratio theta = dm/dp lies in [0.4, 2.8] it is the unlimited
  third-order (kappa = 1/3) reconstruction: exact interface values of
  quadratics, and identical to koren (whose third-order range contains it);
* third order in L1 on the interface values of a smooth periodic wave
  (extrema included), second order in the maximum norm (the cells next to an
  extremum, where its cap of 1.6 or its extremum branch binds);
* unlike the TVD limiters it keeps a slope at an isolated extremum;
* no new extrema: each face value stays within the range of its 3-cell
  stencil; a step (theta = 0 or infinite) gives the cell value;
* mirror symmetry and invariance under affine maps of the data;
* in whole runs, a periodic density wave converges at better than second
  order, with an error comparable to koren's.

This is the limiter function of the compact third-order limiter alone: the
grid-scale smoothness switch that Cada & Torrilhon add in front of it takes a
length parameter that the paper does not give, and is not used.
"""
import numpy as np
import pytest

from test_oracle_limiters5 import _averages, _wave_error


def test_quadratic_interface_values_exact_in_the_smooth_range(orc):
    # p(x) = 2 + x + 3 x^2 on [0.3, 1.3]: monotone, dm/dp within [0.4, 2.8]
    p = lambda x: 2 + x + 3 * x * x  # noqa: E731
    P = lambda x: 2 * x + x * x / 2 + x ** 3  # noqa: E731
    a, xe = _averages(P, 24, 0.3, 1.3)
    dm, dp = a[1:-1] - a[:-2], a[2:] - a[1:-1]
    th = dm / dp
    assert th.min() > 0.4 and th.max() < 2.8
    wl_, wr_ = orc.reconstruct("cada3", a)
    i = np.arange(1, 23)
    np.testing.assert_allclose(wl_[i], p(xe[i + 1]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(wr_[i], p(xe[i]), rtol=0, atol=1e-13)
    wk, wkr = orc.reconstruct("koren", a)
    np.testing.assert_allclose(wl_[i], wk[i], rtol=0, atol=1e-14)
    np.testing.assert_allclose(wr_[i], wkr[i], rtol=0, atol=1e-14)


def test_third_order_in_l1_on_a_smooth_wave(orc):
    errs = {"L1": [], "Linf": []}
    ns = (64, 128, 256)
    for n in ns:
        F = lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi)  # noqa: E731
        a, xe = _averages(F, n)
        wl_, wr_ = orc.reconstruct("cada3", a)
        i = np.arange(1, n - 1)
        d = np.concatenate([wl_[i] - np.sin(2 * np.pi * xe[i + 1]),
                            wr_[i] - np.sin(2 * np.pi * xe[i])])
        errs["L1"].append(np.abs(d).mean())
        errs["Linf"].append(np.abs(d).max())
    o1 = np.log2(np.array(errs["L1"][:-1]) / np.array(errs["L1"][1:]))
    oi = np.log2(np.array(errs["Linf"][:-1]) / np.array(errs["Linf"][1:]))
    assert o1.min() > 2.9, (errs, o1)
    assert oi.min() > 1.9, (errs, oi)


def test_no_new_extrema_and_steps(orc):
    rng = np.random.Generator(np.random.PCG64(12))
    a = rng.uniform(-1.0, 1.0, 400)
    wl_, wr_ = orc.reconstruct("cada3", a)
    for i in range(1, 399):
        lo, hi = a[i - 1:i + 2].min(), a[i - 1:i + 2].max()
        assert lo - 1e-15 <= wl_[i] <= hi + 1e-15 and lo - 1e-15 <= wr_[i] <= hi + 1e-15
    # a step: the cells on either side keep their value at the step
    s = np.where(np.arange(20) < 10, 1.0, 5.0)
    wl_, wr_ = orc.reconstruct("cada3", s)
    assert wl_[9] == 1.0 and wr_[10] == 5.0
    # an isolated extremum keeps a slope (TVD limiters return the cell value)
    wl_, wr_ = orc.reconstruct("cada3", np.array([0.0, 1.0, 0.0]))
    assert 0.0 < wl_[1] < 1.0 and wl_[1] == wr_[1]
    wk, _ = orc.reconstruct("koren", np.array([0.0, 1.0, 0.0]))
    assert wk[1] == 1.0


def test_mirror_and_affine_invariance(orc):
    rng = np.random.Generator(np.random.PCG64(13))
    a = rng.uniform(0.5, 2.0, 50)
    wl_, wr_ = orc.reconstruct("cada3", a)
    wl2, wr2 = orc.reconstruct("cada3", a[::-1].copy())
    i = np.arange(1, 49)
    np.testing.assert_array_equal(wl_[i], wr2[::-1][i])
    np.testing.assert_array_equal(wr_[i], wl2[::-1][i])
    for s, t in ((2.0, 0.0), (-1.0, 0.0), (0.5, 3.0)):
        wl3, wr3 = orc.reconstruct("cada3", s * a + t)
        np.testing.assert_allclose(wl3[i], s * wl_[i] + t, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(wr3[i], s * wr_[i] + t, rtol=1e-13, atol=1e-13)


def test_density_wave_converges(orc):
    e = [_wave_error(orc, n, "cada3") for n in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders.min() > 2.1, (e, orders)
    ek = _wave_error(orc, 128, "koren")
    ev = _wave_error(orc, 128, "vanleer")
    assert e[-1] < 1.5 * ek and e[-1] < 0.5 * ev, (e, ek, ev)


def test_saturation_for_steep_ratios(orc):
    # Cada & Torrilhon's LimO3 caps the limiter function at 1.6: for slope
    # ratios theta = dm/dp above 2.8 (where the third-order phi3 = (2 + theta)/3
    # passes 1.6) the face increment no longer grows with dm, it stays
    # 1.6 dp / 2; just below 2.8 it still follows phi3 (continuous at 2.8)
    for theta in (3.0, 5.0, 10.0, 100.0):
        for dp in (1.0, -0.5):
            wl_, _ = orc.reconstruct("cada3", np.array([-theta * dp, 0.0, dp]))
            assert abs(wl_[1] - 0.8 * dp) < 1e-14 * abs(dp), (theta, dp, wl_[1])
    for theta in (2.0, 2.7):
        wl_, _ = orc.reconstruct("cada3", np.array([-theta, 0.0, 1.0]))
        assert abs(wl_[1] - (2.0 + theta) / 6.0) < 1e-14, (theta, wl_[1])
    lo, _ = orc.reconstruct("cada3", np.array([-2.8 * (1 - 1e-9), 0.0, 1.0]))
    hi, _ = orc.reconstruct("cada3", np.array([-2.8 * (1 + 1e-9), 0.0, 1.0]))
    assert abs(lo[1] - hi[1]) < 1e-9
