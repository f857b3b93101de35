"""Pins of the oracle's venk limiter (Venkatakrishnan 1995, the smooth
limiter of the limiter table, two ghost cells) in its 1D form: the central
increment (c - a)/4 from the cell centre to each face, limited by the smooth
function of the ratio of the stencil's range to that increment, the smaller
factor of the two faces for the cell.  Facts its definition fixes, none
retyping its formula:

* a value worked out by hand with fractions: the stencil (0, 1, 3/2) has the
  increment 3/8, range ratios 4/3 (right) and 8/3 (left), factors 20/23 and
  56/53, so the faces are 1 +- 15/46;
* linear data are reconstructed exactly (both ratios are 2, where the factor
  is 1);
* at an extremum, and next to a flat run, the faces keep the cell value;
* no new extrema (each face stays between its cell and its neighbour);
* mirror symmetry and invariance under affine maps of the data;
* second order on a smooth wave in L1, between minmod and vanleer in error.
"""
from fractions import Fraction

import numpy as np

from test_oracle_limiters5 import _averages


def test_worked_example(orc):
    wl_, wr_ = orc.reconstruct("venk", np.array([0.0, 1.0, 1.5]))
    assert abs(wl_[1] - float(Fraction(61, 46))) < 4e-16
    assert abs(wr_[1] - float(Fraction(31, 46))) < 4e-16
    # the same cell reached from a stencil whose left factor binds instead
    wl_, wr_ = orc.reconstruct("venk", np.array([-0.5, 0.0, 1.0]))
    assert abs(wl_[1] - float(Fraction(15, 46))) < 4e-16
    assert abs(wr_[1] + float(Fraction(15, 46))) < 4e-16


def test_linear_data_exact(orc):
    x = np.arange(10.0)
    for w in (2.0 + 0.5 * x, 1.0 - 3.0 * x):
        wl_, wr_ = orc.reconstruct("venk", w)
        s = 0.5 * (w[1] - w[0])
        np.testing.assert_allclose(wl_[1:-1], w[1:-1] + s, rtol=0, atol=1e-14)
        np.testing.assert_allclose(wr_[1:-1], w[1:-1] - s, rtol=0, atol=1e-14)


def test_extrema_and_flat_runs_keep_the_cell_value(orc):
    for row in ([0.0, 1.0, 0.5], [2.0, 1.0, 3.0], [1.0, 1.0, 4.0], [4.0, 2.0, 2.0]):
        wl_, wr_ = orc.reconstruct("venk", np.array(row))
        assert wl_[1] == row[1] and wr_[1] == row[1], row


def test_no_new_extrema(orc):
    rng = np.random.Generator(np.random.PCG64(21))
    w = rng.uniform(-1.0, 1.0, 500)
    wl_, wr_ = orc.reconstruct("venk", w)
    for i in range(1, 499):
        assert min(w[i], w[i + 1]) - 1e-15 <= wl_[i] <= max(w[i], w[i + 1]) + 1e-15
        assert min(w[i], w[i - 1]) - 1e-15 <= wr_[i] <= max(w[i], w[i - 1]) + 1e-15


def test_mirror_and_affine_invariance(orc):
    rng = np.random.Generator(np.random.PCG64(22))
    a = rng.uniform(0.5, 2.0, 60)
    wl_, wr_ = orc.reconstruct("venk", a)
    wl2, wr2 = orc.reconstruct("venk", a[::-1].copy())
    i = np.arange(1, 59)
    np.testing.assert_allclose(wl_[i], wr2[::-1][i], rtol=0, atol=1e-15)
    np.testing.assert_allclose(wr_[i], wl2[::-1][i], rtol=0, atol=1e-15)
    for s, t in ((2.0, 0.0), (-1.0, 0.0), (0.5, 3.0)):
        wl3, wr3 = orc.reconstruct("venk", s * a + t)
        np.testing.assert_allclose(wl3[i], s * wl_[i] + t, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(wr3[i], s * wr_[i] + t, rtol=1e-13, atol=1e-13)


def test_second_order_on_a_smooth_wave(orc):
    errs = {}
    for lim in ("venk", "minmod", "vanleer"):
        e = []
        for n in (64, 128, 256):
            F = lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi)  # noqa: E731
            a, xe = _averages(F, n)
            wl_, wr_ = orc.reconstruct(lim, a)
            i = np.arange(1, n - 1)
            d = np.concatenate([wl_[i] - np.sin(2 * np.pi * xe[i + 1]),
                                wr_[i] - np.sin(2 * np.pi * xe[i])])
            e.append(np.abs(d).mean())
        errs[lim] = e
    o = np.log2(np.array(errs["venk"][:-1]) / np.array(errs["venk"][1:]))
    assert o.min() > 1.8, (errs, o)
    assert errs["venk"][-1] < errs["minmod"][-1], errs
