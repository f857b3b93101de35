"""Pins of the oracle's five-point limiters of the limiter table (mp5, weno5,
wenoz5, wenozp5; three ghost cells) against facts fixed by their definitions: exact
interface values of quadratics (any convex combination of the exact
third-order candidates) and, for mp5's fifth-order interface polynomial, of
monotone quartics; measured fifth order on smooth monotone data; no new
extrema across a jump; mirror symmetry; and, in whole runs, a third-order
(time-limited) advection of a density wave against second order for vanleer,
with the ghost width of three cells across block faces and level changes.
"""
import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl

LIMS5 = ["mp5", "weno5", "wenoz5", "wenozp5"]


def _averages(F, n, x0=0.0, x1=1.0):
    # exact cell averages from an antiderivative F; returns (averages, edges)
    h = (x1 - x0) / n
    xe = x0 + h * np.arange(n + 1)
    return (F(xe[1:]) - F(xe[:-1])) / h, xe


@pytest.mark.parametrize("lim", LIMS5)
def test_quadratic_interface_values_exact(orc, lim):
    # p(x) = 2 + x + 3 x^2 (monotone on [0, 1]); P its antiderivative
    p = lambda x: 2 + x + 3 * x * x  # noqa: E731
    P = lambda x: 2 * x + x * x / 2 + x ** 3  # noqa: E731
    a, xe = _averages(P, 24)
    wl_, wr_ = orc.reconstruct(lim, a)
    i = np.arange(2, 22)
    np.testing.assert_allclose(wl_[i], p(xe[i + 1]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(wr_[i], p(xe[i]), rtol=0, atol=1e-13)


def test_mp5_quartic_exact(orc):
    # the interface polynomial of mp5 is exact up to degree 4; on monotone data
    # the monotonicity constraint leaves it untouched
    p = lambda x: 1 + x + 0.3 * x ** 2 + 0.1 * x ** 3 + 0.05 * x ** 4  # noqa: E731
    P = lambda x: x + x ** 2 / 2 + 0.1 * x ** 3 + 0.025 * x ** 4 + 0.01 * x ** 5  # noqa: E731
    a, xe = _averages(P, 20)
    wl_, wr_ = orc.reconstruct("mp5", a)
    i = np.arange(2, 18)
    np.testing.assert_allclose(wl_[i], p(xe[i + 1]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(wr_[i], p(xe[i]), rtol=0, atol=1e-13)
    # weno5 is not (nonlinear weights): a different, finite error
    wl_, _ = orc.reconstruct("weno5", a)
    assert 1e-12 < np.abs(wl_[i] - p(xe[i + 1])).max() < 1e-5


def test_mp5_bound_by_hand(orc):
    # (0, 0, 0.1, 1, 1): the interface polynomial (0.1*47 + 27 - 3)/60 = 28.7/60
    # lies between v_i = 0.1 and v_i + minmod(0.9, 4 * 0.1) = 0.5: kept
    wl_, _ = orc.reconstruct("mp5", np.array([0.0, 0.0, 0.1, 1.0, 1.0]))
    assert wl_[2] == pytest.approx(28.7 / 60, rel=1e-15)
    # (0, 0, 0.05, 1, 1): 26.35/60 exceeds 0.05 + 4 * 0.05 = 0.25; the mixed-sign
    # second differences give minmod4 = 0, so the bounds are [0.05, 0.25] and
    # the result is the upper limit v_i + 4 (v_i - v_{i-1}) = 0.25
    wl_, _ = orc.reconstruct("mp5", np.array([0.0, 0.0, 0.05, 1.0, 1.0]))
    assert wl_[2] == pytest.approx(0.25, rel=1e-15)


@pytest.mark.parametrize("lim", LIMS5)
def test_fifth_order_on_smooth_data(orc, lim):
    errs = []
    for n in (32, 64, 128):
        a, xe = _averages(np.exp, n)
        wl_, _ = orc.reconstruct(lim, a)
        i = np.arange(3, n - 3)
        errs.append(np.abs(wl_[i] - np.exp(xe[i + 1])).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.7), orders
    wk, _ = orc.reconstruct("koren", _averages(np.exp, 64)[0])
    assert errs[1] < 1e-3 * np.abs(wk[3:61] - np.exp(_averages(np.exp, 64)[1][4:62])).max()


@pytest.mark.parametrize("lim", LIMS5)
def test_no_new_extrema_across_a_jump(orc, lim):
    # a jump on a monotone ramp (a ramp has no extremum, so a face value
    # outside its neighbours' range would be a new one)
    a = np.where(np.arange(40) < 17, 1.0, 3.0) + 0.002 * np.arange(40)
    wl_, wr_ = orc.reconstruct(lim, a)
    # weno5's eps = 1e-6 is comparable to the smoothness indicators of the
    # small ramp, so the jump keeps a weight of order 1e-6: essentially, not
    # strictly, non-oscillatory; mp5 and wenoz5 stay within round-off
    tol = 1e-5 if lim == "weno5" else 1e-12
    for i in range(2, 38):
        lo, hi = a[i - 2:i + 3].min(), a[i - 2:i + 3].max()
        assert lo - tol <= wl_[i] <= hi + tol and lo - tol <= wr_[i] <= hi + tol, (i, lim)
    if lim == "mp5":
        # mp5 keeps each face value between its two cells there
        for i in (15, 16, 17):
            assert min(a[i], a[i + 1]) - 1e-12 <= wl_[i] <= max(a[i], a[i + 1]) + 1e-12


@pytest.mark.parametrize("lim", LIMS5)
def test_mirror_symmetry(orc, lim):
    rng = np.random.Generator(np.random.PCG64(5))
    a = rng.uniform(0.5, 2.0, 30)
    wl_, wr_ = orc.reconstruct(lim, a)
    wl2, wr2 = orc.reconstruct(lim, a[::-1].copy())
    i = np.arange(2, 28)
    assert np.array_equal(wl_[i], wr2[::-1][i]) and np.array_equal(wr_[i], wl2[::-1][i])


def _density_wave(n, lim, bnx=16):
    # 1D periodic density wave in a uniform flow (an entropy mode): after one
    # period the exact solution is the initial state
    cfg = wl.Config(ndim=1, block_nx=(bnx, 1, 1), flux="hll", limiter=lim, time="ssprk3",
                    precision="fp64", glm=False, courant=0.6)
    inst = wl.Instance(base_blocks=(n // bnx, 1, 1), gamma=5.0 / 3.0)
    meta = wl.uniform_meta((n // bnx, 1, 1))

    def prim(inst, x, y, z):
        zero = np.zeros_like(x)
        return wl.conserved_from_primitive(inst.gamma, 1.0 + 0.2 * np.sin(2 * np.pi * x),
                                           1.0 + zero, zero, zero, 1.0 + zero, 0.5 + zero,
                                           zero, zero)
    U = wl._fill_from_function(cfg, [inst], meta, prim)
    return wl.Workload("density_wave", cfg, [inst], meta, U)


def _wave_error(orc, n, lim):
    W = _density_wave(n, lim)
    U, t, ns, st = orc.mesh_for(W).run(W.U, 1.0)
    assert st == 0 and abs(t[0] - 1.0) < 1e-14
    return np.abs(U[0] - W.U[0]).mean()


@pytest.mark.parametrize("lim", LIMS5)
def test_density_wave_converges_third_order(orc, lim):
    # SSPRK3 at a fixed Courant number caps the order at 3; vanleer gives 2.
    # The five-point spatial error is so small that it can cancel against the
    # time error at one resolution, so the order is taken over 32 -> 256.
    e = [_wave_error(orc, n, lim) for n in (32, 64, 128, 256)]
    order = np.log2(e[0] / e[-1]) / 3
    assert order > 2.7, (lim, e, order)
    ev = [_wave_error(orc, n, "vanleer") for n in (64, 128)]
    assert e[2] < 0.2 * ev[-1]


def test_ghost_width_three_across_levels(orc):
    # a five-point limiter widens the ghost fill to 3 cells, also across level
    # changes; a uniform flow stays uniform on an AMR mesh
    W = wl.small_amr_2d(field="uniform")
    W.cfg.limiter = "weno5"
    m = orc.mesh_for(W)
    assert m.ng == 3
    assert m.fill_ghosts(W.U).shape == (9, W.nblocks, (8 + 6) ** 2)
    dt, ch = m.cfl(W.U)
    out, st = m.stage(0, dt, ch, W.U, W.U)
    assert st == 0 and np.abs(out - W.U).max() < 1e-14 * np.abs(W.U).max()
    W.cfg.limiter = "vanleer"
    W.cfg.level_limiter = {2: "mp5"}
    assert orc.mesh_for(W).ng == 3
    W.cfg.level_limiter = None
    assert orc.mesh_for(W).ng == 2


def test_wenozp5_fifth_order_at_smooth_extrema(orc):
    # WENO-Z+ (Acker, Borges & Costa 2016) keeps fifth order where the first
    # derivative vanishes (a sine's extrema), with lambda = dx^(2/3) shrinking
    # with the grid
    errs = []
    for n in (40, 80, 160):
        F = lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi)  # noqa: E731
        a, xe = _averages(F, n)
        wl_, _ = orc.reconstruct("wenozp5", a, dx=1.0 / n)
        i = np.arange(3, n - 3)
        errs.append(np.abs(wl_[i] - np.sin(2 * np.pi * xe[i + 1])).max())
    oz = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert oz.min() > 4.5, (errs, oz)


def test_wenozp5_lambda_follows_the_cell_width(orc):
    # the added term lambda (beta_k + eps)/(tau5 + eps), lambda = dx^(2/3),
    # raises the weight of the less smooth candidates.  At a kink (where the
    # candidates' smoothness indicators are comparable) the face values next
    # to it move steadily with dx, by ~1e-3 between dx = 1e-9 and 0.5; the
    # faces whose stencils are all on one side do not move
    a = 0.1 * np.abs(np.arange(12) - 5.3)
    vals = np.array([orc.reconstruct("wenozp5", a, dx=dx)[0] for dx in (1e-9, 1e-3, 1e-1, 0.5)])
    assert np.all(np.diff(vals[:, 4]) < 0) and np.all(np.diff(vals[:, 5]) < 0)
    assert np.all(np.diff(vals[:, 6]) > 0)
    assert abs(vals[-1, 5] - vals[0, 5]) > 1e-3
    np.testing.assert_allclose(vals[:, 2], vals[0, 2], rtol=1e-14)
    # exact for linear data whatever lambda (equal smoothness indicators)
    lin = 0.5 + 0.25 * np.arange(12)
    for dx in (1e-3, 0.5):
        wl_, wr_ = orc.reconstruct("wenozp5", lin, dx=dx)
        i = np.arange(2, 10)
        np.testing.assert_allclose(wl_[i], lin[i] + 0.125, rtol=0, atol=1e-14)
        np.testing.assert_allclose(wr_[i], lin[i] - 0.125, rtol=0, atol=1e-14)


def test_wenozp5_exponent_two_at_a_jump(orc):
    # Next to a jump the stencil crossing it has tau5 ~ beta_2 ~ O(jump^2)
    # while the smooth ones have beta ~ (h p')^2: WENO-Z+ gives the crossing
    # candidate a weight ~ (beta_smooth / tau5)^2 relative to the smooth ones,
    # so the face value on the smooth side keeps the smooth (exact for
    # quadratics) reconstruction to ~1e-9 at h = 0.01; with the exponent 1 of
    # WENO-Z the weight is ~ beta_smooth / tau5 and the face is ~1e-5 off
    h, n, i = 0.01, 12, 6
    xe = 0.5 + h * np.arange(n + 1)
    a = (xe[1:] ** 3 - xe[:-1] ** 3) / (3 * h)  # cell averages of x^2
    a[i + 2:] += 1.0                              # a jump between cells i+1 and i+2
    wl_, _ = orc.reconstruct("wenozp5", a, dx=h)
    assert abs(wl_[i] - xe[i + 1] ** 2) < 1e-7
    wz, _ = orc.reconstruct("wenoz5", a, dx=h)
    assert abs(wz[i] - xe[i + 1] ** 2) > 1e-6  # the exponent-1 weights do not get there
