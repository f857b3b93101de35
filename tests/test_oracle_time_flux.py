"""Pins of the oracle's wider scheme family: the TVD Lax-Friedrichs flux and the
SSPRK(4,3) / SSPRK(5,4) time steppers of the paper's scheme tables (Sect. 3).

None of these retypes an oracle formula: the stage coefficients are measured
from the oracle's own stage output and checked for the order they must reach
on a nonlinear ODE, the in-place buffer schedule of orc_run is checked against
a composition of stages into separate arrays, and the flux is checked where it
must coincide with HLL, for rotation covariance and by convergence to the exact
Euler solution.
"""
import math

import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl
from util import euler_exact, rel_l1


def _state(rho, u, v, w, p, bx, by, bz, psi=0.0):
    return np.array([rho, u, v, w, p, bx, by, bz, psi], float)


def _rand_state(rng):
    return np.concatenate([rng.uniform(0.5, 2.0, 1), rng.uniform(-1, 1, 3),
                           rng.uniform(0.3, 2.0, 1), rng.uniform(-1.5, 1.5, 3),
                           rng.uniform(-0.1, 0.1, 1)])


# ----------------------------------------------------------------------------
# TVD Lax-Friedrichs
# ----------------------------------------------------------------------------

def test_tvdlf_consistency_with_physical_flux(orc):
    # equal states: every solver returns the physical flux
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(40):
        w = _rand_state(rng)
        for d in range(3):
            f1 = orc.face_flux("tvdlf", 1, 5 / 3, 1.3, d, w, w)
            f2 = orc.face_flux("hll", 1, 5 / 3, 1.3, d, w, w)
            np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-13)


def test_tvdlf_equals_hll_for_symmetric_speeds(orc):
    # u_L = u_R = 0 and equal fast speeds: the Davis bounds are -c_f, +c_f and
    # HLL reduces to the local Lax-Friedrichs flux
    rng = np.random.Generator(np.random.PCG64(12))
    for _ in range(40):
        rho, p = rng.uniform(0.5, 2), rng.uniform(0.3, 2)
        bx, by, bz = rng.uniform(-1.5, 1.5, 3)
        wl_ = _state(rho, 0.0, rng.uniform(-1, 1), rng.uniform(-1, 1), p, bx, by, bz)
        wr_ = _state(rho, 0.0, rng.uniform(-1, 1), rng.uniform(-1, 1), p, bx, -by, -bz)
        f1 = orc.face_flux("tvdlf", 0, 1.4, 1.0, 0, wl_, wr_)
        f2 = orc.face_flux("hll", 0, 1.4, 1.0, 0, wl_, wr_)
        np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-13)


def test_tvdlf_more_diffusive_than_hll(orc):
    # a stationary contact: HLL with its tighter speed bounds diffuses less
    wl_ = _state(1.0, 0.3, 0, 0, 1.0, 0.0, 0.0, 0.0)
    wr_ = _state(0.2, 0.3, 0, 0, 1.0, 0.0, 0.0, 0.0)
    f_lf = orc.face_flux("tvdlf", 0, 1.4, 1.0, 0, wl_, wr_)
    f_hll = orc.face_flux("hll", 0, 1.4, 1.0, 0, wl_, wr_)
    exact_mass = 0.3 * 1.0  # upwind (left) mass flux of the moving contact
    assert abs(f_lf[0] - exact_mass) > abs(f_hll[0] - exact_mass)


def test_tvdlf_rotation_covariance(orc):
    rng = np.random.Generator(np.random.PCG64(13))
    perm = lambda w: np.array([w[0], w[3], w[1], w[2], w[4], w[7], w[5], w[6], w[8]])
    for _ in range(30):
        a, b = _rand_state(rng), _rand_state(rng)
        fx = orc.face_flux("tvdlf", 1, 5 / 3, 2.0, 0, a, b)
        fy = orc.face_flux("tvdlf", 1, 5 / 3, 2.0, 1, perm(a), perm(b))
        np.testing.assert_allclose(fy, perm(fx), rtol=1e-13, atol=1e-14)


def test_tvdlf_sod_converges_to_euler_exact(orc):
    errs = []
    for n in (200, 400, 800):
        W = wl.riemann_1d((1.0, 0, 0, 0, 1.0, 0, 0), (0.125, 0, 0, 0, 0.1, 0, 0), n=n,
                          gamma=1.4, bx=0.0, t_end=0.2, flux="tvdlf", time="ssprk3")
        U, t, ns, st = orc.mesh_for(W).run(W.U, 0.2)
        x = (np.arange(n) + 0.5) / n
        ex = euler_exact((1.0, 0, 1.0), (0.125, 0, 0.1), 1.4, x, 0.2, x0=0.5)
        errs.append(np.abs(U[0, 0] - ex[0]).mean())
    assert errs[-1] < 8e-3, errs
    assert errs[0] / errs[-1] > 2.0, errs


# ----------------------------------------------------------------------------
# SSPRK(4,3), SSPRK(5,4)
# ----------------------------------------------------------------------------

def _euler_L(orc, m, U, ch):
    """L(U) from one SSPRK(2,2) stage 0 (out = U + dt L(U)) with dt = 1e-3."""
    m0 = orc.Mesh(dataclass_replace(m.cfg, time="ssprk2"), m.instances, m.meta)
    out, st = m0.stage(0, 1e-3, ch, U, U)
    return (out - U) / 1e-3


def dataclass_replace(cfg, **kw):
    import dataclasses
    return dataclasses.replace(cfg, **kw)


def _smooth_case(time):
    W = wl.cp_alfven(16)
    W.cfg.time = time
    W.cfg.glm = False
    return W


@pytest.mark.parametrize("time", ["ssprk43", "ssprk54"])
def test_stage_applies_tabulated_coefficients(orc, time):
    # measure (a, b, c) of every stage from the stage output itself:
    # out - b Uk = a U0 + (b c dt) L(Uk), least squares over all cells
    W = _smooth_case(time)
    m = orc.mesh_for(W)
    rng = np.random.Generator(np.random.PCG64(21))
    U0 = W.U.copy()
    Uk = W.U * (1 + 0.01 * rng.standard_normal(W.U.shape))
    Uk[8] = 0.0
    U0[8] = 0.0
    L = _euler_L(orc, m, Uk, 1.0)
    dt = 2e-3
    for k in range(orc.num_stages(time)):
        co = orc.stage_coeffs6(time, k)
        out, st = m.stage(k, dt, 1.0, U0, Uk)
        assert st == 0
        # unknowns (a, b, bc): out = a U0 + b Uk + bc dt L
        A = np.stack([U0[:8].ravel(), Uk[:8].ravel(), dt * L[:8].ravel()], axis=1)
        sol, *_ = np.linalg.lstsq(A, out[:8].ravel(), rcond=None)
        a, b, bc = sol
        assert abs(a - co[0]) < 1e-6 and abs(b - co[1]) < 1e-6, (k, sol, co)
        assert abs(bc - co[1] * co[2]) < 1e-4, (k, sol, co)
        if not (time == "ssprk54" and k == 4):  # there U0 = w carries the rest
            assert abs(co[0] + co[1] - 1.0) < 1e-14  # consistency of each stage
    if time == "ssprk54":
        U2 = W.U * (1 + 0.01 * rng.standard_normal(W.U.shape))
        U2[8] = 0.0
        out, out2, st = m.stage2(3, dt, 1.0, U0, Uk, U2)
        co = orc.stage_coeffs6(time, 3)
        A = np.stack([U2[:8].ravel(), Uk[:8].ravel(), dt * L[:8].ravel()], axis=1)
        (a2, b2, bc2), *_ = np.linalg.lstsq(A, out2[:8].ravel(), rcond=None)
        assert abs(a2 - co[3]) < 1e-6 and abs(b2 - co[4]) < 1e-6
        assert abs(bc2 - co[4] * co[5]) < 1e-4
        # the last step u5 = w + b4 (u4 + c4 dt L(u4)) keeps constants:
        # the weights of u2, u3 (in w) and u4 add up to one
        co4 = orc.stage_coeffs6(time, 4)
        assert co4[0] == 1.0 and abs(co[3] + co[4] + co4[1] - 1.0) < 1e-12


def _ode_step(orc, time, f, y, h):
    """One step of the Shu-Osher scheme defined by the oracle's coefficient
    table, on y' = f(y); stage inputs as the GPU and the oracle chain them."""
    ns = orc.num_stages(time)
    y0 = y
    cur = y
    w = None
    u2 = None
    for k in range(ns):
        a, b, c, a2, b2, c2 = orc.stage_coeffs6(time, k)
        U0 = w if (time == "ssprk54" and k == 4) else y0
        e = cur + c * h * f(cur)
        nxt = e if (a == 0.0 and b == 1.0) else a * U0 + b * e
        if b2 != 0.0:
            w = a2 * u2 + b2 * (cur + c2 * h * f(cur))
        if k == 1:
            u2 = nxt
        cur = nxt
    return cur


@pytest.mark.parametrize("time,order", [("ssprk2", 2), ("ssprk3", 3), ("ssprk43", 3),
                                        ("ssprk54", 4)])
def test_ssprk_nonlinear_order(orc, time, order):
    # nonlinear pendulum y'' = -sin y: global error ~ h^order
    f = lambda y: np.array([y[1], -math.sin(y[0])])

    def solve(h):
        y = np.array([1.0, 0.0])
        for _ in range(int(round(2.0 / h))):
            y = _ode_step(orc, time, f, y, h)
        return y

    ref = solve(1e-3 if order < 4 else 5e-3)
    e = [np.abs(solve(h) - ref).max() for h in (0.1, 0.05, 0.025)]
    p = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(p) > order - 0.3, (time, e, p)


@pytest.mark.parametrize("time", ["ssprk43", "ssprk54"])
def test_stability_polynomial(orc, time):
    # y' = z y: R(z) = sum_j g_j z^j with g_j = 1/j! up to the scheme's order;
    # SSPRK(4,3) of Spiteri & Ruuth has g_4 = 1/48
    zs = np.linspace(-0.5, 0.5, 11)
    R = np.array([_ode_step(orc, time, lambda y, z=z: z * y, np.array([1.0]), 1.0)[0]
                  for z in zs])
    deg = orc.num_stages(time)
    g = np.polynomial.polynomial.polyfit(zs, R, deg)
    want = [1, 1, 0.5, 1 / 6]
    if time == "ssprk43":
        want += [1 / 48]
    else:
        want += [1 / 24]
    np.testing.assert_allclose(g[:len(want)], want, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("time", ["ssprk43", "ssprk54"])
def test_run_buffer_schedule_matches_separate_arrays(orc, time):
    # orc_run reuses three registers in place; a composition of stages into
    # fresh arrays must give the same step bit for bit
    W = wl.cp_alfven(32)
    W.cfg.time = time
    m = orc.mesh_for(W, 4)
    dt, ch = m.cfl(W.U)
    u0 = W.U.copy()
    outs = [None] * 6
    cur = u0
    w = None
    for k in range(orc.num_stages(time)):
        U0 = w if (time == "ssprk54" and k == 4) else u0
        if time == "ssprk54" and k == 3:
            nxt, w, st = m.stage2(k, dt, ch, U0, cur, outs[2])
        else:
            nxt, st = m.stage(k, dt, ch, U0, cur)
        assert st == 0
        outs[k + 1] = nxt
        cur = nxt
    U, t, ns, st = m.run(W.U, 1.0, maxsteps=1)
    assert ns == 1 and st == 0
    assert np.array_equal(U, cur)
    # conservation (periodic box): every stage is a convex combination
    s0, s1 = m.sums(u0), m.sums(U)
    for v in range(8):
        scale = max(abs(s0[0, v]), np.abs(u0[v]).mean())
        assert abs(s1[0, v] - s0[0, v]) <= 1e-13 * scale


@pytest.mark.parametrize("time", ["ssprk43", "ssprk54"])
def test_higher_stage_schemes_on_cp_wave(orc, time):
    # same smooth nonlinear wave: the error stays at the level of SSPRK(3,3)
    # (space-dominated) and converges at second order with the grid
    def err(n, tm):
        W = wl.cp_alfven(n)
        W.cfg.time = tm
        U, t, ns, st = orc.mesh_for(W, 8).run(W.U, 1 / math.sqrt(2))
        assert st == 0
        _, _, _, Ue = wl.cp_alfven_exact(n, 1 / math.sqrt(2))
        return rel_l1(U[7], Ue[7])
    e32, e64 = err(32, time), err(64, time)
    assert math.log2(e32 / e64) > 1.7, (e32, e64)
    assert e64 < 1.2 * err(64, "ssprk3")


# ----------------------------------------------------------------------------
# HLLC (Li 2005 three-wave solver for MHD)
# ----------------------------------------------------------------------------

def test_hllc_consistency_and_rotation(orc):
    rng = np.random.Generator(np.random.PCG64(31))
    perm = lambda w: np.array([w[0], w[3], w[1], w[2], w[4], w[7], w[5], w[6], w[8]])
    for _ in range(40):
        w = _rand_state(rng)
        for d in range(3):
            np.testing.assert_allclose(orc.face_flux("hllc", 1, 5 / 3, 1.3, d, w, w),
                                       orc.face_flux("hll", 1, 5 / 3, 1.3, d, w, w),
                                       rtol=1e-12, atol=1e-13)
        a, b = _rand_state(rng), _rand_state(rng)
        fx = orc.face_flux("hllc", 1, 5 / 3, 2.0, 0, a, b)
        fy = orc.face_flux("hllc", 1, 5 / 3, 2.0, 1, perm(a), perm(b))
        np.testing.assert_allclose(fy, perm(fx), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("bx", [0.0, 0.7])
def test_hllc_resolves_stationary_contact(orc, bx):
    # density jump at rest with continuous p and B: the contact must not move
    # (zero mass flux, momentum flux p_T - B_x^2); HLL smears it
    wl_ = _state(1.0, 0.0, 0, 0, 1.0, bx, 0.4, -0.2)
    wr_ = _state(0.1, 0.0, 0, 0, 1.0, bx, 0.4, -0.2)
    f = orc.face_flux("hllc", 0, 1.4, 1.0, 0, wl_, wr_)
    assert abs(f[0]) < 1e-14
    pt = 1.0 + 0.5 * (bx * bx + 0.16 + 0.04)
    assert abs(f[1] - (pt - bx * bx)) < 1e-13
    assert abs(orc.face_flux("hll", 0, 1.4, 1.0, 0, wl_, wr_)[0]) > 1e-3


def test_hllc_moving_contact_b0(orc):
    # B = 0: HLLC is the Euler HLLC of Toro, exact for an isolated moving contact
    wl_ = _state(1.0, 0.4, 0.1, -0.3, 0.8, 0, 0, 0)
    wr_ = _state(0.3, 0.4, 0.1, -0.3, 0.8, 0, 0, 0)
    f = orc.face_flux("hllc", 0, 1.4, 1.0, 0, wl_, wr_)
    np.testing.assert_allclose(f[:5], [0.4, 0.4 * 0.4 + 0.8, 0.4 * 0.1, 0.4 * -0.3,
                                       (0.8 / 0.4 + 0.5 * (0.16 + 0.01 + 0.09) + 0.8) * 0.4],
                               rtol=1e-13)


def test_hllc_sod_converges_and_beats_hll(orc):
    errs = {}
    for flux in ("hllc", "hll"):
        e = []
        for n in (200, 400, 800):
            W = wl.riemann_1d((1.0, 0, 0, 0, 1.0, 0, 0), (0.125, 0, 0, 0, 0.1, 0, 0), n=n,
                              gamma=1.4, bx=0.0, t_end=0.2, flux=flux, time="ssprk3")
            U, t, ns, st = orc.mesh_for(W).run(W.U, 0.2)
            x = (np.arange(n) + 0.5) / n
            ex = euler_exact((1.0, 0, 1.0), (0.125, 0, 0.1), 1.4, x, 0.2, x0=0.5)
            e.append(np.abs(U[0, 0] - ex[0]).mean())
        errs[flux] = e
    assert errs["hllc"][-1] < 4e-3 and errs["hllc"][0] / errs["hllc"][-1] > 2.5
    assert errs["hllc"][-1] < errs["hll"][-1]  # the contact is sharper
