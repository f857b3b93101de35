"""Pins of the FP64 CPU oracle against facts fixed by mathematics and the paper.

None of these tests retypes an oracle formula and compares: each checks a
property that a dropped term, a wrong sign, a wrong index or a transposed
operand would break (exact solutions, conservation, Rankine-Hugoniot jumps,
linear-wave speeds, closed forms, symmetry, brute force).
"""
import math
import os

import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl
from util import (euler_exact, linear_mode, mhd_shock, mhd_shock_roots, paper_error,
                  rel_l1)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if line:
            out[line[0]] = line[1:]
    return out


def _prim_state(rho, u, v, w, p, bx, by, bz, psi=0.0):
    return np.array([rho, u, v, w, p, bx, by, bz, psi], float)


# ----------------------------------------------------------------------------
# limiters: closed forms, orders and ghost cells of the limiter table
# ----------------------------------------------------------------------------

def test_limiter_exact_on_linear(orc):
    x = np.arange(12.0)
    w = 0.3 + 0.7 * x
    for lim in ("minmod", "vanleer", "koren"):
        wl_, wr_ = orc.reconstruct(lim, w)
        np.testing.assert_allclose(wl_[1:-1], w[1:-1] + 0.35, rtol=0, atol=1e-14)
        np.testing.assert_allclose(wr_[1:-1], w[1:-1] - 0.35, rtol=0, atol=1e-14)


def test_koren_third_order_on_quadratic(orc):
    # cell averages of a monotone quadratic q(x) = x^2 + 5x on [i, i+1]; the
    # limiter is inactive there, so the face value must equal q(i+1) exactly
    i = np.arange(10.0)
    avg = ((i + 1) ** 3 - i ** 3) / 3.0 + 5.0 * ((i + 1) ** 2 - i ** 2) / 2.0
    wl_, wr_ = orc.reconstruct("koren", avg)
    q = lambda x: x * x + 5 * x
    np.testing.assert_allclose(wl_[1:-1], q(i[1:-1] + 1), rtol=1e-13)
    np.testing.assert_allclose(wr_[1:-1], q(i[1:-1]), rtol=1e-13)
    wl2, _ = orc.reconstruct("vanleer", avg)
    assert np.abs(wl2[1:-1] - q(i[1:-1] + 1)).max() > 1e-3  # second order only


def test_limiter_orders_match_table(orc):
    table = _golden("limiter_table.txt")
    f = lambda x: np.tanh(2 * x) + 0.1 * x  # monotone, smooth
    for lim, (order, ghosts) in table.items():
        errs = []
        for n in (40, 80, 160, 320):
            h = 2.0 / n
            edges = -1 + h * np.arange(n + 1)
            F = lambda x: np.log(np.cosh(2 * x)) / 2 + 0.05 * x * x
            avg = (F(edges[1:]) - F(edges[:-1])) / h
            wl_, _ = orc.reconstruct(lim, avg)
            errs.append(np.abs(wl_[1:-1] - f(edges[2:-1])).max())
        p = math.log2(errs[-2] / errs[-1])
        assert p > float(order) - 0.35, (lim, p, errs)
        # the stencil reaches one cell on each side: two ghost cells give every
        # face of the block both of its states
        assert int(ghosts) == 2


def test_limiter_tvd_and_extrema(orc):
    rng = np.random.Generator(np.random.PCG64(11))
    w = rng.uniform(-1, 1, 400)
    for lim in ("minmod", "vanleer", "koren"):
        wl_, wr_ = orc.reconstruct(lim, w)
        for i in range(1, 399):
            lo, hi = min(w[i], w[i + 1]), max(w[i], w[i + 1])
            assert lo - 1e-15 <= wl_[i] <= hi + 1e-15
            lo, hi = min(w[i], w[i - 1]), max(w[i], w[i - 1])
            assert lo - 1e-15 <= wr_[i] <= hi + 1e-15
            if (w[i] - w[i - 1]) * (w[i + 1] - w[i]) <= 0:
                assert wl_[i] == w[i] and wr_[i] == w[i]
        # mirror: reversing the data swaps the two face states
        wl2, wr2 = orc.reconstruct(lim, w[::-1].copy())
        np.testing.assert_allclose(wl2[1:-1], wr_[::-1][1:-1], rtol=0, atol=1e-15)


def test_vanleer_symmetric_limiter(orc):
    # phi(r)/r = phi(1/r): the slope is symmetric in its two differences
    for dm, dp in [(0.3, 1.7), (2.0, 0.1), (1e-3, 5.0)]:
        a = np.array([0.0, dm, dm + dp])
        b = np.array([0.0, dp, dp + dm])
        la, _ = orc.reconstruct("vanleer", a)
        lb, _ = orc.reconstruct("vanleer", b)
        assert abs((la[1] - dm) - (lb[1] - dp)) < 1e-14
        assert abs((la[1] - dm) - dm * dp / (dm + dp)) < 1e-14


# ----------------------------------------------------------------------------
# pointwise physics
# ----------------------------------------------------------------------------

def test_prim_cons_roundtrip_and_energy(orc):
    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(50):
        w = np.concatenate([rng.uniform(0.1, 2, 1), rng.uniform(-2, 2, 3),
                            rng.uniform(0.1, 2, 1), rng.uniform(-2, 2, 4)])
        g = rng.choice([5 / 3, 1.4])
        u = orc.prim_to_cons(g, w)
        # energy = thermal + kinetic + magnetic (magnetic pressure B^2/2)
        ke = 0.5 * w[0] * (w[1:4] ** 2).sum()
        me = 0.5 * (w[5:8] ** 2).sum()
        assert abs(u[4] - (w[4] / (g - 1) + ke + me)) < 1e-13 * u[4]
        np.testing.assert_allclose(orc.cons_to_prim(g, u), w, rtol=1e-12, atol=1e-13)


def test_fast_speed_textbook_form(orc):
    rng = np.random.Generator(np.random.PCG64(2))
    for _ in range(100):
        w = np.concatenate([rng.uniform(0.1, 2, 1), rng.uniform(-2, 2, 3),
                            rng.uniform(0.01, 2, 1), rng.uniform(-2, 2, 3), [0.0]])
        g = 5 / 3
        for d in range(3):
            a2 = g * w[4] / w[0]
            b2 = (w[5:8] ** 2).sum() / w[0]
            bn2 = w[5 + d] ** 2 / w[0]
            ref = math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)))
            assert abs(orc.fast_speed(g, w, d) - ref) < 1e-12 * ref
    # B = 0: sound speed; B along the normal: max(a, b)
    w = _prim_state(2.0, 0, 0, 0, 3.0, 0, 0, 0)
    assert abs(orc.fast_speed(1.4, w, 0) - math.sqrt(1.4 * 3 / 2)) < 1e-14
    w = _prim_state(1.0, 0, 0, 0, 0.6, 3.0, 0, 0)
    assert abs(orc.fast_speed(5 / 3, w, 0) - 3.0) < 1e-14


# ----------------------------------------------------------------------------
# Riemann solvers
# ----------------------------------------------------------------------------

def _rand_state(rng):
    return np.concatenate([rng.uniform(0.2, 2, 1), rng.uniform(-1, 1, 3), rng.uniform(0.2, 2, 1),
                           rng.uniform(-1.5, 1.5, 3), rng.uniform(-0.1, 0.1, 1)])


def test_flux_consistency_hll_equals_hlld(orc):
    # equal states: both solvers must return the same physical flux
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(50):
        w = _rand_state(rng)
        for d in range(3):
            for glm in (0, 1):
                f1 = orc.face_flux("hll", glm, 5 / 3, 1.3, d, w, w)
                f2 = orc.face_flux("hlld", glm, 5 / 3, 1.3, d, w, w)
                np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-13)


def test_flux_rotation_covariance(orc):
    # cyclic relabelling x->y->z of a state relabels the flux the same way
    rng = np.random.Generator(np.random.PCG64(4))
    perm = lambda w: np.array([w[0], w[3], w[1], w[2], w[4], w[7], w[5], w[6], w[8]])
    for _ in range(30):
        a, b = _rand_state(rng), _rand_state(rng)
        for fl in ("hll", "hlld"):
            fx = orc.face_flux(fl, 1, 5 / 3, 2.0, 0, a, b)
            fy = orc.face_flux(fl, 1, 5 / 3, 2.0, 1, perm(a), perm(b))
            np.testing.assert_allclose(fy, perm(fx), rtol=1e-13, atol=1e-14)


def test_hlld_resolves_stationary_contact(orc):
    # density jump only, u = 0, p, B, v_t continuous: HLLD returns zero mass
    # flux (exact contact), HLL diffuses it
    a = _prim_state(1.0, 0.0, 0.3, -0.2, 0.8, 0.7, 0.4, -0.5)
    b = a.copy()
    b[0] = 0.2
    f_hlld = orc.face_flux("hlld", 0, 5 / 3, 1.0, 0, a, b)
    f_hll = orc.face_flux("hll", 0, 5 / 3, 1.0, 0, a, b)
    assert abs(f_hlld[0]) < 1e-15
    assert abs(f_hll[0]) > 1e-2
    fa = orc.face_flux("hlld", 0, 5 / 3, 1.0, 0, a, a)
    np.testing.assert_allclose(f_hlld[1:8], fa[1:8], rtol=0, atol=1e-14)


def test_hlld_resolves_rotational_discontinuity(orc):
    # isolated left-going Alfven discontinuity: [v_t] = sgn(Bx) [B_t]/sqrt(rho),
    # rho, p, u, |B_t| continuous.  The interface sees the right state, so HLLD
    # must return F(U_R), and the jumps obey F_R - F_L = lambda (U_R - U_L) with
    # lambda = -|Bx|/sqrt(rho).
    for bx in (0.8, -0.6):
        rho, p = 1.3, 0.9
        th = 1.1
        btl = np.array([0.6, 0.0])
        btr = 0.6 * np.array([math.cos(th), math.sin(th)])
        vtl = np.array([0.1, -0.2])
        vtr = vtl + np.sign(bx) * (btr - btl) / math.sqrt(rho)
        a = _prim_state(rho, 0.0, vtl[0], vtl[1], p, bx, btl[0], btl[1])
        b = _prim_state(rho, 0.0, vtr[0], vtr[1], p, bx, btr[0], btr[1])
        f = orc.face_flux("hlld", 0, 5 / 3, 1.0, 0, a, b)
        fr = orc.face_flux("hlld", 0, 5 / 3, 1.0, 0, b, b)
        fl = orc.face_flux("hlld", 0, 5 / 3, 1.0, 0, a, a)
        np.testing.assert_allclose(f, fr, rtol=0, atol=2e-14)
        ua = orc.prim_to_cons(5 / 3, a)
        ub = orc.prim_to_cons(5 / 3, b)
        lam = -abs(bx) / math.sqrt(rho)
        np.testing.assert_allclose(fr - fl, lam * (ub - ua), rtol=0, atol=1e-13)


def test_exact_shock_states_satisfy_rh_with_oracle_flux(orc):
    # the physical flux (HLL of equal states) obeys F_d - F_u = s (U_d - U_u)
    # on the three exact shocks of the shock adiabatic
    for which in ("fast", "intermediate", "slow"):
        up, dn, s = mhd_shock(2.5, 0.1, 40.0, 5 / 3, which=which)
        wu = np.array(list(up) + [0.0])
        wd = np.array(list(dn) + [0.0])
        fu = orc.face_flux("hll", 0, 5 / 3, 1.0, 0, wu, wu)
        fd = orc.face_flux("hll", 0, 5 / 3, 1.0, 0, wd, wd)
        uu = orc.prim_to_cons(5 / 3, wu)
        ud = orc.prim_to_cons(5 / 3, wd)
        jump = (fd - fu) - s * (ud - uu)
        assert np.abs(jump[[0, 1, 2, 3, 4, 6, 7]]).max() < 1e-11 * np.abs(fd).max(), which


def test_paper_alfven_shock_flips_by():
    # Sect. 3.2.1: with delta = 2.5, upstream beta 0.1 and theta = 40 degrees,
    # the intermediate root is an Alfven shock across which B_y changes sign
    g = _golden("alfven_shock_params.txt")
    up, dn, s = mhd_shock(float(g["delta"][0]), float(g["beta"][0]), float(g["theta_deg"][0]),
                          float(g["gamma"][0]), which="intermediate",
                          rho1=float(g["rho_up"][0]), p1=float(g["p_up"][0]))
    assert up[6] * dn[6] < 0
    roots, _ = mhd_shock_roots(2.5, 0.1, 40.0, 5 / 3)
    assert len(roots) == 3


def test_glm_interface_solve_signs(orc):
    # upwinding of the 2x2 (B_n, psi) system: a pure right-going GLM wave
    # (psi = c_h B_n jump) passes through unchanged: the interface takes the
    # left state, so F(B_n) = psi_L and F(psi) = c_h^2 B_nL
    ch = 1.7
    a = _prim_state(1.0, 0, 0, 0, 1.0, 0.3, 0, 0, 0.2)
    b = a.copy()
    b[5] += 0.05
    b[8] += ch * 0.05
    f = orc.face_flux("hll", 1, 5 / 3, ch, 0, a, b)
    assert abs(f[5] - 0.2) < 1e-15 and abs(f[8] - ch * ch * 0.3) < 1e-14


# ----------------------------------------------------------------------------
# stage coefficients and the Runge-Kutta order
# ----------------------------------------------------------------------------

def _measured_coeffs(orc, time):
    # run stages on two uniform states (flux divergence exactly 0) to read the
    # convex-combination weights off the oracle's own stage
    W = wl.cp_alfven(16)
    W.cfg.time = time
    W.cfg.glm = False
    m = orc.mesh_for(W)
    nb, nc = W.nblocks, W.ncell
    U0 = np.zeros((9, nb, nc))
    Uk = np.zeros((9, nb, nc))
    base = orc.prim_to_cons(5 / 3, _prim_state(1.0, 0.1, 0.2, 0.3, 1.0, 0.5, 0.2, 0.1))
    for v in range(9):
        U0[v] = base[v] * 1.0
        Uk[v] = base[v] * 1.0
    U0[0] = 1.0
    Uk[0] = 2.0
    coeffs = []
    for k in range(2 if time == "ssprk2" else 3):
        out, st = m.stage(k, 1e-3, 1.0, U0, Uk)
        # out_rho = a * 1 + b * 2  and a + b = 1
        b = out[0, 0, 0] - 1.0
        coeffs.append((1.0 - b, b))
    return coeffs


@pytest.mark.parametrize("time,order", [("ssprk2", 2), ("ssprk3", 3)])
def test_ssprk_stability_polynomial_order(orc, time, order):
    coeffs = _measured_coeffs(orc, time)
    # Shu-Osher recursion for y' = z y: y_{k+1} = a_k y0 + b_k (y_k + z y_k)
    z = np.array([1e-2, 2e-2, 4e-2])
    y = np.ones_like(z)
    y0 = np.ones_like(z)
    for a, b in coeffs:
        y = a * y0 + b * (y + z * y)
    err = np.abs(y - np.exp(z))
    p = np.log2(err[1:] / err[:-1])
    assert np.all(np.abs(p - (order + 1)) < 0.15), (p, coeffs)


# ----------------------------------------------------------------------------
# whole-scheme pins
# ----------------------------------------------------------------------------

def _cp_error(orc, n, lim="vanleer", flux="hlld", threads=8):
    W = wl.cp_alfven(n, limiter=lim, flux=flux)
    m = orc.mesh_for(W, threads)
    U, t, ns, st = m.run(W.U, 1 / math.sqrt(2))
    assert st == 0 and abs(t[0] - 1 / math.sqrt(2)) < 1e-15
    _, _, _, Ue = wl.cp_alfven_exact(n, 1 / math.sqrt(2))
    vs = (1, 2, 3, 5, 6, 7)
    return sum(np.abs(U[v] - Ue[v]).sum() for v in vs) / sum(np.abs(Ue[v]).sum() for v in vs)


def test_cp_alfven_wave_second_order(orc):
    # exact nonlinear solution (Sect. 3, via Porth 2014): measured L1 order ~ 2
    e = [_cp_error(orc, n) for n in (32, 64, 128)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[-1] > 1.8, (e, orders)
    assert e[-1] < 1.5e-3
    ek = _cp_error(orc, 64, "koren")
    assert ek < e[1]  # third-order reconstruction beats second order
    eh = _cp_error(orc, 64, "vanleer", "hll")
    assert eh > e[1]  # HLL is more diffusive for the Alfven wave
    # the exact solution travels towards -n: a quarter period later the scheme
    # matches that direction and is O(1) off the opposite one
    W = wl.cp_alfven(64)
    tq = 0.25 / math.sqrt(2)
    U, *_ = orc.mesh_for(W, 8).run(W.U, tq)
    _, _, _, Up = wl.cp_alfven_exact(64, tq)
    _, _, _, Um = wl.cp_alfven_exact(64, -tq)
    assert rel_l1(U[7], Up[7]) < 0.02
    assert rel_l1(U[7], Um[7]) > 0.5


def test_conservation_periodic(orc):
    W = wl.c2_orszag_tang(128)
    m = orc.mesh_for(W, 8)
    s0 = m.sums(W.U)
    U, t, ns, st = m.run(W.U, 1.0, maxsteps=10)
    s1 = m.sums(U)
    assert ns == 10 and st == 0
    for v in range(8):
        scale = max(np.abs(s0[0, v]), np.abs(W.U[v]).mean(), 1e-300)
        assert abs(s1[0, v] - s0[0, v]) <= 1e-13 * scale, (v, s0[0, v], s1[0, v])
    # with alpha_p = 0 the glm field is conserved too
    W.cfg.glm_alpha = 0.0
    W.U[8] = 0.01 * np.sin(np.arange(W.U.shape[2]))[None, :]
    m = orc.mesh_for(W, 8)
    s0 = m.sums(W.U)
    U, t, ns, st = m.run(W.U, 1.0, maxsteps=5)
    assert abs(m.sums(U)[0, 8] - s0[0, 8]) < 1e-15


def test_free_stream_preserved(orc):
    W = wl.small_amr_2d(field="uniform")
    m = orc.mesh_for(W)
    dt, ch = m.cfl(W.U)
    out, st = m.stage(0, dt, ch, W.U, W.U)
    # uniform flow over a three-level mesh: round-off only (restriction sums)
    assert np.abs(out - W.U).max() < 1e-14 * np.abs(W.U).max()
    Wu = wl.cp_alfven(32)
    Wu.U[:] = W.U[:, :1, :1]
    m = orc.mesh_for(Wu)
    out, st = m.stage(0, 1e-2, 1.0, Wu.U, Wu.U)
    assert np.array_equal(out[:8], Wu.U[:8])  # bitwise on a single level


def test_sod_b0_converges_to_euler_exact(orc):
    # B = 0 ideal MHD is the Euler system: compare with the exact solution
    errs = []
    for n in (200, 400, 800):
        W = wl.riemann_1d((1.0, 0, 0, 0, 1.0, 0, 0), (0.125, 0, 0, 0, 0.1, 0, 0), n=n,
                          gamma=1.4, bx=0.0, t_end=0.2, flux="hlld", time="ssprk3")
        m = orc.mesh_for(W)
        U, t, ns, st = m.run(W.U, 0.2)
        x = (np.arange(n) + 0.5) / n
        ex = euler_exact((1.0, 0, 1.0), (0.125, 0, 0.1), 1.4, x, 0.2, x0=0.5)
        errs.append(np.abs(U[0, 0] - ex[0]).mean())
    assert errs[-1] < 4e-3, errs
    assert errs[0] / errs[-1] > 2.5, errs


@pytest.mark.parametrize("which", ["fast+", "slow+", "alfven+", "entropy"])
def test_linear_waves_travel_at_eigen_speeds(orc, which):
    # small-amplitude eigenmode of the primitive system; after one period on a
    # periodic line the state must return, with second-order convergence
    g = 5 / 3
    st0 = (1.0, 0.0, 0.0, 0.0, 0.6, 0.7, 0.9, 0.3) if which != "entropy" else \
        (1.0, 0.4, 0.0, 0.0, 0.6, 0.7, 0.9, 0.3)
    lam, r = linear_mode(st0, g, which)
    eps = 1e-5
    errs = []
    for n in (64, 128, 256):
        cfg = wl.Config(ndim=1, block_nx=(n // 4, 1, 1), flux="hlld", limiter="vanleer",
                        time="ssprk3", glm=False, courant=0.6)
        inst = wl.Instance(base_blocks=(4, 1, 1), gamma=g, t_end=1.0 / abs(lam))
        meta = wl.uniform_meta((4, 1, 1))
        x = (np.arange(n) + 0.5) / n
        s = np.sin(2 * math.pi * x)
        W0 = [st0[0] + eps * r[0] * s, st0[1] + eps * r[1] * s, st0[2] + eps * r[2] * s,
              st0[3] + eps * r[3] * s, st0[4] + eps * r[4] * s, st0[5] + 0 * s,
              st0[6] + eps * r[5] * s, st0[7] + eps * r[6] * s]
        U = wl.conserved_from_primitive(g, *W0).reshape(9, 4, n // 4)
        m = orc.Mesh(cfg, [inst], meta)
        U1, t, ns, stt = m.run(U, 1.0 / abs(lam))
        dev = (U1 - U)[[0, 1, 2, 3, 4, 6, 7]]
        errs.append(np.abs(dev).mean() / eps)
    p = math.log2(errs[1] / errs[2])
    assert p > 1.7, (which, errs)
    assert errs[-1] < 0.05


def test_glm_wave_speed(orc):
    # psi = eps sin(kx), B_n = 0, B = 0: the GLM pair obeys the wave equation at
    # speed c_h: psi = eps sin(kx) cos(k c_h t), B_n = -(eps/c_h) cos(kx) sin(k c_h t)
    n = 256
    eps = 1e-6
    cfg = wl.Config(ndim=1, block_nx=(n, 1, 1), flux="hll", limiter="vanleer", time="ssprk3",
                    glm=True, glm_alpha=0.0, courant=0.5)
    inst = wl.Instance(base_blocks=(1, 1, 1), gamma=5 / 3, t_end=0.3)
    x = (np.arange(n) + 0.5) / n
    z = 0 * x
    U = wl.conserved_from_primitive(5 / 3, 1 + z, z, z, z, 1 + z, z, z, z,
                                    eps * np.sin(2 * math.pi * x)).reshape(9, 1, n)
    m = orc.Mesh(cfg, [inst], wl.uniform_meta((1, 1, 1)))
    dt, ch = m.cfl(U)
    U1, t, ns, st = m.run(U, 0.3)
    k = 2 * math.pi
    psi_ex = eps * np.sin(k * x) * math.cos(k * ch[0] * 0.3)
    bx_ex = -(eps / ch[0]) * np.cos(k * x) * math.sin(k * ch[0] * 0.3)
    assert paper_error(U1[8, 0], psi_ex) < 5e-3
    assert paper_error(U1[5, 0], bx_ex) < 5e-3


def test_glm_damping_after_each_euler_substep(orc):
    # uniform psi: fluxes cancel, and damping E = exp(-alpha c_h dt/dx) after each
    # sub-step turns one SSPRK3 step into psi0 (1/3 + E/2 + E^3/6)
    W = wl.cp_alfven(16)
    W.cfg.glm_alpha = 0.7
    U = np.zeros_like(W.U)
    U[:] = orc.prim_to_cons(5 / 3, _prim_state(1, 0, 0, 0, 1, 0.5, 0.5, 0, 0.3))[:, None, None]
    m = orc.mesh_for(W)
    dt, ch = 1e-2, 2.0
    A, _ = m.stage(0, dt, ch, U, U)
    B, _ = m.stage(1, dt, ch, U, A)
    C, _ = m.stage(2, dt, ch, U, B)
    E = math.exp(-0.7 * ch * dt / (1 / 16))
    assert abs(C[8, 0, 0] - 0.3 * (1 / 3 + E / 2 + E ** 3 / 6)) < 1e-15


def test_cfl_maxsum_uniform(orc):
    W = wl.c2_orszag_tang(64)
    w = _prim_state(1.2, 0.3, -0.4, 0.1, 0.9, 0.5, -0.7, 0.2)
    U = np.zeros_like(W.U)
    U[:] = orc.prim_to_cons(5 / 3, w)[:, None, None]
    m = orc.mesh_for(W)
    dt, ch = m.cfl(U, t=0.0, t_end=1.0)
    sp = [abs(w[1 + d]) + orc.fast_speed(5 / 3, w, d) for d in range(2)]
    assert abs(dt[0] - 0.8 / (sp[0] * 64 + sp[1] * 64)) < 1e-15
    assert ch[0] == max(sp)
    dt2, _ = m.cfl(U, t=0.999999, t_end=1.0)
    assert abs(dt2[0] - 1e-6) < 1e-16


def test_mirror_symmetric_riemann(orc):
    a = (0.8, 0.2, 0.1, -0.3, 0.7, 0.6, 0.2)
    b = (0.3, -0.4, 0.0, 0.2, 0.2, -0.5, 0.4)
    mir = lambda s: (s[0], -s[1], s[2], s[3], s[4], s[5], s[6])
    W1 = wl.riemann_1d(a, b, n=256, nblocks=4, flux="hlld", time="ssprk3")
    W2 = wl.riemann_1d(mir(b), mir(a), n=256, nblocks=4, flux="hlld", time="ssprk3", bx=-0.75)
    U1, *_ = orc.mesh_for(W1).run(W1.U, 0.08)
    U2, *_ = orc.mesh_for(W2).run(W2.U, 0.08)
    f1 = U1.reshape(9, -1)
    f2 = U2.reshape(9, -1)[:, ::-1]
    sign = np.array([1, -1, 1, 1, 1, -1, 1, 1, 1])
    d = np.abs(f1 - sign[:, None] * f2).max(axis=1) / np.abs(f1).max(axis=1).clip(1e-300)
    assert d.max() < 1e-12, d


def test_exact_fast_shock_propagates(orc):
    # an isolated exact fast shock (Rankine-Hugoniot) must stay one shock moving
    # at the theoretical speed with the theoretical downstream plateau
    up, dn, s = mhd_shock(2.5, 0.1, 40.0, 5 / 3, which="fast")
    n = 800
    t_end = 0.04
    W = wl.riemann_1d(dn[:5] + dn[6:], up[:5] + up[6:], n=n, gamma=5 / 3, bx=up[5],
                      t_end=t_end, x0=0.3, flux="hlld", time="ssprk3")
    U, t, ns, st = orc.mesh_for(W).run(W.U, t_end)
    rho = U[0].ravel()
    x = (np.arange(n) + 0.5) / n
    pos = x[np.argmin(np.abs(rho - 0.5 * (up[0] + dn[0])))]
    assert abs(pos - (0.3 + s * t_end)) < 3.0 / n, (pos, 0.3 + s * t_end)
    down = x < 0.25
    assert np.abs(rho[down] - dn[0]).max() < 1e-6 * dn[0]
    by = U[6].ravel()
    assert np.abs(by[down] - dn[6]).max() < 1e-6 * abs(dn[6])
    assert np.abs(rho[x > pos + 6.0 / n] - up[0]).max() < 1e-9


def test_shu_osher_b0_runs_and_converges(orc):
    g = _golden("shu_osher_ic.txt")
    rl, vl, pl = (float(v) for v in g["left"])
    n_low = int(g["n_low"][0])
    t_end = float(g["t_end"][0])
    W = wl.shu_osher(n=n_low, t_end=t_end)
    # the generator uses the same left state (within the paper's 3-digit print)
    w0 = W.U[:, 0, 0]
    assert abs(w0[0] - rl) < 5e-3 and abs(w0[1] / w0[0] - vl) < 5e-3
    U, t, ns, st = orc.mesh_for(W).run(W.U, t_end)
    assert st == 0 and abs(t[0] - t_end) < 1e-15
    assert np.all(U[0] > 0)
    Wh = wl.shu_osher(n=2048, nblocks=8, t_end=t_end)
    Uh, *_ = orc.mesh_for(Wh, 8).run(Wh.U, t_end)
    rh = Uh[0].reshape(-1).reshape(n_low, 8).mean(axis=1)
    assert paper_error(U[0].ravel(), rh) < 0.05


def test_small_values_reported(orc):
    W = wl.cp_alfven(32)
    U = W.U.copy()
    U[4, 3, 17] = 0.3  # total energy below the magnetic energy: p < 0
    m = orc.mesh_for(W)
    dt, ch = m.cfl(W.U)
    out, st = m.stage(0, dt, ch, U, U)
    assert st == 4
    out, st = m.stage(0, dt, ch, W.U, W.U)
    assert st == 0


def test_invalid_meshes_rejected(orc):
    W = wl.small_amr_2d()
    meta = W.block_meta.copy()
    with pytest.raises(ValueError):
        orc.Mesh(W.cfg, W.instances, meta[1:])  # hole
    with pytest.raises(ValueError):
        orc.Mesh(W.cfg, W.instances, np.concatenate([meta, meta[:1]]))  # duplicate
    # two levels apart across a face
    cfg = wl.Config(ndim=2, block_nx=(8, 8, 1))
    inst = wl.Instance(base_blocks=(2, 1, 1))
    bad = [(0, 0, 1, 0, 0)] + [(0, 1, 0, 1, 0), (0, 1, 1, 1, 0), (0, 1, 1, 0, 0)] + \
          [(0, 2, 0, 0, 0), (0, 2, 1, 0, 0), (0, 2, 0, 1, 0), (0, 2, 1, 1, 0)]
    with pytest.raises(ValueError):
        orc.Mesh(cfg, [inst], np.array(bad, np.int32))


def _swap_xy_error(U, meta, nx):
    # U(x, y, z) against U(y, x, z) with (m_x, m_y) and (B_x, B_y) exchanged,
    # relative to each variable's scale
    index = {tuple(r): b for b, r in enumerate(meta.tolist())}
    sc = np.maximum(np.abs(U).max(axis=(1, 2)), 1e-300)[:, None, None, None]
    worst = 0.0
    for b, (q, L, i, j, k) in enumerate(meta.tolist()):
        A = U[:, b].reshape(9, nx, nx, nx)
        B = U[:, index[(q, L, j, i, k)]].reshape(9, nx, nx, nx).transpose(0, 1, 3, 2)
        B = B[[0, 2, 1, 3, 4, 6, 5, 7, 8]]
        worst = max(worst, float((np.abs(A - B) / sc).max()))
    return worst


def test_blast_xy_swap_symmetry(orc):
    # the 3D AMR blast with B0 along (1, 1, 0) is symmetric under x <-> y (the
    # mesh too): any index or sign slip in one direction's flux breaks it
    W = wl.c4_blast_amr(base=2, levels=3, bnx=8, shell=(0.2, 0.26), precision="fp64")
    U, t, ns, st = orc.mesh_for(W, 4).run(W.U, 1e30, maxsteps=3)
    assert st == 0 and np.abs(U - W.U).max() > 1e-2
    assert _swap_xy_error(U, W.block_meta, 8) < 1e-12
    # control: a field off the diagonal is not symmetric
    W.U[6] *= 0.5
    U, *_ = orc.mesh_for(W, 4).run(W.U, 1e30, maxsteps=3)
    assert _swap_xy_error(U, W.block_meta, 8) > 1e-6
