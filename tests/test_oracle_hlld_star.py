"""Pins of the oracle's HLLD (Miyoshi & Kusano 2005, the flux-scheme table of
Sect. 3) at its star states and where their formulas degenerate.

The tangential single-star velocity and field of MK05 divide by
D = rho (S - u)(S - S_M) - B_x^2, which vanishes when the outer wave speed
equals the Alfven speed: a side with no tangential field whose fast speed is
the Alfven speed (B_x^2 > gamma p).  There the oracle keeps v* = v and B* = B
(|D| <= 1e-8 max(|rho (S - u)(S - S_M)|, B_x^2)).  At B_x = 0 the rotational
waves coincide with the contact, the double-star regions have zero width (so
the value of sgn(0) cannot show in the flux) and the flux is the single-star
(contact-resolving) flux.  Each test compares with an exact solution, a
textbook closed form or a jump condition, written independently of the
oracle's formulas:

* a resting contact in pressure balance with a purely normal field: the exact
  flux is that of either side (zero mass, energy and tangential fluxes);
* a moving contact with a small tangential field B_t = delta: the exact flux is
  F(U_L) at every delta, on both sides of the degeneracy threshold, so the
  flux is continuous there and approaches the delta = 0 flux at O(delta);
* B_x = 0: Toro's HLLC flux of the Euler equations (Riemann Solvers and
  Numerical Methods for Fluid Dynamics, Sect. 10.4) with the total pressure in
  place of p and the tangential field carried as B_t / rho, which the
  induction equation advects when B_x = 0;
* inside a single-star region: the star state recovered from the flux obeys
  the jump conditions across the outer wave (MK05 eqs. 43-48), the energy
  jump with its B_x (v.B - v*.B*) term included.
"""
import math

import numpy as np
import pytest

G = 5.0 / 3.0


def _w(rho, u, v, w, p, bx, by, bz):
    return np.array([rho, u, v, w, p, bx, by, bz, 0.0], float)


def _phys_flux_x(w, g=G):
    """Ideal-MHD flux along x of a primitive state (no glm), written from the
    conservation laws: mass, momentum with total pressure and Maxwell stress,
    energy, induction."""
    rho, u, v, ww, p, bx, by, bz = w[:8]
    b2 = bx * bx + by * by + bz * bz
    pt = p + 0.5 * b2
    e = p / (g - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * b2
    vb = u * bx + v * by + ww * bz
    return np.array([rho * u, rho * u * u + pt - bx * bx, rho * u * v - bx * by,
                     rho * u * ww - bx * bz, (e + pt) * u - bx * vb, 0.0,
                     by * u - bx * v, bz * u - bx * ww, 0.0])


def _rot(w, d):
    """The x-frame state w relabelled so that direction d is the normal."""
    out = w.copy()
    for c0 in (1, 5):
        vec = w[c0:c0 + 3]
        out[c0:c0 + 3] = np.roll(vec, d)
    return out


def _rot_flux(f, d):
    out = f.copy()
    for c0 in (1, 5):
        out[c0:c0 + 3] = np.roll(f[c0:c0 + 3], d)
    return out


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("light_left", [True, False])
@pytest.mark.parametrize("bx", [1.0, -1.3])
def test_resting_contact_with_normal_field_takes_degenerate_branch(orc, d, light_left, bx):
    # p = 0.3, B = (bx, 0, 0): B_x^2 > gamma p on both sides, so each side's
    # fast speed is its Alfven speed and rho c_f^2 = B_x^2.  The outer speeds
    # are -/+ the lighter side's c_f, S_M = 0, hence D = 0 on the lighter side.
    p = 0.3
    assert bx * bx > G * p
    rl, rr = (0.2, 1.0) if light_left else (1.0, 0.2)
    a, b = _w(rl, 0, 0, 0, p, bx, 0, 0), _w(rr, 0, 0, 0, p, bx, 0, 0)
    # D of the lighter side from closed forms (c_f^2 = B_x^2 / rho when the
    # tangential field vanishes and B_x^2 > gamma p)
    rho_l = min(rl, rr)
    s = math.sqrt(bx * bx / rho_l)
    assert abs(rho_l * s * s - bx * bx) <= 1e-12 * bx * bx
    f = orc.face_flux("hlld", 0, G, 1.0, d, _rot(a, d), _rot(b, d))
    exact = _rot_flux(_phys_flux_x(a), d)
    np.testing.assert_allclose(exact, _rot_flux(_phys_flux_x(b), d), rtol=0, atol=1e-15)
    # zero mass, energy and tangential fluxes; normal momentum flux p - B_x^2/2
    np.testing.assert_allclose(f, exact, rtol=0, atol=1e-14)
    assert abs(f[1 + d] - (p - 0.5 * bx * bx)) < 1e-14


DELTAS = [1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-9, 1e-12, 0.0]


def _degeneracy_ratio(wl, wr, g=G):
    """|D_L| / max(|rho (S_L - u_L)(S_L - S_M)|, B_x^2) of the left side, with
    the outer speeds of MK05 eq. (67) and S_M of MK05 eq. (38) evaluated from
    closed forms (fast speed as the larger root of the magnetosonic quartic)."""
    def cf(w):
        rho, p, bx, by, bz = w[0], w[4], w[5], w[6], w[7]
        a2 = g * p / rho
        b2 = (bx * bx + by * by + bz * bz) / rho
        bx2 = bx * bx / rho
        return math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * bx2)))
    cmax = max(cf(wl), cf(wr))
    sl = min(wl[1], wr[1]) - cmax
    sr = max(wl[1], wr[1]) + cmax
    ptl = wl[4] + 0.5 * float(wl[5:8] @ wl[5:8])
    ptr = wr[4] + 0.5 * float(wr[5:8] @ wr[5:8])
    ml = wl[0] * (sl - wl[1])
    mr = wr[0] * (sr - wr[1])
    sm = (mr * wr[1] - ml * wl[1] - ptr + ptl) / (mr - ml)
    big = ml * (sl - sm)
    bx2 = wl[5] ** 2
    return abs(big - bx2) / max(abs(big), bx2)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_moving_contact_exact_across_degeneracy_threshold(orc, d):
    # a contact moving at u0 = 0.4 with equal p, v_t and B_t = delta (1, 1/2)
    # on both sides, lighter fluid on the left: the exact interface flux is
    # F(U_L).  Small delta puts the left side inside the degeneracy threshold,
    # larger delta outside; both must give the exact flux, so the flux is
    # continuous where the branch switches and within O(delta) of delta = 0.
    p, bx = 0.3, 1.0
    ratios, fluxes = [], []
    for delta in DELTAS:
        a = _w(0.2, 0.4, 0.3, -0.1, p, bx, delta, 0.5 * delta)
        b = _w(1.0, 0.4, 0.3, -0.1, p, bx, delta, 0.5 * delta)
        r = _degeneracy_ratio(a, b)
        ratios.append(r)
        f = orc.face_flux("hlld", 0, G, 1.0, d, _rot(a, d), _rot(b, d))
        exact = _rot_flux(_phys_flux_x(a), d)
        # just outside the threshold the star formulas divide by a small D:
        # their rounding grows like 1/ratio there
        tol = 2e-14 * (max(1.0, 1e-6 / r) if r > 1e-8 else 1.0)
        np.testing.assert_allclose(f, exact, rtol=0, atol=tol)
        fluxes.append(f)
    # the sweep spans both branches of the 1e-8 threshold
    assert ratios[0] > 1e-8 and ratios[1] > 1e-8
    assert all(r <= 1e-8 for r in ratios[4:])
    f0 = fluxes[-1]
    for delta, f in zip(DELTAS[:-1], fluxes[:-1]):
        assert np.abs(f - f0).max() <= 2.0 * delta + 1e-14, (delta, f - f0)


def _hllc_bx0(wl, wr, g=G):
    """Toro's HLLC flux (single-star states, contact speed S*) with the total
    pressure p_T = p + B_t^2/2 in place of p, B_t carried as a density-weighted
    passive quantity (B*_t = B_t rho*/rho) and the outer speeds
    S_L = min(u) - max(c_f), S_R = max(u) + max(c_f), c_f^2 = a^2 + B_t^2/rho."""
    def side(w):
        rho, u, v, ww, p, bx, by, bz = w[:8]
        assert bx == 0.0
        bt2 = by * by + bz * bz
        pt = p + 0.5 * bt2
        E = p / (g - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * bt2
        U = np.array([rho, rho * u, rho * v, rho * ww, E, 0.0, by, bz, 0.0])
        return U, pt, math.sqrt(g * p / rho + bt2 / rho)
    UL, ptl, cl = side(wl)
    UR, ptr, cr = side(wr)
    sl = min(wl[1], wr[1]) - max(cl, cr)
    sr = max(wl[1], wr[1]) + max(cl, cr)
    rl, ul, rr, ur = wl[0], wl[1], wr[0], wr[1]
    # Toro eq. (10.37): contact speed
    ss = (ptr - ptl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))
    FL, FR = _phys_flux_x(wl, g), _phys_flux_x(wr, g)

    def star(w, U, pt, s):
        rho, u = w[0], w[1]
        fac = rho * (s - u) / (s - ss)
        # Toro eq. (10.39) with p -> p_T and E including the magnetic energy
        Es = U[4] / rho + (ss - u) * (ss + pt / (rho * (s - u)))
        return np.array([fac, fac * ss, fac * w[2], fac * w[3], fac * Es, 0.0,
                         fac * w[6] / rho, fac * w[7] / rho, 0.0])
    if sl >= 0:
        return FL
    if sr <= 0:
        return FR
    if ss >= 0:
        return FL + sl * (star(wl, UL, ptl, sl) - UL)
    return FR + sr * (star(wr, UR, ptr, sr) - UR)


def test_bx_zero_equals_single_star_flux(orc):
    # B_x = 0: sgn(B_x) = 0, the rotational waves coincide with the contact and
    # the flux is the single-star flux; random states with tangential fields,
    # including supersonic ones where an outer state is upwind
    rng = np.random.Generator(np.random.PCG64(2024))
    n_star = 0
    for _ in range(300):
        def rnd():
            return _w(rng.uniform(0.1, 2.0), rng.uniform(-1.5, 1.5), rng.uniform(-1, 1),
                      rng.uniform(-1, 1), rng.uniform(0.05, 2.0), 0.0,
                      rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5))
        a, b = rnd(), rnd()
        ref = _hllc_bx0(a, b)
        n_star += int(abs(ref[0] - _phys_flux_x(a)[0]) > 1e-12 and
                      abs(ref[0] - _phys_flux_x(b)[0]) > 1e-12)
        for d in range(3):
            f = orc.face_flux("hlld", 0, G, 1.0, d, _rot(a, d), _rot(b, d))
            np.testing.assert_allclose(f, _rot_flux(ref, d), rtol=1e-12, atol=1e-13)
    assert n_star > 200  # most faces sit inside the fan


def _outer_region_speeds(wl, wr, g=G):
    """S_L, S_R (outer speeds as in the oracle's reading), S_M (MK05 eq. 38)
    and the rotational speeds S*_L, S*_R (MK05 eq. 51) from closed forms."""
    def cf(w):
        rho, p, bx, by, bz = w[0], w[4], w[5], w[6], w[7]
        a2 = g * p / rho
        b2 = (bx * bx + by * by + bz * bz) / rho
        return math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * bx * bx / rho)))
    cmax = max(cf(wl), cf(wr))
    sl = min(wl[1], wr[1]) - cmax
    sr = max(wl[1], wr[1]) + cmax
    ptl = wl[4] + 0.5 * float(wl[5:8] @ wl[5:8])
    ptr = wr[4] + 0.5 * float(wr[5:8] @ wr[5:8])
    ml, mr = wl[0] * (sl - wl[1]), wr[0] * (sr - wr[1])
    sm = (mr * wr[1] - ml * wl[1] - ptr + ptl) / (mr - ml)
    rsl = ml / (sl - sm)
    rsr = mr / (sr - sm)
    bx = abs(wl[5])
    return sl, sr, sm, sm - bx / math.sqrt(rsl), sm + bx / math.sqrt(rsr)


def _cons(w, g=G):
    rho, u, v, ww, p, bx, by, bz = w[:8]
    e = p / (g - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * (bx * bx + by * by + bz * bz)
    return np.array([rho, rho * u, rho * v, rho * ww, e, bx, by, bz, 0.0])


@pytest.mark.parametrize("side", ["left", "right"])
def test_single_star_state_obeys_jump_conditions(orc, side):
    # Where x/t = 0 lies between an outer wave S and its rotational wave, the
    # HLLD flux is F_K + S (U*_K - U_K).  The single-star state of MK05 is the
    # state joined to U_K by the jump conditions across S with the intermediate
    # fan's S_M and total pressure p_T*: its flux is the physical one,
    #   (rho* S_M, rho* S_M^2 + p_T* - B_x^2, rho* S_M v*_t - B_x B*_t,
    #    (e* + p_T*) S_M - B_x v*.B*, B*_t S_M - B_x v*_t).
    # Recover U* = U_K + (F - F_K)/S from the oracle's flux, p_T* from its
    # normal momentum flux, and check the other components, the energy flux in
    # particular (MK05 eq. 48).
    rng = np.random.Generator(np.random.PCG64(77 if side == "left" else 78))
    hits = 0
    for _ in range(4000):
        u0 = rng.uniform(0.8, 3.0) * (1 if side == "left" else -1)
        a = _w(rng.uniform(0.3, 2.0), u0 + rng.uniform(-0.3, 0.3), rng.uniform(-1, 1),
               rng.uniform(-1, 1), rng.uniform(0.1, 1.5), rng.choice([-1, 1]) * rng.uniform(0.1, 0.8),
               rng.uniform(-1, 1), rng.uniform(-1, 1))
        b = _w(rng.uniform(0.3, 2.0), u0 + rng.uniform(-0.3, 0.3), rng.uniform(-1, 1),
               rng.uniform(-1, 1), rng.uniform(0.1, 1.5), a[5], rng.uniform(-1, 1),
               rng.uniform(-1, 1))
        sl, sr, sm, ssl, ssr = _outer_region_speeds(a, b)
        if side == "left" and not (sl < -1e-3 and ssl > 1e-3):
            continue
        if side == "right" and not (ssr < -1e-3 and sr > 1e-3):
            continue
        hits += 1
        wk, s = (a, sl) if side == "left" else (b, sr)
        f = orc.face_flux("hlld", 0, G, 1.0, 0, a, b)
        us = _cons(wk) + (f - _phys_flux_x(wk)) / s
        rho_s, smv = us[0], us[1] / us[0]
        assert abs(smv - sm) < 1e-11 * max(1.0, abs(sm))
        vs, bs = us[1:4] / rho_s, us[5:8]
        bx = wk[5]
        pts = f[1] - rho_s * smv * smv + bx * bx
        expect = np.array([rho_s * smv, f[1], rho_s * smv * vs[1] - bx * bs[1],
                           rho_s * smv * vs[2] - bx * bs[2],
                           (us[4] + pts) * smv - bx * float(vs @ bs), 0.0,
                           bs[1] * smv - bx * vs[1], bs[2] * smv - bx * vs[2], 0.0])
        np.testing.assert_allclose(f, expect, rtol=1e-10, atol=1e-11)
    assert hits > 100
