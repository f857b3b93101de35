"""Independent reference solutions used to pin the oracle.

Nothing here calls the oracle or the GPU library.  Each function states a
textbook result:

* ``paper_error``          the normalised error of Sect. 3.2.3, eq. (error):
                           E = sqrt(sum (u - r)^2 / sum r^2).
* ``euler_exact``          exact Riemann solution of the Euler equations
                           (pressure function + Newton iteration, sampling of the
                           wave fan), the B = 0 limit of ideal MHD.
* ``mhd_shock``            an exact planar oblique MHD shock from the
                           Rankine-Hugoniot conditions for a given compression
                           ratio, upstream beta and field angle (the construction
                           described in Sect. 3.2.1).
* ``linear_mode``          right eigenvectors of the 1D primitive-variable
                           quasi-linear ideal-MHD system.
"""
from __future__ import annotations

import math

import numpy as np


def paper_error(u, r):
    u = np.asarray(u, float)
    r = np.asarray(r, float)
    return math.sqrt(float(((u - r) ** 2).sum()) / float((r ** 2).sum()))


def rel_linf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


# ----------------------------------------------------------------------------
# exact Euler Riemann solver
# ----------------------------------------------------------------------------

def _pfun(p, rho, pk, ck, g):
    """Velocity change across a shock (p > pk) or rarefaction (p <= pk), and its
    derivative with respect to p."""
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (p + B))
    else:
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def euler_exact(left, right, g, x, t, x0=0.0):
    """Exact solution (rho, u, p) at points x and time t; left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _pfun(p, rl, pl, cl, g)
        fr, dfr = _pfun(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(1e-10, p - dp)
        if abs(p_new - p) < 1e-14 * p:
            p = p_new
            break
        p = p_new
    fl, _ = _pfun(p, rl, pl, cl, g)
    fr, _ = _pfun(p, rr, pr, cr, g)
    us = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    x = np.asarray(x, float)
    out = np.zeros((3, x.size))
    gm = (g - 1.0) / (g + 1.0)
    for n, xi in enumerate(x.ravel()):
        s = (xi - x0) / t
        if s <= us:
            if p > pl:
                sh = ul - cl * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                if s <= sh:
                    out[:, n] = (rl, ul, pl)
                else:
                    out[:, n] = (rl * (p / pl + gm) / (gm * p / pl + 1), us, p)
            else:
                cs = cl * (p / pl) ** ((g - 1) / (2 * g))
                if s <= ul - cl:
                    out[:, n] = (rl, ul, pl)
                elif s >= us - cs:
                    out[:, n] = (rl * (p / pl) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    out[:, n] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if p > pr:
                sh = ur + cr * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
                if s >= sh:
                    out[:, n] = (rr, ur, pr)
                else:
                    out[:, n] = (rr * (p / pr + gm) / (gm * p / pr + 1), us, p)
            else:
                cs = cr * (p / pr) ** ((g - 1) / (2 * g))
                if s >= ur + cr:
                    out[:, n] = (rr, ur, pr)
                elif s <= us + cs:
                    out[:, n] = (rr * (p / pr) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    out[:, n] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out


# ----------------------------------------------------------------------------
# exact oblique MHD shock (Rankine-Hugoniot)
# ----------------------------------------------------------------------------

def _downstream(U1, delta, rho1, p1, bx, by1, g):
    """Downstream state for upstream normal speed U1 (shock frame, v1 = 0) and
    compression delta, from mass, tangential momentum, induction and normal
    momentum conservation; returns the energy-flux residual too."""
    j = rho1 * U1
    u2 = U1 / delta
    rho2 = delta * rho1
    by2 = by1 * (rho1 * U1 * U1 - bx * bx) / (rho1 * U1 * U1 / delta - bx * bx)
    v2 = bx * (by2 - by1) / j
    p2 = p1 + rho1 * U1 * U1 * (1.0 - 1.0 / delta) + 0.5 * (by1 * by1 - by2 * by2)
    e1 = p1 / (g - 1) + 0.5 * rho1 * U1 * U1 + 0.5 * (bx * bx + by1 * by1)
    e2 = p2 / (g - 1) + 0.5 * rho2 * (u2 * u2 + v2 * v2) + 0.5 * (bx * bx + by2 * by2)
    pt1 = p1 + 0.5 * (bx * bx + by1 * by1)
    pt2 = p2 + 0.5 * (bx * bx + by2 * by2)
    fe1 = (e1 + pt1) * U1 - bx * (U1 * bx)
    fe2 = (e2 + pt2) * u2 - bx * (u2 * bx + v2 * by2)
    return (rho2, u2, v2, p2, by2), fe1 - fe2


def mhd_shock_roots(delta, beta, theta_deg, gamma, rho1=1.0, p1=None):
    """All upstream shock-frame speeds U1 for which the compression delta
    satisfies the energy condition (slow, intermediate, fast roots ascending)."""
    from scipy.optimize import brentq
    if p1 is None:
        p1 = 1.0 / gamma
    B = math.sqrt(2.0 * p1 / beta)
    th = math.radians(theta_deg)
    bx, by1 = -B * math.cos(th), B * math.sin(th)
    f = lambda U: _downstream(U, delta, rho1, p1, bx, by1, gamma)[1]
    grid = np.geomspace(1e-3, 50.0, 20000)
    vals = []
    for U in grid:
        try:
            vals.append(f(U))
        except ZeroDivisionError:
            vals.append(np.nan)
    roots = []
    for a, b, fa, fb in zip(grid[:-1], grid[1:], vals[:-1], vals[1:]):
        if np.isfinite(fa) and np.isfinite(fb) and fa * fb < 0:
            # skip the pole of by2 (sign change through infinity)
            if abs(fa) < 1e3 and abs(fb) < 1e3:
                roots.append(brentq(f, a, b, xtol=1e-15, rtol=1e-15))
    return roots, (rho1, p1, bx, by1)


def mhd_shock(delta, beta, theta_deg, gamma, which="fast", rho1=1.0, p1=None):
    """Exact shock moving in +x into a resting upstream on the right.

    Returns (upstream_prim, downstream_prim, speed) with prim = (rho, u, v, w, p,
    bx, by, bz), in the frame where the upstream is at rest."""
    roots, (rho1, p1, bx, by1) = mhd_shock_roots(delta, beta, theta_deg, gamma, rho1, p1)
    # physical roots need positive downstream pressure
    good = []
    for U in roots:
        (rho2, u2, v2, p2, by2), _ = _downstream(U, delta, rho1, p1, bx, by1, gamma)
        if p2 > 0:
            good.append(U)
    if which == "fast":
        U1 = max(good)
    elif which == "slow":
        U1 = min(good)
    else:
        U1 = sorted(good)[len(good) // 2]
    (rho2, u2, v2, p2, by2), _ = _downstream(U1, delta, rho1, p1, bx, by1, gamma)
    # shock frame: upstream flows in -x at -U1; all velocities flip sign, the
    # tangential jump flips with them.  Lab frame: add U1.
    up = (rho1, 0.0, 0.0, 0.0, p1, bx, by1, 0.0)
    down = (rho2, -u2 + U1, -v2, 0.0, p2, bx, by2, 0.0)
    return up, down, U1


# ----------------------------------------------------------------------------
# linear waves
# ----------------------------------------------------------------------------

def primitive_matrix(rho, u, v, w, p, bx, by, bz, g):
    """A(W) of W_t + A W_x = 0 for W = (rho, u, v, w, p, By, Bz), B_x constant."""
    return np.array([
        [u, rho, 0, 0, 0, 0, 0],
        [0, u, 0, 0, 1 / rho, by / rho, bz / rho],
        [0, 0, u, 0, 0, -bx / rho, 0],
        [0, 0, 0, u, 0, 0, -bx / rho],
        [0, g * p, 0, 0, u, 0, 0],
        [0, by, -bx, 0, 0, u, 0],
        [0, bz, 0, -bx, 0, 0, u],
    ], float)


def linear_mode(state, g, which):
    """Eigenvalue and right eigenvector (rho, u, v, w, p, By, Bz) of a wave family:
    'fast+', 'slow+', 'alfven+', 'entropy' ... (sorted eigenvalues)."""
    rho, u, v, w, p, bx, by, bz = state
    A = primitive_matrix(rho, u, v, w, p, bx, by, bz, g)
    lam, R = np.linalg.eig(A)
    order = np.argsort(lam.real)
    lam = lam.real[order]
    R = R.real[:, order]
    idx = {"fast-": 0, "alfven-": 1, "slow-": 2, "entropy": 3, "slow+": 4,
           "alfven+": 5, "fast+": 6}[which]
    r = R[:, idx]
    return lam[idx], r / np.abs(r).max()
