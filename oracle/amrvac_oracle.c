/*
 * FP64 CPU oracle for the ideal-MHD + glm block update (MPI-AMRVAC 3.0,
 * Keppens et al. 2023).  TEST INFRASTRUCTURE ONLY: used by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg; never by the GPU library.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, IEEE
 * division and square root), see oracle/__init__.py.
 *
 * Readings where the paper names a method without printing it (each one is a
 * published method the paper cites, restated here from its definition):
 *  - equations: ideal MHD in conservative form with magnetic pressure B^2/2,
 *    plus the mixed glm field psi of Dedner et al. 2002 (Sect. 3.2, Table of
 *    monopole control, option `glm`); psi enters only through the interface
 *    solve and an exponential damping after each Euler sub-step; no
 *    non-conservative sources.
 *  - reconstruction on primitive variables (Sect. 3 reconstructs primitives by
 *    default) with the two-ghost-cell limiters `minmod`, `vanleer`, `koren`,
 *    `superbee`, `woodward`, `mcbeta` (beta = 1.4) and `albada` of the limiter
 *    table (order 3 for koren, 2 for the others); albada in its TVD form
 *    (zero slope at extrema, like the others); `cada3` (Cada & Torrilhon
 *    2009, third order, two ghost cells, see cada3_phi); `venk`
 *    (Venkatakrishnan 1995, see venk_phi; smoothing constant 0); and the
 *    three-ghost-cell five-point `mp5`, `weno5`, `wenoz5` and `wenozp5` (see
 *    mp5_plus, weno5_plus).
 *  - a face whose reconstructed density or pressure is not positive falls back
 *    to first order (cell values) on both sides (Sect. 7.4 mentions checks on
 *    reconstructions; the fallback form is our reading).
 *  - HLL (Harten 1983) with Davis speed bounds; HLLD (Miyoshi & Kusano 2005)
 *    with outer speeds min/max(u) -/+ max(c_f) and a degeneracy threshold.
 *  - SSPRK(2,2), SSPRK(3,3) (Gottlieb 2005), SSPRK(4,3) and SSPRK(5,4)
 *    (Spiteri & Ruuth 2002) in Shu-Osher form (Sect. 3, time-integration
 *    table); psi is damped over each Euler part's time step.
 *  - TVD Lax-Friedrichs flux with the fastest local signal speed; HLLC for
 *    MHD in the three-wave form of Li 2005 (see hllc_local).
 *  - CFL: dt = C / max over cells of sum_d (|v_d| + c_f,d)/dx_d, from U^n,
 *    global per instance, no subcycling; c_h = max (|v_d| + c_f,d).
 *  - AMR ghost values (the paper gives no operators): same level -> copy;
 *    finer -> mean of the 2^d children; coarser -> coarse value plus
 *    minmod-limited slopes times +-1/4 coarse cell, on conserved variables.
 *    Requires full 2:1 balance (checked at creation).
 *  - per-level schemes (Sect. 3): a block's faces use the flux and limiter of
 *    its level (level_flux / level_limiter, -1 = the global choice).
 *  - refluxing (cfg.reflux): after each stage the coarse cell next to a finer
 *    neighbour replaces that face's coarse flux by the mean of the fine fluxes
 *    through it (conservative AMR, Sect. 3).
 *  - outflow boundary: a ghost takes the value of the nearest in-domain cell of
 *    its own level (zero gradient, Sect. 3.1.1 and Sect. 3.2.1).
 *  - symmetric (reflecting) wall: a ghost takes the mirror cell across the
 *    boundary with the normal momentum and normal magnetic field negated
 *    (scalars, tangential components and psi even; see value_at).
 *  - fix_small_values (Sect. 7.4 bootstrapping, off by default): after every
 *    stage, cells below small_density / small_pressure are replaced by the
 *    floors or by the average over their non-small same-level face
 *    neighbours, on primitive variables, never changing B (orc_fix_small).
 */
#include "amrvac_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NV ORC_NVAR
/* ghost cells per block face: 2 for the two-ghost-cell limiters, 3 for the
 * five-point ones (mp5, weno5, wenoz5); per mesh in orc_mesh.ng */
#define NG 2
#define NG5 3
enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BXV = 5, BYV = 6, BZV = 7, PSI = 8 };
enum { ST_OK = 0, ST_SMALL = 4 };

typedef struct {
  int inst, level, idx[3];
} blockinfo;

struct orc_mesh {
  orc_config cfg;
  int ninst;
  orc_instance* inst;
  int nblocks;
  blockinfo* blk;
  int ncell;
  int nthreads;
  /* hash map (inst, level, i, j, k) -> leaf block id (>= 0) or -1 (refined) */
  size_t hcap;
  uint64_t* hkey;
  int* hval;
  unsigned char* hused;
  /* refluxing: per block and face the kind of neighbour (0 same level or
   * boundary, 1 finer, 2 coarser) and the stage's face fluxes there,
   * [block][face][var][tangential cells] */
  unsigned char* fkind;
  double* facef;
  int farea;
  int ng; /* ghost width: NG5 when any level uses a five-point limiter, else NG */
};

/* ------------------------------------------------------------------------ */
/* block map                                                                 */
/* ------------------------------------------------------------------------ */

static uint64_t mkkey(int inst, int L, long i, long j, long k) {
  return ((uint64_t)inst << 43) | ((uint64_t)L << 39) | ((uint64_t)i << 26) |
         ((uint64_t)j << 13) | (uint64_t)k;
}

static size_t hslot(const orc_mesh* m, uint64_t key) {
  uint64_t h = key * 0x9E3779B97F4A7C15ull;
  return (size_t)(h >> 17) & (m->hcap - 1);
}

/* returns >= 0 leaf id, -1 refined, -2 nothing at this level */
static int hget(const orc_mesh* m, uint64_t key) {
  size_t s = hslot(m, key);
  while (m->hused[s]) {
    if (m->hkey[s] == key) return m->hval[s];
    s = (s + 1) & (m->hcap - 1);
  }
  return -2;
}

/* insert; returns the previous value (-2 if absent) */
static int hput(orc_mesh* m, uint64_t key, int val) {
  size_t s = hslot(m, key);
  while (m->hused[s]) {
    if (m->hkey[s] == key) {
      int old = m->hval[s];
      m->hval[s] = val;
      return old;
    }
    s = (s + 1) & (m->hcap - 1);
  }
  m->hused[s] = 1;
  m->hkey[s] = key;
  m->hval[s] = val;
  return -2;
}

static long cells_at_level(const orc_mesh* m, int inst, int L, int d) {
  return (long)m->inst[inst].base[d] * m->cfg.nx[d] << L;
}

static long blocks_at_level(const orc_mesh* m, int inst, int L, int d) {
  if (d >= m->cfg.ndim) return 1;
  return (long)m->inst[inst].base[d] << L;
}

/* ------------------------------------------------------------------------ */
/* pointwise physics                                                         */
/* ------------------------------------------------------------------------ */

void orc_cons_to_prim(double gamma, const double* u, double* w) {
  double rho = u[RHO];
  double vx = u[MX] / rho, vy = u[MY] / rho, vz = u[MZ] / rho;
  double ke = 0.5 * (u[MX] * vx + u[MY] * vy + u[MZ] * vz);
  double me = 0.5 * (u[BXV] * u[BXV] + u[BYV] * u[BYV] + u[BZV] * u[BZV]);
  w[RHO] = rho;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = (gamma - 1.0) * (u[EN] - ke - me);
  w[5] = u[BXV];
  w[6] = u[BYV];
  w[7] = u[BZV];
  w[8] = u[PSI];
}

void orc_prim_to_cons(double gamma, const double* w, double* u) {
  double rho = w[0];
  u[RHO] = rho;
  u[MX] = rho * w[1];
  u[MY] = rho * w[2];
  u[MZ] = rho * w[3];
  u[EN] = w[4] / (gamma - 1.0) + 0.5 * rho * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) +
          0.5 * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
  u[BXV] = w[5];
  u[BYV] = w[6];
  u[BZV] = w[7];
  u[PSI] = w[8];
}

/* fast magnetosonic speed along dir, cancellation-free form
 * c_f^2 = (a^2 + b^2 + sqrt((a^2 - b^2)^2 + 4 a^2 b_t^2)) / 2 */
double orc_fast_speed(double gamma, const double* w, int dir) {
  int t1 = (dir + 1) % 3, t2 = (dir + 2) % 3;
  double rho = w[0];
  double a2 = gamma * w[4] / rho;
  double bn = w[5 + dir], b1 = w[5 + t1], b2t = w[5 + t2];
  double bt2 = (b1 * b1 + b2t * b2t) / rho;
  double b2 = (bn * bn + b1 * b1 + b2t * b2t) / rho;
  double dd = a2 - b2;
  double cf2 = 0.5 * (a2 + b2 + sqrt(dd * dd + 4.0 * a2 * bt2));
  return sqrt(cf2);
}

/* ------------------------------------------------------------------------ */
/* limiters (limiter table of Sect. 3.1.1)                                   */
/* ------------------------------------------------------------------------ */

static double sgn(double x) { return (x > 0.0) - (x < 0.0); }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

static double minmod2(double a, double b) {
  if (a * b > 0.0) return sgn(a) * dmin(fabs(a), fabs(b));
  return 0.0;
}

/* slope of the symmetric TVD limiters of the limiter table, phi(r) dp with
 * r = dm/dp > 0 (the caller handles dm dp <= 0):
 *   3 superbee (Roe 1985):      phi = max(min(2r, 1), min(r, 2))
 *   4 woodward (van Leer 1977, monotonized central): phi = min(2r, (1+r)/2, 2)
 *   5 mcbeta (van Leer 1977):   phi = min(beta r, (1+r)/2, beta), beta = 1.4
 *   6 albada (van Albada 1982): phi = (r^2 + r)/(r^2 + 1) */
static double sym_slope(int lim, double dm, double dp) {
  double am = fabs(dm), ap = fabs(dp);
  switch (lim) {
    case 3: return sgn(dp) * dmax(dmin(2.0 * am, ap), dmin(am, 2.0 * ap));
    case 4: return sgn(dp) * dmin(dmin(2.0 * am, 0.5 * (am + ap)), 2.0 * ap);
    case 5: return sgn(dp) * dmin(dmin(1.4 * am, 0.5 * (am + ap)), 1.4 * ap);
    default: return dm * dp * (dm + dp) / (dm * dm + dp * dp);
  }
}

/* 10 cada3 (Cada & Torrilhon 2009, the compact third-order limiter LimO3):
 * with theta = dm/dp and the third-order (kappa = 1/3) polynomial
 * phi3 = (2 + theta)/3,
 *   phi(theta) = max(0, min(phi3, max(-theta/2, min(2 theta, phi3, 1.6)))),
 * and the face value b + phi(theta) dp / 2 (b where dp = 0, the limit of
 * phi dp).  Unlike the TVD limiters it keeps a slope at extrema (theta < 0),
 * where it follows phi3 as long as phi3 <= -theta/2. */
static double cada3_phi(double theta) {
  const double p3 = (2.0 + theta) / 3.0;
  return dmax(0.0, dmin(p3, dmax(-0.5 * theta, dmin(dmin(2.0 * theta, p3), 1.6))));
}

static double cada3_face(double dm, double dp) {
  if (dp == 0.0) return 0.0;
  return 0.5 * cada3_phi(dm / dp) * dp;
}

/* 12 venk (Venkatakrishnan 1995), on the 1D stencil (a, b, c) of a cell: the
 * unlimited increment from the cell centre to its faces is the central
 * difference d2 = +-(c - a)/4; a face whose increment d2 has the sign of
 * D = max(a, b, c) - b (d2 > 0) or D = min(a, b, c) - b (d2 < 0) is limited by
 *   phi(y) = (y^2 + 2 y)/(y^2 + y + 2),  y = D/d2 >= 0,
 * written (D^2 + 2 D d2)/(D^2 + 2 d2^2 + D d2), the smooth replacement of
 * min(1, y); the cell takes the smaller of its two faces' factors, and its
 * face values are b +- phi d2.  The smoothing constant eps^2 = (K dx)^3 of the
 * original is taken as 0 (the paper gives no K). */
static double venk_phi(double D, double d2) {
  return (D * D + 2.0 * D * d2) / (D * D + 2.0 * d2 * d2 + D * d2);
}

/* the limited increment phi d2 from b to its right face (the left face gets
 * the opposite) */
static double venk_increment(double a, double b, double c) {
  const double d2 = 0.25 * (c - a);
  if (d2 == 0.0) return 0.0;
  const double up = dmax(dmax(a, b), c) - b, dn = dmin(dmin(a, b), c) - b;
  const double phr = venk_phi(d2 > 0.0 ? up : dn, d2);   /* right face: +d2 */
  const double phl = venk_phi(d2 > 0.0 ? dn : up, -d2);  /* left face: -d2 */
  return dmin(phr, phl) * d2;
}

/* left state at the right face (i+1/2) of the cell with values (a, b, c) */
static double recon_plus(int lim, double a, double b, double c) {
  double dm = b - a, dp = c - b;
  if (lim == 10) return b + cada3_face(dm, dp);
  if (lim == 12) return b + venk_increment(a, b, c);
  if (!(dm * dp > 0.0)) return b;
  if (lim >= 3) return b + 0.5 * sym_slope(lim, dm, dp);
  switch (lim) {
    case 0: return b + 0.5 * minmod2(dm, dp);
    case 1: return b + 0.5 * (2.0 * dm * dp / (dm + dp));
    default: {
      /* Koren: phi(r) = max(0, min(2r, (2+r)/3, 2)) with r = dm/dp, times dp */
      double am = fabs(dm), ap = fabs(dp);
      double lim3 = dmin(dmin(2.0 * am, (am + 2.0 * ap) / 3.0), 2.0 * ap);
      return b + 0.5 * sgn(dp) * lim3;
    }
  }
}

/* right state at the left face (i-1/2) of the cell with values (a, b, c) */
static double recon_minus(int lim, double a, double b, double c) {
  double dm = b - a, dp = c - b;
  /* cada3: the same rule on the mirrored stencil (c, b, a) */
  if (lim == 10) return b + cada3_face(-dp, -dm);
  if (lim == 12) return b - venk_increment(a, b, c);
  if (!(dm * dp > 0.0)) return b;
  if (lim >= 3) return b - 0.5 * sym_slope(lim, dm, dp);
  switch (lim) {
    case 0: return b - 0.5 * minmod2(dm, dp);
    case 1: return b - 0.5 * (2.0 * dm * dp / (dm + dp));
    default: {
      double am = fabs(dm), ap = fabs(dp);
      double lim3 = dmin(dmin(2.0 * ap, (ap + 2.0 * am) / 3.0), 2.0 * am);
      return b - 0.5 * sgn(dm) * lim3;
    }
  }
}

void orc_reconstruct(int limiter, const double* w, int n, double* wl, double* wr) {
  for (int i = 1; i + 1 < n; i++) {
    wl[i] = recon_plus(limiter, w[i - 1], w[i], w[i + 1]);
    wr[i] = recon_minus(limiter, w[i - 1], w[i], w[i + 1]);
  }
}

/* Five-point limiters of the limiter table (3 ghost cells), each giving the
 * left state at the face i+1/2 of cell i from v = (v_{i-2}, ..., v_{i+2}); the
 * right state at i-1/2 is the same formula on the mirrored stencil.
 *   7 mp5 (Suresh & Huynh 1997): the fifth-order interface polynomial
 *     (2 v_{i-2} - 13 v_{i-1} + 47 v_i + 27 v_{i+1} - 3 v_{i+2}) / 60, kept when
 *     it lies between v_i and the monotonicity bound v_i + minmod(v_{i+1} - v_i,
 *     4 (v_i - v_{i-1})); otherwise clipped to the interval built from the
 *     upper limit v_i + 4 (v_i - v_{i-1}), the median and the large-curvature
 *     values with the minmod4 of the second differences.
 *   8 weno5 (Jiang & Shu 1996): convex combination of the three third-order
 *     candidates with the smoothness indicators beta_k and the linear weights
 *     (1, 6, 3)/10, alpha_k = d_k / (eps + beta_k)^2, eps = 1e-6.
 *   9 wenoz5 (Borges et al. 2008): the same candidates with
 *     alpha_k = d_k (1 + tau5 / (beta_k + eps)), tau5 = |beta_0 - beta_2|,
 *     exponent 1, eps = 1e-40.
 *  11 wenozp5 (WENO-Z+, Acker, Borges & Costa 2016): the same candidates with
 *     alpha_k = d_k (1 + (tau5 / (beta_k + eps))^2
 *                      + lambda (beta_k + eps) / (tau5 + eps)),
 *     eps = 1e-40, lambda = dx^(2/3) with dx the cell width along the
 *     reconstruction (the value the authors recommend). */
static double minmod4(double w, double x, double y, double z) {
  if (w > 0.0 && x > 0.0 && y > 0.0 && z > 0.0) return dmin(dmin(w, x), dmin(y, z));
  if (w < 0.0 && x < 0.0 && y < 0.0 && z < 0.0) return dmax(dmax(w, x), dmax(y, z));
  return 0.0;
}

static double mp5_plus(const double* v) {
  const double a = 4.0;
  const double vm2 = v[0], vm1 = v[1], v0 = v[2], vp1 = v[3], vp2 = v[4];
  const double vor = (2.0 * vm2 - 13.0 * vm1 + 47.0 * v0 + 27.0 * vp1 - 3.0 * vp2) / 60.0;
  const double vmp = v0 + minmod2(vp1 - v0, a * (v0 - vm1));
  if ((vor - v0) * (vor - vmp) <= 0.0) return vor;
  const double djm1 = vm2 - 2.0 * vm1 + v0;
  const double dj = vm1 - 2.0 * v0 + vp1;
  const double djp1 = v0 - 2.0 * vp1 + vp2;
  const double dp = minmod4(4.0 * dj - djp1, 4.0 * djp1 - dj, dj, djp1);
  const double dm = minmod4(4.0 * dj - djm1, 4.0 * djm1 - dj, dj, djm1);
  const double vul = v0 + a * (v0 - vm1);
  const double vav = 0.5 * (v0 + vp1);
  const double vmd = vav - 0.5 * dp;
  const double vlc = v0 + 0.5 * (v0 - vm1) + 4.0 / 3.0 * dm;
  const double vmin = dmax(dmin(dmin(v0, vp1), vmd), dmin(dmin(v0, vul), vlc));
  const double vmax = dmin(dmax(dmax(v0, vp1), vmd), dmax(dmax(v0, vul), vlc));
  return vor + minmod2(vmin - vor, vmax - vor);
}

/* kind: 0 weno5, 1 wenoz5, 2 wenozp5; dx: cell width along the
 * reconstruction (wenozp5's lambda) */
static double weno5_plus(int kind, const double* v, double dx) {
  const double vm2 = v[0], vm1 = v[1], v0 = v[2], vp1 = v[3], vp2 = v[4];
  const double c13 = 13.0 / 12.0;
  const double t0 = vm2 - 2.0 * vm1 + v0, u0 = vm2 - 4.0 * vm1 + 3.0 * v0;
  const double t1 = vm1 - 2.0 * v0 + vp1, u1 = vm1 - vp1;
  const double t2 = v0 - 2.0 * vp1 + vp2, u2 = 3.0 * v0 - 4.0 * vp1 + vp2;
  const double b0 = c13 * t0 * t0 + 0.25 * u0 * u0;
  const double b1 = c13 * t1 * t1 + 0.25 * u1 * u1;
  const double b2 = c13 * t2 * t2 + 0.25 * u2 * u2;
  const double q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
  const double q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
  const double q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
  double a0, a1, a2;
  if (kind == 2) {
    /* WENO-Z+ (Acker, Borges & Costa 2016): the Z weights with exponent 2
     * plus lambda (beta_k + eps)/(tau5 + eps), which raises the weight of
     * the less smooth candidates; lambda = dx^(2/3) */
    const double eps = 1e-40, tau = fabs(b0 - b2), lam = pow(dx, 2.0 / 3.0);
    const double r0 = tau / (b0 + eps), r1 = tau / (b1 + eps), r2 = tau / (b2 + eps);
    a0 = 0.1 * (1.0 + r0 * r0 + lam * (b0 + eps) / (tau + eps));
    a1 = 0.6 * (1.0 + r1 * r1 + lam * (b1 + eps) / (tau + eps));
    a2 = 0.3 * (1.0 + r2 * r2 + lam * (b2 + eps) / (tau + eps));
  } else if (kind == 1) {
    const double eps = 1e-40, tau = fabs(b0 - b2);
    a0 = 0.1 * (1.0 + tau / (b0 + eps));
    a1 = 0.6 * (1.0 + tau / (b1 + eps));
    a2 = 0.3 * (1.0 + tau / (b2 + eps));
  } else {
    const double eps = 1e-6;
    a0 = 0.1 / ((eps + b0) * (eps + b0));
    a1 = 0.6 / ((eps + b1) * (eps + b1));
    a2 = 0.3 / ((eps + b2) * (eps + b2));
  }
  const double sa = a0 + a1 + a2;
  return (a0 * q0 + a1 * q1 + a2 * q2) / sa;
}

static double recon5_plus(int lim, const double* v, double dx) {
  return lim == 7 ? mp5_plus(v) : weno5_plus(lim == 9 ? 1 : (lim == 11 ? 2 : 0), v, dx);
}

/* right state at i-1/2 of cell i from v = (v_{i-2}, ..., v_{i+2}) */
static double recon5_minus(int lim, const double* v, double dx) {
  const double r[5] = {v[4], v[3], v[2], v[1], v[0]};
  return recon5_plus(lim, r, dx);
}

void orc_reconstruct5(int limiter, const double* w, int n, double dx, double* wl, double* wr) {
  for (int i = 2; i + 2 < n; i++) {
    wl[i] = recon5_plus(limiter, w + i - 2, dx);
    wr[i] = recon5_minus(limiter, w + i - 2, dx);
  }
}

/* the five-point limiters (three ghost cells): mp5, weno5, wenoz5, wenozp5 */
static int five_point(int lim) { return lim == 7 || lim == 8 || lim == 9 || lim == 11; }

int orc_ghost_width(const orc_mesh* m) { return m->ng; }

/* ------------------------------------------------------------------------ */
/* Riemann solvers in the face frame: x = face normal                        */
/* local prim q = (rho, u, v, w, p, Bx, By, Bz);  local cons U, flux F.      */
/* ------------------------------------------------------------------------ */

static void local_cons_flux(double g, const double* q, double bx, double* U, double* F,
                            double* pt_out) {
  double rho = q[0], u = q[1], v = q[2], w = q[3], p = q[4], by = q[6], bz = q[7];
  double b2 = bx * bx + by * by + bz * bz;
  double pt = p + 0.5 * b2;
  double e = p / (g - 1.0) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * b2;
  double vb = u * bx + v * by + w * bz;
  U[0] = rho;
  U[1] = rho * u;
  U[2] = rho * v;
  U[3] = rho * w;
  U[4] = e;
  U[5] = bx;
  U[6] = by;
  U[7] = bz;
  F[0] = rho * u;
  F[1] = rho * u * u + pt - bx * bx;
  F[2] = rho * u * v - bx * by;
  F[3] = rho * u * w - bx * bz;
  F[4] = (e + pt) * u - bx * vb;
  F[5] = 0.0;
  F[6] = by * u - bx * v;
  F[7] = bz * u - bx * w;
  *pt_out = pt;
}

static double local_fast(double g, const double* q, double bx) {
  double rho = q[0];
  double a2 = g * q[4] / rho;
  double bt2 = (q[6] * q[6] + q[7] * q[7]) / rho;
  double b2 = (bx * bx + q[6] * q[6] + q[7] * q[7]) / rho;
  double dd = a2 - b2;
  return sqrt(0.5 * (a2 + b2 + sqrt(dd * dd + 4.0 * a2 * bt2)));
}

/* HLL, Harten, Lax & van Leer 1983 */
static void hll_local(double g, const double* ql, const double* qr, double bx, double* f) {
  double UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(g, ql, bx, UL, FL, &ptl);
  local_cons_flux(g, qr, bx, UR, FR, &ptr);
  double cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  double sl = dmin(ql[1] - cfl, qr[1] - cfr);
  double sr = dmax(ql[1] + cfl, qr[1] + cfr);
  for (int c = 0; c < 8; c++) {
    if (sl >= 0.0) f[c] = FL[c];
    else if (sr <= 0.0) f[c] = FR[c];
    else f[c] = (sr * FL[c] - sl * FR[c] + sl * sr * (UR[c] - UL[c])) / (sr - sl);
  }
}

/* TVD Lax-Friedrichs (the `tvdlf' flux of the flux-scheme table, Sect. 3.2.1):
 * the local Lax-Friedrichs flux with the fastest signal speed of the two sides,
 * c_max = max(|u_L| + c_fL, |u_R| + c_fR):
 *   F = (F_L + F_R)/2 - c_max (U_R - U_L)/2 */
static void tvdlf_local(double g, const double* ql, const double* qr, double bx, double* f) {
  double UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(g, ql, bx, UL, FL, &ptl);
  local_cons_flux(g, qr, bx, UR, FR, &ptr);
  double cl = fabs(ql[1]) + local_fast(g, ql, bx), cr = fabs(qr[1]) + local_fast(g, qr, bx);
  double cmax = dmax(cl, cr);
  for (int c = 0; c < 8; c++) f[c] = 0.5 * (FL[c] + FR[c]) - 0.5 * cmax * (UR[c] - UL[c]);
}

/* HLLC for MHD (the `hllc' flux of the flux-scheme table; the paper prints no
 * formulas and cites a review, so this restates the three-wave solver of
 * Li 2005): HLL speeds; the HLL state U* = (S_R U_R - S_L U_L - F_R + F_L) /
 * (S_R - S_L) gives the contact speed S_M (its momentum over its density),
 * the star magnetic field B* (normal component B_x) and the star velocity v*
 * (its momentum over its density);
 * p_T* = rho_L (S_L - u_L)(S_M - u_L) + p_TL; per side K
 *   rho*_K = rho_K (S_K - u_K)/(S_K - S_M),  (rho u)*_K = rho*_K S_M,
 *   (rho v_t)*_K = [rho_K v_tK (S_K - u_K) - (B_x B*_t - B_x B_tK)]/(S_K - S_M),
 *   e*_K = [e_K (S_K - u_K) + p_T* S_M - p_TK u_K - B_x (v*.B* - v_K.B_K)]/(S_K - S_M),
 * flux F*_K = F_K + S_K (U*_K - U_K), region by S_L, S_M, S_R. */
static void hllc_local(double g, const double* ql, const double* qr, double bx, double* f) {
  double UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(g, ql, bx, UL, FL, &ptl);
  local_cons_flux(g, qr, bx, UR, FR, &ptr);
  double cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  double sl = dmin(ql[1] - cfl, qr[1] - cfr);
  double sr = dmax(ql[1] + cfl, qr[1] + cfr);
  if (sl >= 0.0) {
    for (int c = 0; c < 8; c++) f[c] = FL[c];
    return;
  }
  if (sr <= 0.0) {
    for (int c = 0; c < 8; c++) f[c] = FR[c];
    return;
  }
  double uh[8];
  for (int c = 0; c < 8; c++) uh[c] = (sr * UR[c] - sl * UL[c] - FR[c] + FL[c]) / (sr - sl);
  const double sm = uh[1] / uh[0];
  const double vs[3] = {sm, uh[2] / uh[0], uh[3] / uh[0]};
  const double bs[3] = {bx, uh[6], uh[7]};
  const double pts = ql[0] * (sl - ql[1]) * (sm - ql[1]) + ptl;
  const double vbs = vs[0] * bs[0] + vs[1] * bs[1] + vs[2] * bs[2];
  const double* q = sm >= 0.0 ? ql : qr;
  const double* U = sm >= 0.0 ? UL : UR;
  const double* F = sm >= 0.0 ? FL : FR;
  const double S = sm >= 0.0 ? sl : sr;
  const double pt = sm >= 0.0 ? ptl : ptr;
  const double su = S - q[1], ssm = S - sm;
  const double vb = q[1] * bx + q[2] * q[6] + q[3] * q[7];
  double Us[8];
  Us[0] = q[0] * su / ssm;
  Us[1] = Us[0] * sm;
  Us[2] = (q[0] * q[2] * su - (bx * bs[1] - bx * q[6])) / ssm;
  Us[3] = (q[0] * q[3] * su - (bx * bs[2] - bx * q[7])) / ssm;
  Us[4] = (U[4] * su + pts * sm - pt * q[1] - bx * (vbs - vb)) / ssm;
  Us[5] = bx;
  Us[6] = bs[1];
  Us[7] = bs[2];
  for (int c = 0; c < 8; c++) f[c] = F[c] + S * (Us[c] - U[c]);
}

/* one side of the HLLD single-star state, Miyoshi & Kusano 2005 */
typedef struct {
  double rs, vs, ws, bys, bzs, es;
} star_t;

static star_t hlld_star(double g, const double* q, const double* U, double pt, double s,
                        double sm, double pts, double bx) {
  (void)g;
  star_t r;
  double rho = q[0], u = q[1], v = q[2], w = q[3], by = q[6], bz = q[7];
  double su = s - u;
  r.rs = rho * su / (s - sm);
  double big = rho * su * (s - sm);
  double den = big - bx * bx;
  double scale = dmax(fabs(big), bx * bx);
  if (fabs(den) <= 1e-8 * scale) {
    r.vs = v;
    r.ws = w;
    r.bys = by;
    r.bzs = bz;
  } else {
    double tv = bx * (sm - u) / den;
    double tb = (rho * su * su - bx * bx) / den;
    r.vs = v - by * tv;
    r.ws = w - bz * tv;
    r.bys = by * tb;
    r.bzs = bz * tb;
  }
  double vb = u * bx + v * by + w * bz;
  double vbs = sm * bx + r.vs * r.bys + r.ws * r.bzs;
  r.es = (su * U[4] - pt * u + pts * sm + bx * (vb - vbs)) / (s - sm);
  return r;
}

static void hlld_local(double g, const double* ql, const double* qr, double bx, double* f) {
  double UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(g, ql, bx, UL, FL, &ptl);
  local_cons_flux(g, qr, bx, UR, FR, &ptr);
  double cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  double ul = ql[1], ur = qr[1];
  double cmax = dmax(cfl, cfr);
  double sl = dmin(ul, ur) - cmax;
  double sr = dmax(ul, ur) + cmax;
  if (sl > 0.0) {
    for (int c = 0; c < 8; c++) f[c] = FL[c];
    return;
  }
  if (sr < 0.0) {
    for (int c = 0; c < 8; c++) f[c] = FR[c];
    return;
  }
  double rl = ql[0], rr = qr[0];
  double sul = sl - ul, sur = sr - ur;
  double den = sur * rr - sul * rl;
  double sm = (sur * rr * ur - sul * rl * ul - ptr + ptl) / den;
  double pts = (sur * rr * ptl - sul * rl * ptr + rl * rr * sur * sul * (ur - ul)) / den;
  star_t L = hlld_star(g, ql, UL, ptl, sl, sm, pts, bx);
  star_t R = hlld_star(g, qr, UR, ptr, sr, sm, pts, bx);
  double sqrl = sqrt(L.rs), sqrr = sqrt(R.rs);
  double ssl = sm - fabs(bx) / sqrl, ssr = sm + fabs(bx) / sqrr;
  double sb = sgn(bx);
  double ssum = sqrl + sqrr;
  double vss = (sqrl * L.vs + sqrr * R.vs + (R.bys - L.bys) * sb) / ssum;
  double wss = (sqrl * L.ws + sqrr * R.ws + (R.bzs - L.bzs) * sb) / ssum;
  double byss = (sqrl * R.bys + sqrr * L.bys + sqrl * sqrr * (R.vs - L.vs) * sb) / ssum;
  double bzss = (sqrl * R.bzs + sqrr * L.bzs + sqrl * sqrr * (R.ws - L.ws) * sb) / ssum;
  double vbss = sm * bx + vss * byss + wss * bzss;
  double essl = L.es - sqrl * (sm * bx + L.vs * L.bys + L.ws * L.bzs - vbss) * sb;
  double essr = R.es + sqrr * (sm * bx + R.vs * R.bys + R.ws * R.bzs - vbss) * sb;

  /* star and double-star conserved states */
  double USL[8] = {L.rs, L.rs * sm, L.rs * L.vs, L.rs * L.ws, L.es, bx, L.bys, L.bzs};
  double USR[8] = {R.rs, R.rs * sm, R.rs * R.vs, R.rs * R.ws, R.es, bx, R.bys, R.bzs};
  double USSL[8] = {L.rs, L.rs * sm, L.rs * vss, L.rs * wss, essl, bx, byss, bzss};
  double USSR[8] = {R.rs, R.rs * sm, R.rs * vss, R.rs * wss, essr, bx, byss, bzss};
  for (int c = 0; c < 8; c++) {
    double fsl = FL[c] + sl * (USL[c] - UL[c]);
    double fsr = FR[c] + sr * (USR[c] - UR[c]);
    if (ssl >= 0.0) f[c] = fsl;
    else if (sm >= 0.0) f[c] = fsl + ssl * (USSL[c] - USL[c]);
    else if (ssr >= 0.0) f[c] = fsr + ssr * (USSR[c] - USR[c]);
    else f[c] = fsr;
  }
}

/* Face flux along dir from primitive states wl, wr (global frame, 9 entries).
 * glm: B_n* and psi* from the (B_n, psi) subsystem (Dedner 2002), then the MHD
 * flux with B_n = B_n* on both sides; F(B_n) = psi*, F(psi) = c_h^2 B_n*.
 * Without glm: B_n = mean of the two sides, F(B_n) = F(psi) = 0. */
void orc_face_flux(int flux, int glm, double gamma, double ch, int dir, const double* wl,
                   const double* wr, double* f) {
  int t1 = (dir + 1) % 3, t2 = (dir + 2) % 3;
  double bnl = wl[5 + dir], bnr = wr[5 + dir];
  double bns, psis;
  if (glm) {
    bns = 0.5 * (bnl + bnr) - (wr[8] - wl[8]) / (2.0 * ch);
    psis = 0.5 * (wl[8] + wr[8]) - 0.5 * ch * (bnr - bnl);
  } else {
    bns = 0.5 * (bnl + bnr);
    psis = 0.0;
  }
  double ql[8] = {wl[0], wl[1 + dir], wl[1 + t1], wl[1 + t2], wl[4], bns, wl[5 + t1], wl[5 + t2]};
  double qr[8] = {wr[0], wr[1 + dir], wr[1 + t1], wr[1 + t2], wr[4], bns, wr[5 + t1], wr[5 + t2]};
  double fl[8];
  if (flux == 0) hll_local(gamma, ql, qr, bns, fl);
  else if (flux == 1) hlld_local(gamma, ql, qr, bns, fl);
  else if (flux == 2) tvdlf_local(gamma, ql, qr, bns, fl);
  else hllc_local(gamma, ql, qr, bns, fl);
  f[RHO] = fl[0];
  f[MX + dir] = fl[1];
  f[MX + t1] = fl[2];
  f[MX + t2] = fl[3];
  f[EN] = fl[4];
  f[BXV + dir] = glm ? psis : 0.0;
  f[BXV + t1] = fl[6];
  f[BXV + t2] = fl[7];
  f[PSI] = glm ? ch * ch * bns : 0.0;
}

/* Shu-Osher coefficients of stage k (Sect. 3, time-integration table):
 *   out  = a  U0 + b  (Uk + c  dt L(Uk))
 *   out2 = a2 U2 + b2 (Uk + c2 dt L(Uk))   (b2 != 0 only in stage 3 of SSPRK(5,4))
 * SSPRK(2,2) (Heun) and SSPRK(3,3): Gottlieb 2005.  SSPRK(4,3) and SSPRK(5,4):
 * the optimal schemes of Spiteri & Ruuth 2002 (cited by the table), written as
 *   SSPRK(4,3): u1 = u0 + dt/2 L(u0); u2 = u1 + dt/2 L(u1);
 *               u3 = 2/3 u0 + 1/3 (u2 + dt/2 L(u2)); u4 = u3 + dt/2 L(u3)
 *   SSPRK(5,4): u1 = u0 + 0.391752226571890 dt L(u0)
 *               u2 = 0.444370493651235 u0 + 0.555629506348765 u1
 *                    + 0.368410593050371 dt L(u1)
 *               u3 = 0.620101851488403 u0 + 0.379898148511597 u2
 *                    + 0.251891774271694 dt L(u2)
 *               u4 = 0.178079954393132 u0 + 0.821920045606868 u3
 *                    + 0.544974750228521 dt L(u3)
 *               u5 = 0.517231671970585 u2 + 0.096059710526147 u3
 *                    + 0.063692468666290 dt L(u3) + 0.386708617503269 u4
 *                    + 0.226007483236906 dt L(u4)
 * For SSPRK(5,4) stage 3 also returns w = 0.517... u2 + 0.096... u3 + 0.0636...
 * dt L(u3) (out2), and stage 4 is u5 = w + 0.386... u4 + 0.226... dt L(u4) with
 * U0 = w.  co = {a, b, c, a2, b2, c2}. */
void orc_stage_coeffs6(int time, int k, double* co) {
  double a = 0.0, b = 1.0, c = 1.0, a2 = 0.0, b2 = 0.0, c2 = 0.0;
  if (time == 0) {
    if (k == 1) a = 0.5, b = 0.5;
  } else if (time == 1) {
    if (k == 1) a = 0.75, b = 0.25;
    else if (k == 2) a = 1.0 / 3.0, b = 2.0 / 3.0;
  } else if (time == 2) {
    c = 0.5;
    if (k == 2) a = 2.0 / 3.0, b = 1.0 / 3.0;
  } else {
    switch (k) {
      case 0: c = 0.391752226571890; break;
      case 1:
        a = 0.444370493651235, b = 0.555629506348765;
        c = 0.368410593050371 / b;
        break;
      case 2:
        a = 0.620101851488403, b = 0.379898148511597;
        c = 0.251891774271694 / b;
        break;
      case 3:
        a = 0.178079954393132, b = 0.821920045606868;
        c = 0.544974750228521 / b;
        a2 = 0.517231671970585, b2 = 0.096059710526147;
        c2 = 0.063692468666290 / b2;
        break;
      default:
        a = 1.0, b = 0.386708617503269;
        c = 0.226007483236906 / b;
        break;
    }
  }
  co[0] = a, co[1] = b, co[2] = c, co[3] = a2, co[4] = b2, co[5] = c2;
}

int orc_num_stages(int time) { return time == 0 ? 2 : time == 1 ? 3 : time == 2 ? 4 : 5; }

void orc_stage_coeffs(int time, int k, double* a, double* b) {
  double co[6];
  orc_stage_coeffs6(time, k, co);
  *a = co[0];
  *b = co[1];
}

/* ------------------------------------------------------------------------ */
/* ghost values                                                              */
/* ------------------------------------------------------------------------ */

static int is_active(const orc_mesh* m, int d) { return d < m->cfg.ndim; }

/* Conserved value of the level-L cell p of instance inst (p may lie outside
 * the domain).  Recursive definition of the AMR ghost value. */
static void value_in(const orc_mesh* m, const double* U, int inst, int L, const long* p,
                     double* out);

/* value of the level-L cell p of an instance, p anywhere up to a few cells
 * outside the domain: periodic wrap; outflow takes the nearest in-domain cell
 * of the level (zero gradient); a symmetric (reflecting) wall takes the
 * mirror cell across the boundary with the normal momentum and the normal
 * magnetic field negated */
static void value_at(const orc_mesh* m, const double* U, int inst, int L, const long* pin,
                     double* out) {
  long p[3] = {pin[0], pin[1], pin[2]};
  int flip[3] = {0, 0, 0};
  for (int d = 0; d < 3; d++) {
    if (!is_active(m, d)) {
      p[d] = 0;
      continue;
    }
    long N = cells_at_level(m, inst, L, d);
    if (p[d] < 0 || p[d] >= N) {
      const int bc = m->cfg.bc[d][p[d] < 0 ? 0 : 1];
      if (bc == 0) {
        p[d] = ((p[d] % N) + N) % N;
      } else if (bc == 2) {
        p[d] = p[d] < 0 ? -1 - p[d] : 2 * N - 1 - p[d];
        flip[d] = 1;
      } else {
        p[d] = p[d] < 0 ? 0 : N - 1;
      }
    }
  }
  value_in(m, U, inst, L, p, out);
  for (int d = 0; d < 3; d++)
    if (flip[d]) {
      out[MX + d] = -out[MX + d];
      out[BXV + d] = -out[BXV + d];
    }
}

/* value of the in-domain level-L cell p: leaf copy, restriction or
 * prolongation */
static void value_in(const orc_mesh* m, const double* U, int inst, int L, const long* p,
                     double* out) {
  long bp[3], c[3];
  for (int d = 0; d < 3; d++) {
    bp[d] = p[d] / m->cfg.nx[d];
    c[d] = p[d] - bp[d] * m->cfg.nx[d];
  }
  int r = hget(m, mkkey(inst, L, bp[0], bp[1], bp[2]));
  if (r >= 0) {
    long cell = (c[2] * m->cfg.nx[1] + c[1]) * m->cfg.nx[0] + c[0];
    for (int v = 0; v < NV; v++)
      out[v] = U[((size_t)v * m->nblocks + r) * m->ncell + cell];
    return;
  }
  if (r == -1) {
    /* finer: mean of the 2^d children, children loop z, y, x (x fastest) */
    double sum[NV] = {0};
    int nchild = 0;
    for (int oz = 0; oz < (is_active(m, 2) ? 2 : 1); oz++)
      for (int oy = 0; oy < (is_active(m, 1) ? 2 : 1); oy++)
        for (int ox = 0; ox < 2; ox++) {
          long q[3] = {2 * p[0] + ox, is_active(m, 1) ? 2 * p[1] + oy : 0,
                       is_active(m, 2) ? 2 * p[2] + oz : 0};
          double tmp[NV];
          value_at(m, U, inst, L + 1, q, tmp);
          for (int v = 0; v < NV; v++) sum[v] += tmp[v];
          nchild++;
        }
    for (int v = 0; v < NV; v++) out[v] = sum[v] * (1.0 / nchild);
    return;
  }
  /* coarser: prolongation from the parent-level cell q = floor(p/2) */
  long q[3], o[3];
  for (int d = 0; d < 3; d++) {
    q[d] = is_active(m, d) ? p[d] / 2 : 0;
    o[d] = p[d] - 2 * q[d];
  }
  double uc[NV];
  value_at(m, U, inst, L - 1, q, uc);
  for (int v = 0; v < NV; v++) out[v] = uc[v];
  for (int d = 0; d < 3; d++) {
    if (!is_active(m, d)) continue;
    long qm[3] = {q[0], q[1], q[2]}, qp[3] = {q[0], q[1], q[2]};
    qm[d] -= 1;
    qp[d] += 1;
    double um[NV], up[NV];
    value_at(m, U, inst, L - 1, qm, um);
    value_at(m, U, inst, L - 1, qp, up);
    double wgt = o[d] == 0 ? -0.25 : 0.25;
    for (int v = 0; v < NV; v++) out[v] = out[v] + wgt * minmod2(uc[v] - um[v], up[v] - uc[v]);
  }
}

/* ------------------------------------------------------------------------ */
/* mesh construction                                                         */
/* ------------------------------------------------------------------------ */

void orc_destroy(orc_mesh* m) {
  if (!m) return;
  free(m->fkind);
  free(m->facef);
  free(m->inst);
  free(m->blk);
  free(m->hkey);
  free(m->hval);
  free(m->hused);
  free(m);
}

void orc_set_threads(orc_mesh* m, int n) { m->nthreads = n < 1 ? 1 : n; }

orc_mesh* orc_create(const orc_config* cfg, int ninst, const orc_instance* inst, int nblocks,
                     const int32_t* meta, char* err, int errlen) {
#define FAIL(...)                                   \
  do {                                              \
    if (err) snprintf(err, (size_t)errlen, __VA_ARGS__); \
    orc_destroy(m);                                 \
    return NULL;                                    \
  } while (0)
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  if (!m) return NULL;
  m->cfg = *cfg;
  m->ninst = ninst;
  m->nblocks = nblocks;
  m->nthreads = 1;
  if (cfg->ndim < 1 || cfg->ndim > 3) FAIL("ndim must be 1..3");
  if (cfg->limiter < 0 || cfg->limiter > 12) FAIL("limiter must be 0..12");
  for (int d = 0; d < cfg->ndim; d++)
    for (int side = 0; side < 2; side++)
      if (cfg->bc[d][side] < 0 || cfg->bc[d][side] > 2) FAIL("bc must be 0..2");
  m->ng = five_point(cfg->limiter) ? NG5 : NG;
  for (int L = 0; L < 16; L++) {
    if (cfg->level_limiter[L] > 12) FAIL("level_limiter must be -1..12");
    if (cfg->level_limiter[L] >= 0 && five_point(cfg->level_limiter[L])) m->ng = NG5;
  }
  for (int d = 0; d < 3; d++) {
    if (d >= cfg->ndim) m->cfg.nx[d] = 1;
    else if (cfg->nx[d] < m->ng) FAIL("block must have at least as many cells as ghost cells");
  }
  m->ncell = m->cfg.nx[0] * m->cfg.nx[1] * m->cfg.nx[2];
  m->inst = (orc_instance*)malloc(sizeof(orc_instance) * (size_t)ninst);
  m->blk = (blockinfo*)malloc(sizeof(blockinfo) * (size_t)(nblocks > 0 ? nblocks : 1));
  memcpy(m->inst, inst, sizeof(orc_instance) * (size_t)ninst);
  for (int q = 0; q < ninst; q++)
    for (int d = cfg->ndim; d < 3; d++) m->inst[q].base[d] = 1;
  int maxlev = 0;
  for (int b = 0; b < nblocks; b++) {
    const int32_t* r = meta + 5 * b;
    m->blk[b].inst = r[0];
    m->blk[b].level = r[1];
    for (int d = 0; d < 3; d++) m->blk[b].idx[d] = d < cfg->ndim ? r[2 + d] : 0;
    if (r[0] < 0 || r[0] >= ninst) FAIL("block %d: bad instance", b);
    if (r[1] < 0 || r[1] > 15) FAIL("block %d: bad level", b);
    for (int d = 0; d < cfg->ndim; d++)
      if (r[2 + d] < 0 || r[2 + d] >= blocks_at_level(m, r[0], r[1], d) || r[2 + d] >= 8192)
        FAIL("block %d: index out of range", b);
    if (r[1] > maxlev) maxlev = r[1];
  }
  size_t cap = 16;
  while (cap < (size_t)4 * (size_t)(nblocks + 1) * (size_t)(maxlev + 1)) cap <<= 1;
  m->hcap = cap;
  m->hkey = (uint64_t*)calloc(cap, sizeof(uint64_t));
  m->hval = (int*)calloc(cap, sizeof(int));
  m->hused = (unsigned char*)calloc(cap, 1);
  for (int b = 0; b < nblocks; b++) {
    blockinfo* B = &m->blk[b];
    if (hput(m, mkkey(B->inst, B->level, B->idx[0], B->idx[1], B->idx[2]), b) != -2)
      FAIL("block %d duplicates another block", b);
  }
  for (int b = 0; b < nblocks; b++) {
    blockinfo* B = &m->blk[b];
    long p[3] = {B->idx[0], B->idx[1], B->idx[2]};
    for (int L = B->level - 1; L >= 0; L--) {
      for (int d = 0; d < 3; d++) p[d] /= 2;
      int old = hget(m, mkkey(B->inst, L, p[0], p[1], p[2]));
      if (old >= 0) FAIL("block %d overlaps block %d", b, old);
      hput(m, mkkey(B->inst, L, p[0], p[1], p[2]), -1);
    }
  }
  /* coverage: every level-0 position is a leaf or refined; every refined
   * position has all children present */
  for (int q = 0; q < ninst; q++) {
    for (long k = 0; k < blocks_at_level(m, q, 0, 2); k++)
      for (long j = 0; j < blocks_at_level(m, q, 0, 1); j++)
        for (long i = 0; i < blocks_at_level(m, q, 0, 0); i++)
          if (hget(m, mkkey(q, 0, i, j, k)) == -2) FAIL("instance %d: hole at level 0", q);
  }
  for (size_t s = 0; s < m->hcap; s++) {
    if (!m->hused[s] || m->hval[s] != -1) continue;
    uint64_t key = m->hkey[s];
    int q = (int)(key >> 43), L = (int)((key >> 39) & 15);
    long i = (long)((key >> 26) & 8191), j = (long)((key >> 13) & 8191), k = (long)(key & 8191);
    for (int oz = 0; oz < (cfg->ndim > 2 ? 2 : 1); oz++)
      for (int oy = 0; oy < (cfg->ndim > 1 ? 2 : 1); oy++)
        for (int ox = 0; ox < 2; ox++)
          if (hget(m, mkkey(q, L + 1, 2 * i + ox, 2 * j + oy, 2 * k + oz)) == -2)
            FAIL("instance %d: hole below level %d", q, L);
  }
  /* full 2:1 balance: the leaf covering any neighbour position of a leaf at
   * level L is at level >= L-1 */
  for (int b = 0; b < nblocks; b++) {
    blockinfo* B = &m->blk[b];
    int lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
      lo[d] = d < cfg->ndim ? -1 : 0;
      hi[d] = d < cfg->ndim ? 1 : 0;
    }
    for (int dz = lo[2]; dz <= hi[2]; dz++)
      for (int dy = lo[1]; dy <= hi[1]; dy++)
        for (int dx = lo[0]; dx <= hi[0]; dx++) {
          if (!dx && !dy && !dz) continue;
          long p[3] = {B->idx[0] + dx, B->idx[1] + dy, B->idx[2] + dz};
          int out = 0;
          for (int d = 0; d < cfg->ndim; d++) {
            long N = blocks_at_level(m, B->inst, B->level, d);
            if (p[d] < 0 || p[d] >= N) {
              if (cfg->bc[d][p[d] < 0 ? 0 : 1] == 0) p[d] = ((p[d] % N) + N) % N;
              else out = 1;
            }
          }
          if (out) continue;
          int L = B->level;
          int r = hget(m, mkkey(B->inst, L, p[0], p[1], p[2]));
          while (r == -2 && L > 0) {
            L--;
            for (int d = 0; d < 3; d++) p[d] /= 2;
            r = hget(m, mkkey(B->inst, L, p[0], p[1], p[2]));
          }
          if (r == -2) FAIL("block %d: neighbour not covered", b);
          if (L < B->level - 1) FAIL("block %d (level %d) touches level %d: not 2:1", b, B->level, L);
        }
  }
  if (cfg->reflux) {
    /* face kinds for refluxing: 1 = the neighbour region is finer (this block
     * is the coarse side), 2 = coarser, 0 otherwise */
    m->farea = 1;
    for (int d = 0; d < cfg->ndim; d++) {
      int a = 1;
      for (int e = 0; e < cfg->ndim; e++)
        if (e != d) a *= m->cfg.nx[e];
      if (a > m->farea) m->farea = a;
    }
    m->fkind = (unsigned char*)calloc((size_t)nblocks * 6, 1);
    m->facef = (double*)calloc((size_t)nblocks * 6 * NV * m->farea, sizeof(double));
    for (int b = 0; b < nblocks; b++) {
      const blockinfo* B = &m->blk[b];
      for (int d = 0; d < cfg->ndim; d++)
        for (int side = 0; side < 2; side++) {
          long id[3] = {B->idx[0], B->idx[1], B->idx[2]};
          id[d] += side ? 1 : -1;
          long N = blocks_at_level(m, B->inst, B->level, d);
          if (id[d] < 0 || id[d] >= N) {
            if (cfg->bc[d][side] != 0) continue;
            id[d] = (id[d] % N + N) % N;
          }
          int r = hget(m, mkkey(B->inst, B->level, id[0], id[1], id[2]));
          m->fkind[b * 6 + d * 2 + side] = r >= 0 ? 0 : (r == -1 ? 1 : 2);
        }
    }
  }
  return m;
#undef FAIL
}

/* ------------------------------------------------------------------------ */
/* block operations                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  int P[3];   /* padded extents */
  int g[3];   /* ghost width per dim (2 active, 0 inactive) */
  size_t np;  /* padded cells */
} padinfo;

static padinfo pad_of(const orc_mesh* m) {
  padinfo p;
  p.np = 1;
  for (int d = 0; d < 3; d++) {
    p.g[d] = is_active(m, d) ? m->ng : 0;
    p.P[d] = m->cfg.nx[d] + 2 * p.g[d];
    p.np *= (size_t)p.P[d];
  }
  return p;
}

static size_t pidx(const padinfo* pi, int i, int j, int k) {
  return ((size_t)(k + pi->g[2]) * pi->P[1] + (size_t)(j + pi->g[1])) * pi->P[0] +
         (size_t)(i + pi->g[0]);
}

static void cell_dx(const orc_mesh* m, int inst, int L, double* dx) {
  for (int d = 0; d < 3; d++) {
    if (!is_active(m, d)) dx[d] = 1.0;
    else dx[d] = (m->inst[inst].xmax[d] - m->inst[inst].xmin[d]) / (double)cells_at_level(m, inst, L, d);
  }
}

/* conserved values of block b on its padded box (interior + face slabs);
 * cons[v * np + pidx] */
static void gather_padded(const orc_mesh* m, const double* U, int b, double* cons) {
  padinfo pi = pad_of(m);
  const blockinfo* B = &m->blk[b];
  const int* nx = m->cfg.nx;
  memset(cons, 0, sizeof(double) * NV * pi.np);
  for (int k = -pi.g[2]; k < nx[2] + pi.g[2]; k++)
    for (int j = -pi.g[1]; j < nx[1] + pi.g[1]; j++)
      for (int i = -pi.g[0]; i < nx[0] + pi.g[0]; i++) {
        int outside = (i < 0 || i >= nx[0]) + (j < 0 || j >= nx[1]) + (k < 0 || k >= nx[2]);
        if (outside > 1) continue;
        double u[NV];
        if (!outside) {
          size_t cell = ((size_t)k * nx[1] + j) * nx[0] + i;
          for (int v = 0; v < NV; v++) u[v] = U[((size_t)v * m->nblocks + b) * m->ncell + cell];
        } else {
          long p[3] = {(long)B->idx[0] * nx[0] + i, (long)B->idx[1] * nx[1] + j,
                       (long)B->idx[2] * nx[2] + k};
          value_at(m, U, B->inst, B->level, p, u);
        }
        size_t pc = pidx(&pi, i, j, k);
        for (int v = 0; v < NV; v++) cons[v * pi.np + pc] = u[v];
      }
}

int orc_fill_ghosts(const orc_mesh* m, const double* U, double* padded) {
  padinfo pi = pad_of(m);
  double* tmp = (double*)malloc(sizeof(double) * NV * pi.np);
  for (int b = 0; b < m->nblocks; b++) {
    gather_padded(m, U, b, tmp);
    for (int v = 0; v < NV; v++)
      memcpy(padded + ((size_t)v * m->nblocks + b) * pi.np, tmp + v * pi.np,
             sizeof(double) * pi.np);
  }
  free(tmp);
  return 0;
}

/* small: density or pressure below its floor, or not positive at all */
static int small_prim(const orc_mesh* m, const double* w) {
  return !(w[0] > 0.0 && w[0] >= m->cfg.small_density) ||
         !(w[4] > 0.0 && w[4] >= m->cfg.small_pressure);
}

/* check_small_values reports small values unless fix_small_values repairs
 * them (Sect. 7.4: with the fix on, the bootstrapping replaces the stop) */
static int small_values(const orc_mesh* m, const double* w) {
  if (!m->cfg.check_small_values || m->cfg.fix_small_values) return 0;
  return small_prim(m, w);
}

/* One stage on one block.  scratch: cons/prim padded (NV*np each) + fluxes. */
static int block_stage(const orc_mesh* m, int b, int k, const double* dtv, const double* chv,
                       const double* U0, const double* Uk, const double* U2, double* out,
                       double* out2, double* scratch) {
  padinfo pi = pad_of(m);
  const blockinfo* B = &m->blk[b];
  const int* nx = m->cfg.nx;
  const double gamma = m->inst[B->inst].gamma;
  const double dt = dtv[B->inst], ch = chv[B->inst];
  const size_t nvb = (size_t)m->nblocks * m->ncell;
  int status = ST_OK;

  double co[6];
  orc_stage_coeffs6(m->cfg.time, k, co);
  const int second = out2 != NULL && co[4] != 0.0;

  if (dt == 0.0) {
    /* finished instance: every stage output is the stage input */
    for (int v = 0; v < NV; v++)
      for (int c = 0; c < m->ncell; c++) {
        size_t at = (size_t)v * nvb + (size_t)b * m->ncell + c;
        double u = Uk[at];
        out[at] = u;
        if (second) out2[at] = u;
      }
    return ST_OK;
  }

  double* cons = scratch;
  double* W = scratch + NV * pi.np;
  double* F[3];
  size_t nf[3];
  double* fp = W + NV * pi.np;
  for (int d = 0; d < 3; d++) {
    nf[d] = (size_t)(nx[0] + (d == 0)) * (nx[1] + (d == 1)) * (nx[2] + (d == 2));
    F[d] = fp;
    fp += NV * nf[d];
  }

  /* 1. ghost fill + conserved -> primitive on interior and face slabs */
  gather_padded(m, Uk, b, cons);
  for (int kk = -pi.g[2]; kk < nx[2] + pi.g[2]; kk++)
    for (int j = -pi.g[1]; j < nx[1] + pi.g[1]; j++)
      for (int i = -pi.g[0]; i < nx[0] + pi.g[0]; i++) {
        int outside = (i < 0 || i >= nx[0]) + (j < 0 || j >= nx[1]) + (kk < 0 || kk >= nx[2]);
        if (outside > 1) continue;
        size_t pc = pidx(&pi, i, j, kk);
        double u[NV], w[NV];
        for (int v = 0; v < NV; v++) u[v] = cons[v * pi.np + pc];
        orc_cons_to_prim(gamma, u, w);
        if (small_values(m, w)) status = ST_SMALL;
        for (int v = 0; v < NV; v++) W[v * pi.np + pc] = w[v];
      }

  /* 2. faces: reconstruction, positivity fallback, glm + Riemann flux, with
   * the scheme of this block's level (every face of a block is computed with
   * the block's scheme) */
  const int flux = m->cfg.level_flux[B->level] >= 0 ? m->cfg.level_flux[B->level] : m->cfg.flux;
  const int lim =
      m->cfg.level_limiter[B->level] >= 0 ? m->cfg.level_limiter[B->level] : m->cfg.limiter;
  double dxl[3]; /* this level's cell widths (wenozp5's lambda) */
  cell_dx(m, B->inst, B->level, dxl);
  for (int d = 0; d < m->cfg.ndim; d++) {
    int ext[3] = {nx[0], nx[1], nx[2]};
    ext[d] += 1;
    for (int kk = 0; kk < ext[2]; kk++)
      for (int j = 0; j < ext[1]; j++)
        for (int i = 0; i < ext[0]; i++) {
          /* face between cell (f-1) and cell f along d, f = (i,j,k)[d] */
          int c[3] = {i, j, kk};
          double wl[NV], wr[NV], w1[NV], w0[NV];
          for (int v = 0; v < NV; v++) {
            /* s[t] = cell f - 3 + t along d (the outer two only with 3 ghosts) */
            double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int t = m->ng == NG5 ? 0 : 1; t < (m->ng == NG5 ? 6 : 5); t++) {
              int cc[3] = {c[0], c[1], c[2]};
              cc[d] += t - 3;
              s[t] = W[v * pi.np + pidx(&pi, cc[0], cc[1], cc[2])];
            }
            if (five_point(lim)) {
              wl[v] = recon5_plus(lim, s, dxl[d]);
              wr[v] = recon5_minus(lim, s + 1, dxl[d]);
            } else {
              wl[v] = recon_plus(lim, s[1], s[2], s[3]);
              wr[v] = recon_minus(lim, s[2], s[3], s[4]);
            }
            w0[v] = s[2];
            w1[v] = s[3];
          }
          if (!(wl[0] > 0.0) || !(wl[4] > 0.0) || !(wr[0] > 0.0) || !(wr[4] > 0.0)) {
            for (int v = 0; v < NV; v++) {
              wl[v] = w0[v];
              wr[v] = w1[v];
            }
          }
          double f[NV];
          orc_face_flux(flux, m->cfg.glm, gamma, ch, d, wl, wr, f);
          size_t fi = ((size_t)kk * ext[1] + j) * ext[0] + i;
          for (int v = 0; v < NV; v++) F[d][v * nf[d] + fi] = f[v];
        }
  }

  /* 2b. refluxing: keep the fluxes of this block's level-change faces */
  if (m->cfg.reflux) {
    for (int d = 0; d < m->cfg.ndim; d++) {
      int ext[3] = {nx[0], nx[1], nx[2]};
      ext[d] += 1;
      const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2; /* tangential dims in order */
      for (int side = 0; side < 2; side++) {
        if (!m->fkind[b * 6 + d * 2 + side]) continue;
        double* dst = m->facef + ((size_t)b * 6 + d * 2 + side) * NV * m->farea;
        for (int t2 = 0; t2 < nx[tb]; t2++)
          for (int t1 = 0; t1 < nx[ta]; t1++) {
            int c[3];
            c[d] = side ? nx[d] : 0;
            c[ta] = t1;
            c[tb] = t2;
            size_t fi = ((size_t)c[2] * ext[1] + c[1]) * ext[0] + c[0];
            for (int v = 0; v < NV; v++)
              dst[(size_t)v * m->farea + (size_t)t2 * nx[ta] + t1] = F[d][v * nf[d] + fi];
          }
      }
    }
  }

  /* 3. update: Euler sub-step, psi damping, convex combination */
  double dx[3];
  cell_dx(m, B->inst, B->level, dx);
  double dxmin = dx[0];
  for (int d = 1; d < m->cfg.ndim; d++) dxmin = dmin(dxmin, dx[d]);
  /* psi damping over each Euler part's time step c dt */
  double damp = m->cfg.glm ? exp(-m->cfg.glm_alpha * ch * (co[2] * dt) / dxmin) : 1.0;
  double damp2 = m->cfg.glm ? exp(-m->cfg.glm_alpha * ch * (co[5] * dt) / dxmin) : 1.0;
  const double a = co[0], bb = co[1];
  for (int kk = 0; kk < nx[2]; kk++)
    for (int j = 0; j < nx[1]; j++)
      for (int i = 0; i < nx[0]; i++) {
        size_t cell = ((size_t)kk * nx[1] + j) * nx[0] + i;
        for (int v = 0; v < NV; v++) {
          double acc = 0.0;
          for (int d = 0; d < m->cfg.ndim; d++) {
            int ext[3] = {nx[0], nx[1], nx[2]};
            ext[d] += 1;
            int cm[3] = {i, j, kk}, cp[3] = {i, j, kk};
            cp[d] += 1;
            size_t fm = ((size_t)cm[2] * ext[1] + cm[1]) * ext[0] + cm[0];
            size_t fq = ((size_t)cp[2] * ext[1] + cp[1]) * ext[0] + cp[0];
            acc += (F[d][v * nf[d] + fq] - F[d][v * nf[d] + fm]) / dx[d];
          }
          size_t at = (size_t)v * nvb + (size_t)b * m->ncell + cell;
          double ut = Uk[at] - (co[2] * dt) * acc;
          if (v == PSI) ut = ut * damp;
          /* a plain Euler stage (a = 0, b = 1) does not read U0 */
          double o = (a == 0.0 && bb == 1.0) ? ut : a * U0[at] + bb * ut;
          if (second) {
            double ut2 = Uk[at] - (co[5] * dt) * acc;
            if (v == PSI) ut2 = ut2 * damp2;
            double o2 = co[3] * U2[at] + co[4] * ut2;
            out2[at] = o2; /* U2 and U0 were read above: out2/out may alias them */
          }
          out[at] = o;
        }
      }
  return status;
}

/* ------------------------------------------------------------------------ */
/* refluxing                                                                 */
/* ------------------------------------------------------------------------ */

/* Coarse cells next to a finer neighbour: the stage used the coarse flux of
 * that face; conservation asks for the fine fluxes through it.  One pass over
 * blocks and their faces in a fixed order (a corner cell is corrected by each
 * of its faces in turn). */
static void reflux_pass(const orc_mesh* m, int k, const double* dtv, const double* chv,
                        double* out, double* out2) {
  const int* nx = m->cfg.nx;
  const size_t nvb = (size_t)m->nblocks * m->ncell;
  double co[6];
  orc_stage_coeffs6(m->cfg.time, k, co);
  const int second = out2 != NULL && co[4] != 0.0;
  for (int b = 0; b < m->nblocks; b++) {
    const blockinfo* B = &m->blk[b];
    const double dt = dtv[B->inst], ch = chv[B->inst];
    if (dt == 0.0) continue;
    double dx[3];
    cell_dx(m, B->inst, B->level, dx);
    double dxmin = dx[0];
    for (int d = 1; d < m->cfg.ndim; d++) dxmin = dmin(dxmin, dx[d]);
    const double damp = m->cfg.glm ? exp(-m->cfg.glm_alpha * ch * (co[2] * dt) / dxmin) : 1.0;
    const double damp2 = m->cfg.glm ? exp(-m->cfg.glm_alpha * ch * (co[5] * dt) / dxmin) : 1.0;
    for (int d = 0; d < m->cfg.ndim; d++) {
      const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
      for (int side = 0; side < 2; side++) {
        if (m->fkind[b * 6 + d * 2 + side] != 1) continue;
        const double* fc = m->facef + ((size_t)b * 6 + d * 2 + side) * NV * m->farea;
        for (int t2 = 0; t2 < nx[tb]; t2++)
          for (int t1 = 0; t1 < nx[ta]; t1++) {
            /* fine cells across the face, level L+1 global indices */
            long g[3] = {0, 0, 0};
            g[d] = side ? 2 * ((long)B->idx[d] * nx[d] + nx[d]) : 2 * (long)B->idx[d] * nx[d] - 1;
            long N = cells_at_level(m, B->inst, B->level + 1, d);
            g[d] = (g[d] % N + N) % N; /* periodic (a finer neighbour exists) */
            double fm[NV];
            for (int v = 0; v < NV; v++) fm[v] = 0.0;
            int nf = 0;
            for (int o2 = 0; o2 < (tb < m->cfg.ndim ? 2 : 1); o2++)
              for (int o1 = 0; o1 < (ta < m->cfg.ndim ? 2 : 1); o1++) {
                g[ta] = ta < m->cfg.ndim ? 2 * ((long)B->idx[ta] * nx[ta] + t1) + o1 : 0;
                g[tb] = tb < m->cfg.ndim ? 2 * ((long)B->idx[tb] * nx[tb] + t2) + o2 : 0;
                long bi[3], ci[3];
                for (int e = 0; e < 3; e++) {
                  bi[e] = g[e] / nx[e];
                  ci[e] = g[e] - bi[e] * nx[e];
                }
                int fb = hget(m, mkkey(B->inst, B->level + 1, bi[0], bi[1], bi[2]));
                const double* ff =
                    m->facef + ((size_t)fb * 6 + d * 2 + (1 - side)) * NV * m->farea;
                for (int v = 0; v < NV; v++)
                  fm[v] += ff[(size_t)v * m->farea + ci[tb] * nx[ta] + ci[ta]];
                nf++;
              }
            int c[3];
            c[d] = side ? nx[d] - 1 : 0;
            c[ta] = t1;
            c[tb] = t2;
            size_t cell = ((size_t)c[2] * nx[1] + c[1]) * nx[0] + c[0];
            for (int v = 0; v < NV; v++) {
              double dF = fc[(size_t)v * m->farea + (size_t)t2 * nx[ta] + t1] - fm[v] / nf;
              double dL = (side ? dF : -dF) / dx[d];
              size_t at = (size_t)v * nvb + (size_t)b * m->ncell + cell;
              out[at] += co[1] * (co[2] * dt) * dL * (v == PSI ? damp : 1.0);
              if (second) out2[at] += co[4] * (co[5] * dt) * dL * (v == PSI ? damp2 : 1.0);
            }
          }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* threading over blocks                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_mesh* m;
  int k;
  const double *dt, *ch, *U0, *Uk, *U2;
  double *out, *out2;
  const int32_t* list;
  int n, t, nt;
  int status;
} stage_job;

static size_t scratch_doubles(const orc_mesh* m) {
  padinfo pi = pad_of(m);
  size_t s = 2 * NV * pi.np;
  for (int d = 0; d < 3; d++)
    s += NV * (size_t)(m->cfg.nx[0] + (d == 0)) * (m->cfg.nx[1] + (d == 1)) * (m->cfg.nx[2] + (d == 2));
  return s;
}

static void* stage_worker(void* arg) {
  stage_job* J = (stage_job*)arg;
  double* scratch = (double*)malloc(sizeof(double) * scratch_doubles(J->m));
  J->status = ST_OK;
  for (int q = J->t; q < J->n; q += J->nt) {
    int b = J->list ? J->list[q] : q;
    int s = block_stage(J->m, b, J->k, J->dt, J->ch, J->U0, J->Uk, J->U2, J->out, J->out2,
                        scratch);
    if (s) J->status = s;
  }
  free(scratch);
  return NULL;
}

int orc_stage(const orc_mesh* m, int k, const double* dt, const double* ch, const double* U0,
              const double* Uk, double* out, const int32_t* sub, int nsub) {
  return orc_stage2(m, k, dt, ch, U0, Uk, NULL, out, NULL, sub, nsub);
}

int orc_stage2(const orc_mesh* m, int k, const double* dt, const double* ch, const double* U0,
               const double* Uk, const double* U2, double* out, double* out2,
               const int32_t* sub, int nsub) {
  int n = sub ? nsub : m->nblocks;
  int nt = m->nthreads;
  if (nt > n) nt = n > 0 ? n : 1;
  stage_job* jobs = (stage_job*)calloc((size_t)nt, sizeof(stage_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
  for (int t = 0; t < nt; t++) {
    stage_job J = {m, k, dt, ch, U0, Uk, U2, out, out2, sub, n, t, nt, 0};
    jobs[t] = J;
    if (nt > 1) pthread_create(&th[t], NULL, stage_worker, &jobs[t]);
    else stage_worker(&jobs[t]);
  }
  int status = ST_OK;
  for (int t = 0; t < nt; t++) {
    if (nt > 1) pthread_join(th[t], NULL);
    if (jobs[t].status) status = jobs[t].status;
  }
  free(jobs);
  free(th);
  if (m->cfg.reflux && sub == NULL) reflux_pass(m, k, dt, ch, out, out2);
  return status;
}

/* ------------------------------------------------------------------------ */
/* bootstrapping: fix_small_values (Sect. 7.4)                               */
/* ------------------------------------------------------------------------ */

static int is_small(const orc_mesh* m, double gamma, const double* u) {
  double w[NV];
  orc_cons_to_prim(gamma, u, w);
  return small_prim(m, w);
}

static void cell_of(const orc_mesh* m, const double* U, int b, size_t c, double* u) {
  const size_t nvb = (size_t)m->nblocks * m->ncell;
  for (int v = 0; v < NV; v++) u[v] = U[(size_t)v * nvb + (size_t)b * m->ncell + c];
}

long orc_fix_small(const orc_mesh* m, double* U, int method) {
  const size_t nvb = (size_t)m->nblocks * m->ncell;
  const int* nx = m->cfg.nx;
  unsigned char* flag = (unsigned char*)calloc(nvb, 1);
  long nfix = 0;
  /* 1. find every small cell before changing any */
  for (int b = 0; b < m->nblocks; b++) {
    const double gamma = m->inst[m->blk[b].inst].gamma;
    for (int c = 0; c < m->ncell; c++) {
      double u[NV];
      cell_of(m, U, b, (size_t)c, u);
      flag[(size_t)b * m->ncell + c] = (unsigned char)is_small(m, gamma, u);
    }
  }
  /* 2. fix them; averages read only cells that are not small (never changed) */
  for (int b = 0; b < m->nblocks; b++) {
    const blockinfo* B = &m->blk[b];
    const double gamma = m->inst[B->inst].gamma;
    for (int c = 0; c < m->ncell; c++) {
      if (!flag[(size_t)b * m->ncell + c]) continue;
      nfix++;
      int ijk[3] = {c % nx[0], (c / nx[0]) % nx[1], c / (nx[0] * nx[1])};
      double u[NV], w[NV];
      cell_of(m, U, b, (size_t)c, u);
      double rho, vel[3], p;
      int n = 0;
      double sr = 0.0, sv[3] = {0.0, 0.0, 0.0}, sp = 0.0;
      if (method == 2) {
        for (int d = 0; d < m->cfg.ndim; d++)
          for (int side = 0; side < 2; side++) {
            int q[3] = {ijk[0], ijk[1], ijk[2]};
            q[d] += side ? 1 : -1;
            int nb = b;
            if (q[d] < 0 || q[d] >= nx[d]) {
              /* same-level face neighbour block (periodic wrap); none across
               * a physical boundary or a level change */
              long id[3] = {B->idx[0], B->idx[1], B->idx[2]};
              id[d] += side ? 1 : -1;
              long nbl = blocks_at_level(m, B->inst, B->level, d);
              if (id[d] < 0 || id[d] >= nbl) {
                if (m->cfg.bc[d][side] != 0) continue;
                id[d] = (id[d] % nbl + nbl) % nbl;
              }
              nb = hget(m, mkkey(B->inst, B->level, id[0], id[1], id[2]));
              if (nb < 0) continue;
              q[d] = side ? 0 : nx[d] - 1;
            }
            size_t cc = ((size_t)q[2] * nx[1] + q[1]) * nx[0] + q[0];
            if (flag[(size_t)nb * m->ncell + cc]) continue;
            double un[NV], wn[NV];
            cell_of(m, U, nb, cc, un);
            orc_cons_to_prim(gamma, un, wn);
            sr += wn[0];
            sv[0] += wn[1];
            sv[1] += wn[2];
            sv[2] += wn[3];
            sp += wn[4];
            n++;
          }
      }
      if (n > 0) {
        rho = sr / n;
        vel[0] = sv[0] / n, vel[1] = sv[1] / n, vel[2] = sv[2] / n;
        p = sp / n;
      } else {
        /* replace: floors, velocity kept where the density allows */
        orc_cons_to_prim(gamma, u, w);
        rho = u[0] > m->cfg.small_density ? u[0] : m->cfg.small_density;
        for (int e = 0; e < 3; e++) vel[e] = u[0] > 0.0 ? w[1 + e] : 0.0;
        p = (u[0] > 0.0 && w[4] > m->cfg.small_pressure) ? w[4] : m->cfg.small_pressure;
      }
      double wf[NV] = {rho, vel[0], vel[1], vel[2], p, u[5], u[6], u[7], u[8]};
      double uf[NV];
      orc_prim_to_cons(gamma, wf, uf);
      for (int v = 0; v < NV; v++) U[(size_t)v * nvb + (size_t)b * m->ncell + c] = uf[v];
    }
  }
  free(flag);
  return nfix;
}

/* ------------------------------------------------------------------------ */
/* CFL time step, sums, runs                                                 */
/* ------------------------------------------------------------------------ */

int orc_cfl(const orc_mesh* m, const double* U, const double* t, const double* t_end,
            double* dt, double* ch) {
  const size_t nvb = (size_t)m->nblocks * m->ncell;
  double* smax = (double*)calloc((size_t)m->ninst, sizeof(double));
  for (int q = 0; q < m->ninst; q++) ch[q] = 0.0;
  for (int b = 0; b < m->nblocks; b++) {
    const blockinfo* B = &m->blk[b];
    double dx[3];
    cell_dx(m, B->inst, B->level, dx);
    double g = m->inst[B->inst].gamma;
    for (int c = 0; c < m->ncell; c++) {
      double u[NV], w[NV];
      for (int v = 0; v < NV; v++) u[v] = U[(size_t)v * nvb + (size_t)b * m->ncell + c];
      orc_cons_to_prim(g, u, w);
      double s = 0.0;
      for (int d = 0; d < m->cfg.ndim; d++) {
        double sp = fabs(w[1 + d]) + orc_fast_speed(g, w, d);
        s += sp / dx[d];
        if (sp > ch[B->inst]) ch[B->inst] = sp;
      }
      if (s > smax[B->inst]) smax[B->inst] = s;
    }
  }
  for (int q = 0; q < m->ninst; q++) {
    double d = m->cfg.courant / smax[q];
    double left = t_end[q] - t[q];
    if (left <= 0.0) d = 0.0;
    else if (d >= left) d = left;
    dt[q] = d;
  }
  free(smax);
  return 0;
}

void orc_sums(const orc_mesh* m, const double* U, double* sums) {
  const size_t nvb = (size_t)m->nblocks * m->ncell;
  memset(sums, 0, sizeof(double) * NV * (size_t)m->ninst);
  for (int b = 0; b < m->nblocks; b++) {
    const blockinfo* B = &m->blk[b];
    double dx[3];
    cell_dx(m, B->inst, B->level, dx);
    double dv = dx[0];
    for (int d = 1; d < m->cfg.ndim; d++) dv *= dx[d];
    for (int v = 0; v < NV; v++) {
      double s = 0.0;
      for (int c = 0; c < m->ncell; c++) s += U[(size_t)v * nvb + (size_t)b * m->ncell + c];
      sums[B->inst * NV + v] += s * dv;
    }
  }
}

int orc_run(orc_mesh* m, double* U, double* t, const double* t_end, int maxsteps,
            double fixed_dt, int* nsteps_done) {
  const size_t n = (size_t)NV * m->nblocks * m->ncell;
  double* A = (double*)malloc(sizeof(double) * n);
  double* Bf = (double*)malloc(sizeof(double) * n);
  double* dt = (double*)malloc(sizeof(double) * (size_t)m->ninst);
  double* ch = (double*)malloc(sizeof(double) * (size_t)m->ninst);
  int status = ST_OK, s = 0;
  for (; s < maxsteps; s++) {
    orc_cfl(m, U, t, t_end, dt, ch);
    if (fixed_dt > 0.0)
      for (int q = 0; q < m->ninst; q++) {
        double left = t_end[q] - t[q];
        dt[q] = left <= 0.0 ? 0.0 : (fixed_dt >= left ? left : fixed_dt);
      }
    int any = 0;
    for (int q = 0; q < m->ninst; q++) any |= dt[q] > 0.0;
    if (!any) break;
    int st[5] = {0, 0, 0, 0, 0};
    /* with fix_small_values every stage's (first) output is bootstrapped */
    const int fx = m->cfg.fix_small_values;
#define ORC_FIX(arr) \
  do {               \
    if (fx) orc_fix_small(m, (arr), fx); \
  } while (0)
    if (m->cfg.time == 0) {
      st[0] = orc_stage(m, 0, dt, ch, U, U, A, NULL, 0);
      ORC_FIX(A);
      st[1] = orc_stage(m, 1, dt, ch, U, A, Bf, NULL, 0);
      ORC_FIX(Bf);
      memcpy(U, Bf, sizeof(double) * n);
    } else if (m->cfg.time == 1) {
      st[0] = orc_stage(m, 0, dt, ch, U, U, A, NULL, 0);
      ORC_FIX(A);
      st[1] = orc_stage(m, 1, dt, ch, U, A, Bf, NULL, 0);
      ORC_FIX(Bf);
      st[2] = orc_stage(m, 2, dt, ch, U, Bf, A, NULL, 0);
      ORC_FIX(A);
      memcpy(U, A, sizeof(double) * n);
    } else if (m->cfg.time == 2) {
      /* u1 -> A, u2 -> Bf, u3 -> A, u4 -> U */
      st[0] = orc_stage(m, 0, dt, ch, U, U, A, NULL, 0);
      ORC_FIX(A);
      st[1] = orc_stage(m, 1, dt, ch, U, A, Bf, NULL, 0);
      ORC_FIX(Bf);
      st[2] = orc_stage(m, 2, dt, ch, U, Bf, A, NULL, 0);
      ORC_FIX(A);
      st[3] = orc_stage(m, 3, dt, ch, U, A, U, NULL, 0);
      ORC_FIX(U);
    } else {
      /* u1 -> A, u2 -> Bf, u3 -> A; stage 3: u4 -> Bf (over u2, its own
       * cells) and w -> U (over u0); stage 4: u5 = w + ... -> U */
      st[0] = orc_stage(m, 0, dt, ch, U, U, A, NULL, 0);
      ORC_FIX(A);
      st[1] = orc_stage(m, 1, dt, ch, U, A, Bf, NULL, 0);
      ORC_FIX(Bf);
      st[2] = orc_stage(m, 2, dt, ch, U, Bf, A, NULL, 0);
      ORC_FIX(A);
      st[3] = orc_stage2(m, 3, dt, ch, U, A, Bf, Bf, U, NULL, 0);
      ORC_FIX(Bf);
      st[4] = orc_stage(m, 4, dt, ch, U, Bf, U, NULL, 0);
      ORC_FIX(U);
    }
#undef ORC_FIX
    for (int e = 0; e < 5; e++)
      if (st[e]) status = st[e];
    for (int q = 0; q < m->ninst; q++) {
      if (dt[q] > 0.0 && dt[q] >= t_end[q] - t[q]) t[q] = t_end[q];
      else t[q] += dt[q];
    }
    if (status) {
      s++;
      break;
    }
  }
  if (nsteps_done) *nsteps_done = s;
  free(A);
  free(Bf);
  free(dt);
  free(ch);
  return status;
}
