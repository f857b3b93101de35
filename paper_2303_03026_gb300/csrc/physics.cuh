// Pointwise ideal-MHD + glm physics for the stage kernels, templated on the
// bulk real type (double for AMRVAC_FP64, float for AMRVAC_FP32_BULK).
//
//  - primitive recovery p = (gamma-1)(e - m.v/2 - B^2/2); in the float form the
//    subtraction and the magnetic energy are evaluated in double (the stored
//    floats are exact in double, B_i^2 of a float is exact in double), which
//    removes the cancellation at low plasma beta; the kinetic part m.v/2 is
//    formed in float;
//  - fast magnetosonic speed in the cancellation-free form
//    c_f^2 = (a^2 + b^2 + sqrt((a^2 - b^2)^2 + 4 a^2 b_t^2)) / 2;
//  - face values of the limiter table of Sect. 3.1.1: minmod, vanleer, koren,
//    superbee, woodward, mcbeta, albada, cada3 and venk on three cells, mp5,
//    weno5, wenoz5 and wenozp5 on five;
//  - glm interface solve of the (B_n, psi) pair (Dedner et al. 2002);
//  - HLL (Harten 1983), HLLD (Miyoshi & Kusano 2005), TVDLF and HLLC (Li
//    2005) fluxes.
#pragma once

#include <math.h>

#include "common.cuh"

namespace amrvac {

template <class T> struct Num;
template <> struct Num<double> {
  static constexpr double hlld_eps = 1e-8;
};
template <> struct Num<float> {
  static constexpr float hlld_eps = 1e-5f;
};

// sign with sgn(0) = 0, by selects (no integer-to-float conversion)
template <class T> __device__ __forceinline__ T sgnT(T x) {
  return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
}

// ---------------------------------------------------------------- primitives

__device__ __forceinline__ double pressure_of(double gamma, const double* u, double vx,
                                              double vy, double vz) {
  double ke = 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz);
  double me = 0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  return (gamma - 1.0) * (u[4] - ke - me);
}

__device__ __forceinline__ float pressure_of(double gamma, const float* u, float vx, float vy,
                                             float vz) {
  // (gamma-1)(e - ke) - (gamma-1)/2 B^2 with e, B_i exact in double
  float ke = 0.5f * (u[1] * vx + u[2] * vy + u[3] * vz);
  double bx = u[5], by = u[6], bz = u[7];
  double b2 = fma(bz, bz, fma(by, by, bx * bx));
  double gm1 = gamma - 1.0;
  return (float)fma(-0.5 * gm1, b2, gm1 * ((double)u[4] - (double)ke));
}

// ---- float-float (double-single) helpers: a value is hi + lo with |lo| <= ulp(hi)/2
struct ff2 {
  float hi, lo;
};

// a + b = s + e exactly (Knuth TwoSum)
__device__ __forceinline__ ff2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Same pressure as pressure_of(double, float*, ...) with the subtraction in
// float-float: B_i^2 = hi + lo exactly by FMA, e - ke exactly by TwoSum, the
// remaining sums compensated; one final rounding to float.
__device__ __forceinline__ float pressure_ff(float gm1, const float* u, float vx, float vy,
                                             float vz) {
  float ke = 0.5f * (u[1] * vx + u[2] * vy + u[3] * vz);
  float bx = u[5], by = u[6], bz = u[7];
  float h = __fmul_rn(bx, bx);
  float l = __fmaf_rn(bx, bx, -h);
  float t = __fmul_rn(by, by);
  l = __fadd_rn(l, __fmaf_rn(by, by, -t));
  ff2 s = two_sum(h, t);
  l = __fadd_rn(l, s.lo);
  t = __fmul_rn(bz, bz);
  l = __fadd_rn(l, __fmaf_rn(bz, bz, -t));
  s = two_sum(s.hi, t);
  l = __fadd_rn(l, s.lo);                       // B^2 = s.hi + l
  ff2 a = two_sum(u[4], -ke);                   // e - ke exactly
  ff2 d = two_sum(a.hi, -0.5f * s.hi);          // 0.5 * s.hi is exact
  float rest = __fadd_rn(__fadd_rn(d.lo, a.lo), -0.5f * l);
  return gm1 * __fadd_rn(d.hi, rest);
}

// gm1f: (float)(gamma - 1), used by the float-float pressure
template <class T>
__device__ __forceinline__ void cons2prim(double gamma, const T* u, T* w, bool ff = false,
                                          float gm1f = 0.f) {
  T rho = u[0];
  T ir = T(1) / rho;
  T vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  w[0] = rho;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  if constexpr (sizeof(T) == 4) {
    if (ff) w[4] = pressure_ff(gm1f, (const float*)u, vx, vy, vz);
    else w[4] = pressure_of(gamma, u, vx, vy, vz);
  } else {
    w[4] = pressure_of(gamma, u, vx, vy, vz);
  }
  w[5] = u[5];
  w[6] = u[6];
  w[7] = u[7];
  w[8] = u[8];
}

// fast speed along direction d of a primitive state (global frame)
template <class T>
__device__ __forceinline__ T fast_speed(T gamma, const T* w, int d) {
  int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
  T ir = T(1) / w[0];
  T a2 = gamma * w[4] * ir;
  T bn = w[5 + d], b1 = w[5 + t1], b2 = w[5 + t2];
  T bt = b1 * b1 + b2 * b2;
  T bt2 = bt * ir;
  T bb = (bn * bn + bt) * ir;
  T dd = a2 - bb;
  return sqrt(T(0.5) * (a2 + bb + sqrt(dd * dd + T(4) * a2 * bt2)));
}

// small values (Sect. 7.4): density or pressure below its floor, or not
// positive at all (the floors default to 0)
template <class T> __device__ __forceinline__ bool is_small_prim(T rho, T p, T rho_floor,
                                                                  T p_floor) {
  return !(rho > T(0) && rho >= rho_floor) || !(p > T(0) && p >= p_floor);
}

// ---------------------------------------------------------------- limiters

template <class T> __device__ __forceinline__ T minmod2(T a, T b) {
  return (a * b > T(0)) ? sgnT(a) * fmin(fabs(a), fabs(b)) : T(0);
}

// slope phi(r) dp (r = dm/dp > 0) of the symmetric limiters superbee,
// woodward (monotonized central), mcbeta (beta = 1.4) and van Albada
template <class T> __device__ __forceinline__ T sym_slope(int lim, T dm, T dp) {
  const T am = fabs(dm), ap = fabs(dp);
  if (lim == AMRVAC_LIM_SUPERBEE) return sgnT(dp) * fmax(fmin(T(2) * am, ap), fmin(am, T(2) * ap));
  if (lim == AMRVAC_LIM_WOODWARD)
    return sgnT(dp) * fmin(fmin(T(2) * am, T(0.5) * (am + ap)), T(2) * ap);
  if (lim == AMRVAC_LIM_MCBETA)
    return sgnT(dp) * fmin(fmin(T(1.4) * am, T(0.5) * (am + ap)), T(1.4) * ap);
  return dm * dp * (dm + dp) / (dm * dm + dp * dp);
}

// cada3 (Cada & Torrilhon 2009, the compact third-order limiter function):
// half the limited slope phi(theta) dp / 2, theta = dm/dp, with
// phi = max(0, min(phi3, max(-theta/2, min(2 theta, phi3, 1.6)))) and
// phi3 = (2 + theta)/3, written without the division: s = sgn(dp), a = |dp|,
// t = s dm (= theta a), phi a = max(0, min(p3, max(-t/2, min(2t, p3, 1.6 a))))
// with p3 = (2a + t)/3; 0 where dp = 0 (the limit of phi dp)
template <class T> __device__ __forceinline__ T cada3_half(T dm, T dp) {
  const T s = sgnT(dp), a = fabs(dp), t = s * dm;
  const T p3 = (T(2) * a + t) / T(3);
  const T inner = fmin(fmin(T(2) * t, p3), T(1.6) * a);
  const T pa = fmax(T(0), fmin(p3, fmax(T(-0.5) * t, inner)));
  return T(0.5) * s * pa;
}

// venk (Venkatakrishnan 1995) in 1D: the central increment d = (c - a)/4 from
// the centre of the cell (a, b, c) to its right face (the left face gets -d),
// times phi = (D^2 + 2 D e)/(D^2 + 2 e^2 + D e) per face, e the face's
// increment and D the range of the stencil beyond b on e's side; the cell
// takes the smaller factor of its two faces (smoothing constant 0).  D and e
// are scaled by max(|D|, |e|) first: the denominator is then at least 1, so
// no square underflows into a 0/0 (D has e's sign or is 0)
template <class T> __device__ __forceinline__ T venk_phi(T D, T e) {
  const T m = fmax(fabs(D), fabs(e));
  const T x = D / m, y = e / m;
  return (x * x + T(2) * x * y) / (x * x + T(2) * y * y + x * y);
}

template <class T> __device__ __forceinline__ T venk_increment(T a, T b, T c) {
  const T d = T(0.25) * (c - a);
  if (d == T(0)) return T(0);
  const T up = fmax(fmax(a, b), c) - b, dn = fmin(fmin(a, b), c) - b;
  const T pr = venk_phi(d > T(0) ? up : dn, d);   // right face: +d
  const T pl = venk_phi(d > T(0) ? dn : up, -d);  // left face: -d
  return fmin(pr, pl) * d;
}

// face value at i+1/2 from the cell with values (a, b, c) = (w_{i-1}, w_i, w_{i+1})
template <class T> __device__ __forceinline__ T recon_plus(int lim, T a, T b, T c) {
  T dm = b - a, dp = c - b;
  if (lim == AMRVAC_LIM_VENK) return b + venk_increment(a, b, c);
  if (lim == AMRVAC_LIM_CADA3) return b + cada3_half(dm, dp);  // keeps a slope at extrema
  if (!(dm * dp > T(0))) return b;
  if (lim >= AMRVAC_LIM_SUPERBEE) return b + T(0.5) * sym_slope(lim, dm, dp);
  if (lim == AMRVAC_LIM_MINMOD) return b + T(0.5) * minmod2(dm, dp);
  if (lim == AMRVAC_LIM_VANLEER) return b + T(0.5) * (T(2) * dm * dp / (dm + dp));
  T am = fabs(dm), ap = fabs(dp);
  T l3 = fmin(fmin(T(2) * am, (am + T(2) * ap) / T(3)), T(2) * ap);
  return b + T(0.5) * sgnT(dp) * l3;
}

// face value at i-1/2 from the cell with values (a, b, c)
template <class T> __device__ __forceinline__ T recon_minus(int lim, T a, T b, T c) {
  T dm = b - a, dp = c - b;
  if (lim == AMRVAC_LIM_VENK) return b - venk_increment(a, b, c);
  if (lim == AMRVAC_LIM_CADA3) return b + cada3_half(-dp, -dm);  // the mirrored stencil
  if (!(dm * dp > T(0))) return b;
  if (lim >= AMRVAC_LIM_SUPERBEE) return b - T(0.5) * sym_slope(lim, dm, dp);
  if (lim == AMRVAC_LIM_MINMOD) return b - T(0.5) * minmod2(dm, dp);
  if (lim == AMRVAC_LIM_VANLEER) return b - T(0.5) * (T(2) * dm * dp / (dm + dp));
  T am = fabs(dm), ap = fabs(dp);
  T l3 = fmin(fmin(T(2) * ap, (ap + T(2) * am) / T(3)), T(2) * am);
  return b - T(0.5) * sgnT(dm) * l3;
}

// Five-point limiters of the limiter table (3 ghost cells), face value at
// i+1/2 from v = (v_{i-2}, ..., v_{i+2}); the value at i-1/2 is the same
// formula on the mirrored stencil.
//   mp5 (Suresh & Huynh 1997): fifth-order interface polynomial, kept when it
//     lies between v_i and v_i + minmod(v_{i+1} - v_i, 4 (v_i - v_{i-1})),
//     else clipped into [v_min, v_max] built from the upper limit, the median
//     and the large-curvature values (minmod4 of second differences).
//   weno5 (Jiang & Shu 1996): linear weights (1, 6, 3)/10, alpha_k = d_k /
//     (1e-6 + beta_k)^2.
//   wenoz5 (Borges et al. 2008): alpha_k = d_k (1 + tau5 / (beta_k + eps)),
//     tau5 = |beta_0 - beta_2|, eps = 1e-40 (double) / 1e-36 (float).
//   wenozp5 (WENO-Z+, Acker, Borges & Costa 2016): alpha_k = d_k (1 +
//     (tau5 / (beta_k + eps))^2 + lam (beta_k + eps) / (tau5 + eps)),
//     lam = dx^(2/3) of the level along the reconstruction.
template <class T> __device__ __forceinline__ T minmod4g(T w, T x, T y, T z) {
  if (w > T(0) && x > T(0) && y > T(0) && z > T(0)) return fmin(fmin(w, x), fmin(y, z));
  if (w < T(0) && x < T(0) && y < T(0) && z < T(0)) return fmax(fmax(w, x), fmax(y, z));
  return T(0);
}

template <class T> __device__ __forceinline__ T mp5_face(T vm2, T vm1, T v0, T vp1, T vp2) {
  const T a = T(4);
  const T vor = (T(2) * vm2 - T(13) * vm1 + T(47) * v0 + T(27) * vp1 - T(3) * vp2) / T(60);
  const T vmp = v0 + minmod2(vp1 - v0, a * (v0 - vm1));
  if ((vor - v0) * (vor - vmp) <= T(0)) return vor;
  const T djm1 = vm2 - T(2) * vm1 + v0, dj = vm1 - T(2) * v0 + vp1, djp1 = v0 - T(2) * vp1 + vp2;
  const T dp = minmod4g(T(4) * dj - djp1, T(4) * djp1 - dj, dj, djp1);
  const T dm = minmod4g(T(4) * dj - djm1, T(4) * djm1 - dj, dj, djm1);
  const T vul = v0 + a * (v0 - vm1);
  const T vmd = T(0.5) * (v0 + vp1) - T(0.5) * dp;
  const T vlc = v0 + T(0.5) * (v0 - vm1) + T(4) / T(3) * dm;
  const T vmin = fmax(fmin(fmin(v0, vp1), vmd), fmin(fmin(v0, vul), vlc));
  const T vmax = fmin(fmax(fmax(v0, vp1), vmd), fmax(fmax(v0, vul), vlc));
  return vor + minmod2(vmin - vor, vmax - vor);
}

// explicitly rounded operations (never contracted into an FMA)
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

// Jiang-Shu smoothness indicator 13/12 t^2 + 1/4 u^2, each operation rounded
// as written: the WENO-Z+ weights depend on tau5 = |beta_0 - beta_2|, a
// near-cancellation, so beta is evaluated without FMA contraction (the order
// of a plain left-to-right evaluation)
template <class T> __device__ __forceinline__ T beta_rn(T t, T u) {
  return add_rn(mul_rn(mul_rn(T(13) / T(12), t), t), mul_rn(mul_rn(T(0.25), u), u));
}

// kind: 0 weno5, 1 wenoz5, 2 wenozp5 (lam its lambda)
template <class T>
__device__ __forceinline__ T weno5_face(int kind, T vm2, T vm1, T v0, T vp1, T vp2, T lam) {
  const T c13 = T(13) / T(12);
  const T t0 = vm2 - T(2) * vm1 + v0, u0 = vm2 - T(4) * vm1 + T(3) * v0;
  const T t1 = vm1 - T(2) * v0 + vp1, u1 = vm1 - vp1;
  const T t2 = v0 - T(2) * vp1 + vp2, u2 = T(3) * v0 - T(4) * vp1 + vp2;
  T b0 = c13 * t0 * t0 + T(0.25) * u0 * u0;
  T b1 = c13 * t1 * t1 + T(0.25) * u1 * u1;
  T b2 = c13 * t2 * t2 + T(0.25) * u2 * u2;
  if (kind == 2) {
    // t and u as written (left to right), then beta without contraction
    const T tt0 = add_rn(sub_rn(vm2, mul_rn(T(2), vm1)), v0);
    const T uu0 = add_rn(sub_rn(vm2, mul_rn(T(4), vm1)), mul_rn(T(3), v0));
    const T tt1 = add_rn(sub_rn(vm1, mul_rn(T(2), v0)), vp1), uu1 = sub_rn(vm1, vp1);
    const T tt2 = add_rn(sub_rn(v0, mul_rn(T(2), vp1)), vp2);
    const T uu2 = add_rn(sub_rn(mul_rn(T(3), v0), mul_rn(T(4), vp1)), vp2);
    b0 = beta_rn(tt0, uu0);
    b1 = beta_rn(tt1, uu1);
    b2 = beta_rn(tt2, uu2);
  }
  const T q0 = (T(2) * vm2 - T(7) * vm1 + T(11) * v0) / T(6);
  const T q1 = (-vm1 + T(5) * v0 + T(2) * vp1) / T(6);
  const T q2 = (T(2) * v0 + T(5) * vp1 - vp2) / T(6);
  T a0, a1, a2;
  if (kind == 2) {
    const T eps = sizeof(T) == 8 ? T(1e-40) : T(1e-36), tau = fabs(b0 - b2);
    if constexpr (sizeof(T) == 8) {
      // the weights as written, each operation rounded (no contraction)
      const T te = add_rn(tau, eps);
      auto alpha = [&](T d, T b) {
        const T be = add_rn(b, eps), r = div_rn(tau, be);
        return mul_rn(d, add_rn(add_rn(T(1), mul_rn(r, r)), div_rn(mul_rn(lam, be), te)));
      };
      a0 = alpha(T(0.1), b0);
      a1 = alpha(T(0.6), b1);
      a2 = alpha(T(0.3), b2);
    } else {
      // float: the same weights in a form that cannot overflow.  The lambda
      // term is written L (beta_k + eps)/(beta_max + eps) with
      // L = lam (beta_max + eps)/(tau5 + eps); tau5/(beta_k + eps) is capped at
      // 1e18 and L at 1e36.  While no cap binds this is the definition; a cap
      // binds only where one group of candidates outweighs the rest by more
      // than 1e18 (their weights then keep their ratios) and the sum of the
      // weights stays below 3e36
      const T bm = fmax(fmax(b0, b1), b2) + eps;
      const T L = fmin(lam * bm / (tau + eps), T(1e36));
      const T x0 = fmin(tau / (b0 + eps), T(1e18)), x1 = fmin(tau / (b1 + eps), T(1e18));
      const T x2 = fmin(tau / (b2 + eps), T(1e18));
      a0 = T(0.1) * (T(1) + x0 * x0 + L * ((b0 + eps) / bm));
      a1 = T(0.6) * (T(1) + x1 * x1 + L * ((b1 + eps) / bm));
      a2 = T(0.3) * (T(1) + x2 * x2 + L * ((b2 + eps) / bm));
      const T inv = T(1) / (a0 + a1 + a2);
      return (a0 * inv) * q0 + (a1 * inv) * q1 + (a2 * inv) * q2;
    }
  } else if (kind == 1) {
    const T eps = sizeof(T) == 8 ? T(1e-40) : T(1e-36), tau = fabs(b0 - b2);
    if constexpr (sizeof(T) == 8) {
      a0 = T(0.1) * (T(1) + tau / (b0 + eps));
      a1 = T(0.6) * (T(1) + tau / (b1 + eps));
      a2 = T(0.3) * (T(1) + tau / (b2 + eps));
    } else {
      // float: tau5/(beta_k + eps) overflows once a beta_k is 0 and tau5 is
      // above ~340, so the weights are scaled by the common factor
      // (beta_min + eps)/(beta_min + eps + tau5): a_k = d_k (beta_min + eps +
      // r_k tau5)/(beta_min + eps + tau5) with r_k = (beta_min + eps)/(beta_k +
      // eps) <= 1, so 0 < a_k <= d_k and the normalised weights are unchanged
      const T bm = fmin(fmin(b0, b1), b2) + eps, den = bm + tau;
      a0 = T(0.1) * ((bm + (bm / (b0 + eps)) * tau) / den);
      a1 = T(0.6) * ((bm + (bm / (b1 + eps)) * tau) / den);
      a2 = T(0.3) * ((bm + (bm / (b2 + eps)) * tau) / den);
    }
  } else {
    const T eps = T(1e-6);
    a0 = T(0.1) / ((eps + b0) * (eps + b0));
    a1 = T(0.6) / ((eps + b1) * (eps + b1));
    a2 = T(0.3) / ((eps + b2) * (eps + b2));
  }
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

__device__ __forceinline__ int weno_kind(int lim) {
  return lim == AMRVAC_LIM_WENOZ5 ? 1 : (lim == AMRVAC_LIM_WENOZP5 ? 2 : 0);
}

// left state at i+1/2 of cell i, v = (v_{i-2}, ..., v_{i+2}); lam: the wenozp5
// lambda of the level and direction
template <class T> __device__ __forceinline__ T recon5_plus(int lim, const T* v, T lam) {
  return lim == AMRVAC_LIM_MP5 ? mp5_face(v[0], v[1], v[2], v[3], v[4])
                               : weno5_face(weno_kind(lim), v[0], v[1], v[2], v[3], v[4], lam);
}

// right state at i-1/2 of cell i, v = (v_{i-2}, ..., v_{i+2})
template <class T> __device__ __forceinline__ T recon5_minus(int lim, const T* v, T lam) {
  return lim == AMRVAC_LIM_MP5 ? mp5_face(v[4], v[3], v[2], v[1], v[0])
                               : weno5_face(weno_kind(lim), v[4], v[3], v[2], v[1], v[0], lam);
}

// ---------------------------------------------------------------- Riemann
// local frame: q = (rho, u, v, w, p, -, By, Bz), normal field bx shared.

// ig1 = 1/(gamma - 1)
template <class T>
__device__ __forceinline__ void local_cons_flux(T ig1, const T* q, T bx, T* U, T* F, T& pt) {
  T rho = q[0], u = q[1], v = q[2], w = q[3], p = q[4], by = q[6], bz = q[7];
  T b2 = bx * bx + by * by + bz * bz;
  pt = p + T(0.5) * b2;
  T e = p * ig1 + T(0.5) * rho * (u * u + v * v + w * w) + T(0.5) * b2;
  T vb = u * bx + v * by + w * bz;
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
  F[5] = T(0);
  F[6] = by * u - bx * v;
  F[7] = bz * u - bx * w;
}

template <class T> __device__ __forceinline__ T local_fast(T g, const T* q, T bx) {
  T ir = T(1) / q[0];
  T bt = q[6] * q[6] + q[7] * q[7];
  T a2 = g * q[4] * ir;
  T bt2 = bt * ir;
  T bb = (bx * bx + bt) * ir;
  T dd = a2 - bb;
  return sqrt(T(0.5) * (a2 + bb + sqrt(dd * dd + T(4) * a2 * bt2)));
}

template <class T>
__device__ __forceinline__ void hll_local(T g, T ig1, const T* ql, const T* qr, T bx, T* f) {
  T UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(ig1, ql, bx, UL, FL, ptl);
  local_cons_flux(ig1, qr, bx, UR, FR, ptr);
  T cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  T sl = fmin(ql[1] - cfl, qr[1] - cfr);
  T sr = fmax(ql[1] + cfl, qr[1] + cfr);
  T inv = T(1) / (sr - sl);
#pragma unroll
  for (int c = 0; c < 8; c++) {
    if (sl >= T(0)) f[c] = FL[c];
    else if (sr <= T(0)) f[c] = FR[c];
    else f[c] = (sr * FL[c] - sl * FR[c] + sl * sr * (UR[c] - UL[c])) * inv;
  }
}

// TVD Lax-Friedrichs: (F_L + F_R)/2 - c_max (U_R - U_L)/2 with the fastest
// signal speed of the two sides, c_max = max(|u_L| + c_fL, |u_R| + c_fR)
template <class T>
__device__ __forceinline__ void tvdlf_local(T g, T ig1, const T* ql, const T* qr, T bx, T* f) {
  T UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(ig1, ql, bx, UL, FL, ptl);
  local_cons_flux(ig1, qr, bx, UR, FR, ptr);
  T cmax = fmax(fabs(ql[1]) + local_fast(g, ql, bx), fabs(qr[1]) + local_fast(g, qr, bx));
#pragma unroll
  for (int c = 0; c < 8; c++) f[c] = T(0.5) * (FL[c] + FR[c]) - T(0.5) * cmax * (UR[c] - UL[c]);
}

// HLLC for MHD (Li 2005): HLL speeds; the HLL state gives the contact speed
// S_M, the star field B* (normal component bx) and star velocity v*; total
// pressure p_T* = rho_L (S_L - u_L)(S_M - u_L) + p_TL; the upwind side K of
// S_M: rho* = rho (S - u)/(S - S_M), m* = (rho* S_M, [rho v_t (S - u) -
// bx (B*_t - B_t)]/(S - S_M)), e* = [e (S - u) + p_T* S_M - p_T u -
// bx (v*.B* - v.B)]/(S - S_M); flux F_K + S_K (U*_K - U_K)
template <class T>
__device__ __forceinline__ void hllc_local(T g, T ig1, const T* ql, const T* qr, T bx, T* f) {
  T UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(ig1, ql, bx, UL, FL, ptl);
  local_cons_flux(ig1, qr, bx, UR, FR, ptr);
  const T cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  const T sl = fmin(ql[1] - cfl, qr[1] - cfr);
  const T sr = fmax(ql[1] + cfl, qr[1] + cfr);
  if (sl >= T(0)) {
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = FL[c];
    return;
  }
  if (sr <= T(0)) {
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = FR[c];
    return;
  }
  T uh[8];
#pragma unroll
  for (int c = 0; c < 8; c++) uh[c] = (sr * UR[c] - sl * UL[c] - FR[c] + FL[c]) / (sr - sl);
  const T sm = uh[1] / uh[0];
  const T vy = uh[2] / uh[0], vz = uh[3] / uh[0];
  const T by = uh[6], bz = uh[7];
  const T pts = ql[0] * (sl - ql[1]) * (sm - ql[1]) + ptl;
  const T vbs = sm * bx + vy * by + vz * bz;
  const bool left = sm >= T(0);
  const T* q = left ? ql : qr;
  const T* U = left ? UL : UR;
  const T* F = left ? FL : FR;
  const T S = left ? sl : sr, pt = left ? ptl : ptr;
  const T su = S - q[1], ssm = S - sm;
  const T vb = q[1] * bx + q[2] * q[6] + q[3] * q[7];
  T Us[8];
  Us[0] = q[0] * su / ssm;
  Us[1] = Us[0] * sm;
  Us[2] = (q[0] * q[2] * su - (bx * by - bx * q[6])) / ssm;
  Us[3] = (q[0] * q[3] * su - (bx * bz - bx * q[7])) / ssm;
  Us[4] = (U[4] * su + pts * sm - pt * q[1] - bx * (vbs - vb)) / ssm;
  Us[5] = bx;
  Us[6] = by;
  Us[7] = bz;
#pragma unroll
  for (int c = 0; c < 8; c++) f[c] = F[c] + S * (Us[c] - U[c]);
}

template <class T> struct StarState {
  T rs, vs, ws, bys, bzs, es;
};

template <class T>
__device__ __forceinline__ StarState<T> hlld_star(const T* q, T e, T pt, T s, T sm, T pts,
                                                  T bx) {
  StarState<T> r;
  T rho = q[0], u = q[1], v = q[2], w = q[3], by = q[6], bz = q[7];
  T su = s - u;
  T isd = T(1) / (s - sm);
  r.rs = rho * su * isd;
  T big = rho * su * (s - sm);
  T den = big - bx * bx;
  T scale = fmax(fabs(big), bx * bx);
  if (fabs(den) <= Num<T>::hlld_eps * scale) {
    r.vs = v;
    r.ws = w;
    r.bys = by;
    r.bzs = bz;
  } else {
    T iden = T(1) / den;
    T tv = bx * (sm - u) * iden;
    T tb = (rho * su * su - bx * bx) * iden;
    r.vs = v - by * tv;
    r.ws = w - bz * tv;
    r.bys = by * tb;
    r.bzs = bz * tb;
  }
  T vb = u * bx + v * by + w * bz;
  T vbs = sm * bx + r.vs * r.bys + r.ws * r.bzs;
  r.es = (su * e - pt * u + pts * sm + bx * (vb - vbs)) * isd;
  return r;
}

// physical flux and conserved state of a local state with total pressure pt
// and total energy e already formed
template <class T>
__device__ __forceinline__ void phys_flux_state(const T* q, T bx, T pt, T e, T* U, T* F) {
  T rho = q[0], u = q[1], v = q[2], w = q[3], by = q[6], bz = q[7];
  T mu = rho * u;
  U[0] = rho;
  U[1] = mu;
  U[2] = rho * v;
  U[3] = rho * w;
  U[4] = e;
  U[5] = bx;
  U[6] = by;
  U[7] = bz;
  F[0] = mu;
  F[1] = mu * u + pt - bx * bx;
  F[2] = mu * v - bx * by;
  F[3] = mu * w - bx * bz;
  F[4] = (e + pt) * u - bx * (u * bx + v * by + w * bz);
  F[5] = T(0);
  F[6] = by * u - bx * v;
  F[7] = bz * u - bx * w;
}

// HLLD (Miyoshi & Kusano 2005).  Both single-star states are formed (the
// double-star states average them); the upwind side of the interface is then
// chosen by selects, and the flux is F_s + c1 (U*_s - U_s) + c2 (U**_s - U*_s)
// with (c1, c2) = (0, 0), (S_s, 0) or (S_s, S*_s) for the outer, single-star
// and double-star regions: one physical flux instead of two and no divergent
// region branches.
template <class T>
__device__ __forceinline__ void hlld_local(T g, T ig1, const T* ql, const T* qr, T bx, T* f) {
  T ptl, ptr, el, er;
  {
    T b2 = bx * bx + ql[6] * ql[6] + ql[7] * ql[7];
    ptl = ql[4] + T(0.5) * b2;
    el = ql[4] * ig1 + T(0.5) * ql[0] * (ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]) +
         T(0.5) * b2;
    b2 = bx * bx + qr[6] * qr[6] + qr[7] * qr[7];
    ptr = qr[4] + T(0.5) * b2;
    er = qr[4] * ig1 + T(0.5) * qr[0] * (qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]) +
         T(0.5) * b2;
  }
  T cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  T ul = ql[1], ur = qr[1];
  T cmax = fmax(cfl, cfr);
  T sl = fmin(ul, ur) - cmax;
  T sr = fmax(ul, ur) + cmax;
  T rl = ql[0], rr = qr[0];
  T sul = sl - ul, sur = sr - ur;
  T iden = T(1) / (sur * rr - sul * rl);
  T sm = (sur * rr * ur - sul * rl * ul - ptr + ptl) * iden;
  T pts = (sur * rr * ptl - sul * rl * ptr + rl * rr * sur * sul * (ur - ul)) * iden;
  StarState<T> L = hlld_star(ql, el, ptl, sl, sm, pts, bx);
  StarState<T> R = hlld_star(qr, er, ptr, sr, sm, pts, bx);
  T sqrl = sqrt(L.rs), sqrr = sqrt(R.rs);
  T ssl = sm - fabs(bx) / sqrl, ssr = sm + fabs(bx) / sqrr;
  T sb = sgnT(bx);
  T issum = T(1) / (sqrl + sqrr);
  T vss = (sqrl * L.vs + sqrr * R.vs + (R.bys - L.bys) * sb) * issum;
  T wss = (sqrl * L.ws + sqrr * R.ws + (R.bzs - L.bzs) * sb) * issum;
  T byss = (sqrl * R.bys + sqrr * L.bys + sqrl * sqrr * (R.vs - L.vs) * sb) * issum;
  T bzss = (sqrl * R.bzs + sqrr * L.bzs + sqrl * sqrr * (R.ws - L.ws) * sb) * issum;
  T vbss = sm * bx + vss * byss + wss * bzss;
  T essl = L.es - sqrl * (sm * bx + L.vs * L.bys + L.ws * L.bzs - vbss) * sb;
  T essr = R.es + sqrr * (sm * bx + R.vs * R.bys + R.ws * R.bzs - vbss) * sb;
  // region of the fan that contains x/t = 0 (same tie rules as the oracle)
  const bool left = sm >= T(0);
  const bool outer = left ? (sl > T(0)) : (sr < T(0));
  const bool single = left ? (ssl >= T(0)) : !(ssr >= T(0));
  T q[8];
#pragma unroll
  for (int c = 0; c < 8; c++) q[c] = left ? ql[c] : qr[c];
  T U[8], F[8];
  phys_flux_state(q, bx, left ? ptl : ptr, left ? el : er, U, F);
  const T rs = left ? L.rs : R.rs, vs = left ? L.vs : R.vs, ws = left ? L.ws : R.ws;
  const T bys = left ? L.bys : R.bys, bzs = left ? L.bzs : R.bzs, es = left ? L.es : R.es;
  const T c1 = left ? sl : sr, c2 = left ? ssl : ssr;
  const T US[8] = {rs, rs * sm, rs * vs, rs * ws, es, bx, bys, bzs};
  const T USS[8] = {rs, rs * sm, rs * vss, rs * wss, left ? essl : essr, bx, byss, bzss};
#pragma unroll
  for (int c = 0; c < 8; c++) {
    T fs = F[c] + c1 * (US[c] - U[c]);
    T v = single ? fs : fs + c2 * (USS[c] - US[c]);
    f[c] = outer ? F[c] : v;
  }
}

// Face flux along D from primitive face states wl, wr (global frame).
template <class T, int D>
__device__ __forceinline__ void face_flux_d(int flux, int glm, T g, T ch, const T* wl,
                                            const T* wr, T* f) {
  constexpr int t1 = D == 2 ? 0 : D + 1, t2 = D == 0 ? 2 : D - 1;
  T bnl = wl[5 + D], bnr = wr[5 + D];
  T bns, psis;
  if (glm) {
    bns = T(0.5) * (bnl + bnr) - (wr[8] - wl[8]) / (T(2) * ch);
    psis = T(0.5) * (wl[8] + wr[8]) - T(0.5) * ch * (bnr - bnl);
  } else {
    bns = T(0.5) * (bnl + bnr);
    psis = T(0);
  }
  T ql[8] = {wl[0], wl[1 + D], wl[1 + t1], wl[1 + t2], wl[4], bns, wl[5 + t1], wl[5 + t2]};
  T qr[8] = {wr[0], wr[1 + D], wr[1 + t1], wr[1 + t2], wr[4], bns, wr[5 + t1], wr[5 + t2]};
  T fl[8];
  const T ig1 = T(1) / (g - T(1));
  if (flux == AMRVAC_FLUX_HLL) hll_local(g, ig1, ql, qr, bns, fl);
  else if (flux == AMRVAC_FLUX_HLLD) hlld_local(g, ig1, ql, qr, bns, fl);
  else if (flux == AMRVAC_FLUX_TVDLF) tvdlf_local(g, ig1, ql, qr, bns, fl);
  else hllc_local(g, ig1, ql, qr, bns, fl);
  f[0] = fl[0];
  f[1 + D] = fl[1];
  f[1 + t1] = fl[2];
  f[1 + t2] = fl[3];
  f[4] = fl[4];
  f[5 + D] = glm ? psis : T(0);
  f[5 + t1] = fl[6];
  f[5 + t2] = fl[7];
  f[8] = glm ? ch * ch * bns : T(0);
}

template <class T>
__device__ __forceinline__ void face_flux(int flux, int glm, T g, T ch, int d, const T* wl,
                                          const T* wr, T* f) {
  if (d == 0) face_flux_d<T, 0>(flux, glm, g, ch, wl, wr, f);
  else if (d == 1) face_flux_d<T, 1>(flux, glm, g, ch, wl, wr, f);
  else face_flux_d<T, 2>(flux, glm, g, ch, wl, wr, f);
}

}  // namespace amrvac
