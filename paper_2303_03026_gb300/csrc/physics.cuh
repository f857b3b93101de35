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
//  - minmod / vanleer / koren face values (limiter table of Sect. 3.1.1);
//  - glm interface solve of the (B_n, psi) pair (Dedner et al. 2002);
//  - HLL (Harten 1983) and HLLD (Miyoshi & Kusano 2005) fluxes.
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

template <class T> __device__ __forceinline__ T sgnT(T x) {
  return (T)((x > T(0)) - (x < T(0)));
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
  float ke = 0.5f * (u[1] * vx + u[2] * vy + u[3] * vz);
  double bx = u[5], by = u[6], bz = u[7];
  double me = 0.5 * (bx * bx + by * by + bz * bz);
  return (float)((gamma - 1.0) * ((double)u[4] - (double)ke - me));
}

template <class T>
__device__ __forceinline__ void cons2prim(double gamma, const T* u, T* w) {
  T rho = u[0];
  T vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
  w[0] = rho;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = pressure_of(gamma, u, vx, vy, vz);
  w[5] = u[5];
  w[6] = u[6];
  w[7] = u[7];
  w[8] = u[8];
}

// fast speed along direction d of a primitive state (global frame)
template <class T>
__device__ __forceinline__ T fast_speed(T gamma, const T* w, int d) {
  int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
  T rho = w[0];
  T a2 = gamma * w[4] / rho;
  T bn = w[5 + d], b1 = w[5 + t1], b2 = w[5 + t2];
  T bt2 = (b1 * b1 + b2 * b2) / rho;
  T bb = (bn * bn + b1 * b1 + b2 * b2) / rho;
  T dd = a2 - bb;
  return sqrt(T(0.5) * (a2 + bb + sqrt(dd * dd + T(4) * a2 * bt2)));
}

// ---------------------------------------------------------------- limiters

template <class T> __device__ __forceinline__ T minmod2(T a, T b) {
  return (a * b > T(0)) ? sgnT(a) * fmin(fabs(a), fabs(b)) : T(0);
}

// face value at i+1/2 from the cell with values (a, b, c) = (w_{i-1}, w_i, w_{i+1})
template <class T> __device__ __forceinline__ T recon_plus(int lim, T a, T b, T c) {
  T dm = b - a, dp = c - b;
  if (!(dm * dp > T(0))) return b;
  if (lim == AMRVAC_LIM_MINMOD) return b + T(0.5) * minmod2(dm, dp);
  if (lim == AMRVAC_LIM_VANLEER) return b + T(0.5) * (T(2) * dm * dp / (dm + dp));
  T am = fabs(dm), ap = fabs(dp);
  T l3 = fmin(fmin(T(2) * am, (am + T(2) * ap) / T(3)), T(2) * ap);
  return b + T(0.5) * sgnT(dp) * l3;
}

// face value at i-1/2 from the cell with values (a, b, c)
template <class T> __device__ __forceinline__ T recon_minus(int lim, T a, T b, T c) {
  T dm = b - a, dp = c - b;
  if (!(dm * dp > T(0))) return b;
  if (lim == AMRVAC_LIM_MINMOD) return b - T(0.5) * minmod2(dm, dp);
  if (lim == AMRVAC_LIM_VANLEER) return b - T(0.5) * (T(2) * dm * dp / (dm + dp));
  T am = fabs(dm), ap = fabs(dp);
  T l3 = fmin(fmin(T(2) * ap, (ap + T(2) * am) / T(3)), T(2) * am);
  return b - T(0.5) * sgnT(dm) * l3;
}

// ---------------------------------------------------------------- Riemann
// local frame: q = (rho, u, v, w, p, -, By, Bz), normal field bx shared.

template <class T>
__device__ __forceinline__ void local_cons_flux(T g, const T* q, T bx, T* U, T* F, T& pt) {
  T rho = q[0], u = q[1], v = q[2], w = q[3], p = q[4], by = q[6], bz = q[7];
  T b2 = bx * bx + by * by + bz * bz;
  pt = p + T(0.5) * b2;
  T e = p / (g - T(1)) + T(0.5) * rho * (u * u + v * v + w * w) + T(0.5) * b2;
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
  T rho = q[0];
  T a2 = g * q[4] / rho;
  T bt2 = (q[6] * q[6] + q[7] * q[7]) / rho;
  T bb = (bx * bx + q[6] * q[6] + q[7] * q[7]) / rho;
  T dd = a2 - bb;
  return sqrt(T(0.5) * (a2 + bb + sqrt(dd * dd + T(4) * a2 * bt2)));
}

template <class T>
__device__ __forceinline__ void hll_local(T g, const T* ql, const T* qr, T bx, T* f) {
  T UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(g, ql, bx, UL, FL, ptl);
  local_cons_flux(g, qr, bx, UR, FR, ptr);
  T cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  T sl = fmin(ql[1] - cfl, qr[1] - cfr);
  T sr = fmax(ql[1] + cfl, qr[1] + cfr);
#pragma unroll
  for (int c = 0; c < 8; c++) {
    if (sl >= T(0)) f[c] = FL[c];
    else if (sr <= T(0)) f[c] = FR[c];
    else f[c] = (sr * FL[c] - sl * FR[c] + sl * sr * (UR[c] - UL[c])) / (sr - sl);
  }
}

template <class T> struct StarState {
  T rs, vs, ws, bys, bzs, es;
};

template <class T>
__device__ __forceinline__ StarState<T> hlld_star(const T* q, const T* U, T pt, T s, T sm, T pts,
                                                  T bx) {
  StarState<T> r;
  T rho = q[0], u = q[1], v = q[2], w = q[3], by = q[6], bz = q[7];
  T su = s - u;
  r.rs = rho * su / (s - sm);
  T big = rho * su * (s - sm);
  T den = big - bx * bx;
  T scale = fmax(fabs(big), bx * bx);
  if (fabs(den) <= Num<T>::hlld_eps * scale) {
    r.vs = v;
    r.ws = w;
    r.bys = by;
    r.bzs = bz;
  } else {
    T tv = bx * (sm - u) / den;
    T tb = (rho * su * su - bx * bx) / den;
    r.vs = v - by * tv;
    r.ws = w - bz * tv;
    r.bys = by * tb;
    r.bzs = bz * tb;
  }
  T vb = u * bx + v * by + w * bz;
  T vbs = sm * bx + r.vs * r.bys + r.ws * r.bzs;
  r.es = (su * U[4] - pt * u + pts * sm + bx * (vb - vbs)) / (s - sm);
  return r;
}

template <class T>
__device__ __forceinline__ void hlld_local(T g, const T* ql, const T* qr, T bx, T* f) {
  T UL[8], UR[8], FL[8], FR[8], ptl, ptr;
  local_cons_flux(g, ql, bx, UL, FL, ptl);
  local_cons_flux(g, qr, bx, UR, FR, ptr);
  T cfl = local_fast(g, ql, bx), cfr = local_fast(g, qr, bx);
  T ul = ql[1], ur = qr[1];
  T cmax = fmax(cfl, cfr);
  T sl = fmin(ul, ur) - cmax;
  T sr = fmax(ul, ur) + cmax;
  if (sl > T(0)) {
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = FL[c];
    return;
  }
  if (sr < T(0)) {
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = FR[c];
    return;
  }
  T rl = ql[0], rr = qr[0];
  T sul = sl - ul, sur = sr - ur;
  T den = sur * rr - sul * rl;
  T sm = (sur * rr * ur - sul * rl * ul - ptr + ptl) / den;
  T pts = (sur * rr * ptl - sul * rl * ptr + rl * rr * sur * sul * (ur - ul)) / den;
  StarState<T> L = hlld_star(ql, UL, ptl, sl, sm, pts, bx);
  StarState<T> R = hlld_star(qr, UR, ptr, sr, sm, pts, bx);
  T sqrl = sqrt(L.rs), sqrr = sqrt(R.rs);
  T ssl = sm - fabs(bx) / sqrl, ssr = sm + fabs(bx) / sqrr;
  T sb = sgnT(bx);
  T ssum = sqrl + sqrr;
  T vss = (sqrl * L.vs + sqrr * R.vs + (R.bys - L.bys) * sb) / ssum;
  T wss = (sqrl * L.ws + sqrr * R.ws + (R.bzs - L.bzs) * sb) / ssum;
  T byss = (sqrl * R.bys + sqrr * L.bys + sqrl * sqrr * (R.vs - L.vs) * sb) / ssum;
  T bzss = (sqrl * R.bzs + sqrr * L.bzs + sqrl * sqrr * (R.ws - L.ws) * sb) / ssum;
  T vbss = sm * bx + vss * byss + wss * bzss;
  T essl = L.es - sqrl * (sm * bx + L.vs * L.bys + L.ws * L.bzs - vbss) * sb;
  T essr = R.es + sqrr * (sm * bx + R.vs * R.bys + R.ws * R.bzs - vbss) * sb;
  // select the region of the fan that contains the interface (x/t = 0)
  if (ssl >= T(0)) {
    T US[8] = {L.rs, L.rs * sm, L.rs * L.vs, L.rs * L.ws, L.es, bx, L.bys, L.bzs};
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = FL[c] + sl * (US[c] - UL[c]);
  } else if (sm >= T(0)) {
    T US[8] = {L.rs, L.rs * sm, L.rs * L.vs, L.rs * L.ws, L.es, bx, L.bys, L.bzs};
    T USS[8] = {L.rs, L.rs * sm, L.rs * vss, L.rs * wss, essl, bx, byss, bzss};
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = (FL[c] + sl * (US[c] - UL[c])) + ssl * (USS[c] - US[c]);
  } else if (ssr >= T(0)) {
    T US[8] = {R.rs, R.rs * sm, R.rs * R.vs, R.rs * R.ws, R.es, bx, R.bys, R.bzs};
    T USS[8] = {R.rs, R.rs * sm, R.rs * vss, R.rs * wss, essr, bx, byss, bzss};
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = (FR[c] + sr * (US[c] - UR[c])) + ssr * (USS[c] - US[c]);
  } else {
    T US[8] = {R.rs, R.rs * sm, R.rs * R.vs, R.rs * R.ws, R.es, bx, R.bys, R.bzs};
#pragma unroll
    for (int c = 0; c < 8; c++) f[c] = FR[c] + sr * (US[c] - UR[c]);
  }
}

// Face flux along d from primitive face states wl, wr (global frame).
template <class T>
__device__ __forceinline__ void face_flux(int flux, int glm, T g, T ch, int d, const T* wl,
                                          const T* wr, T* f) {
  int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
  T bnl = wl[5 + d], bnr = wr[5 + d];
  T bns, psis;
  if (glm) {
    bns = T(0.5) * (bnl + bnr) - (wr[8] - wl[8]) / (T(2) * ch);
    psis = T(0.5) * (wl[8] + wr[8]) - T(0.5) * ch * (bnr - bnl);
  } else {
    bns = T(0.5) * (bnl + bnr);
    psis = T(0);
  }
  T ql[8] = {wl[0], wl[1 + d], wl[1 + t1], wl[1 + t2], wl[4], bns, wl[5 + t1], wl[5 + t2]};
  T qr[8] = {wr[0], wr[1 + d], wr[1 + t1], wr[1 + t2], wr[4], bns, wr[5 + t1], wr[5 + t2]};
  T fl[8];
  if (flux == AMRVAC_FLUX_HLL) hll_local(g, ql, qr, bns, fl);
  else hlld_local(g, ql, qr, bns, fl);
  f[0] = fl[0];
  f[1 + d] = fl[1];
  f[1 + t1] = fl[2];
  f[1 + t2] = fl[3];
  f[4] = fl[4];
  f[5 + d] = glm ? psis : T(0);
  f[5 + t1] = fl[6];
  f[5 + t2] = fl[7];
  f[8] = glm ? ch * ch * bns : T(0);
}

}  // namespace amrvac
