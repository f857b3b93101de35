// FP32 face flux with the left and right states packed in float2 lanes.
//
// HLL and HLLD (Miyoshi & Kusano 2005) treat the two sides of a face with the
// same formulas: conserved state, total pressure, fast speed, single-star
// state.  Packing (left, right) into the two halves of a float2 and using the
// packed FP32x2 instructions of sm_100+ (__ffma2_rn, __fadd2_rn, __fmul2_rn)
// evaluates both sides with one instruction.  Formulas, region rules and
// degeneracy threshold are those of hll_local / hlld_local in physics.cuh;
// only the grouping of operations differs (FP32 rounding level).
#pragma once

#include "physics.cuh"

namespace amrvac {

__device__ __forceinline__ float2 sp2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one packed FMA with -1
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, sp2(-1.f), a); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(1.f / a.x, 1.f / a.y); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }

// fast speeds of both sides; bt = B_t^2, bx2 = B_n^2
__device__ __forceinline__ float2 fast2(float g, float2 rho, float2 p, float2 bt, float bx2) {
  float2 ir = rcp2(rho);
  float2 a2 = mul2(mul2(sp2(g), p), ir);
  float2 bt2 = mul2(bt, ir);
  float2 bb = mul2(add2(sp2(bx2), bt), ir);
  float2 dd = sub2(a2, bb);
  float2 sq = sqrt2(fma2(dd, dd, mul2(mul2(sp2(4.f), a2), bt2)));
  return sqrt2(mul2(sp2(0.5f), add2(add2(a2, bb), sq)));
}

// local frame pairs: rho, u, v, w, p, by, bz (x = left, y = right); bx shared
struct Side2 {
  float2 rho, u, v, w, p, by, bz;
};

// total pressure and total energy of both sides; bt = B_t^2 of both sides
__device__ __forceinline__ void pt_e2(const Side2& q, float bx2, float ig1, float2& pt,
                                      float2& e, float2& bt) {
  bt = fma2(q.bz, q.bz, mul2(q.by, q.by));
  float2 b2 = add2(bt, sp2(bx2));
  pt = fma2(b2, sp2(0.5f), q.p);
  float2 uu = fma2(q.w, q.w, fma2(q.v, q.v, mul2(q.u, q.u)));
  e = fma2(q.p, sp2(ig1), fma2(mul2(sp2(0.5f), q.rho), uu, mul2(sp2(0.5f), b2)));
}

// physical flux and conserved state of one side (scalar)
__device__ __forceinline__ void side_flux(float rho, float u, float v, float w, float by,
                                          float bz, float bx, float pt, float e, float* U,
                                          float* F) {
  float mu = rho * u;
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
  F[5] = 0.f;
  F[6] = by * u - bx * v;
  F[7] = bz * u - bx * w;
}

__device__ __forceinline__ void hll_pair(float g, float ig1, const Side2& q, float bx, float* f) {
  const float bx2 = bx * bx;
  float2 pt, e, bt;
  pt_e2(q, bx2, ig1, pt, e, bt);
  float2 cf = fast2(g, q.rho, q.p, bt, bx2);
  float sl = fminf(q.u.x - cf.x, q.u.y - cf.y);
  float sr = fmaxf(q.u.x + cf.x, q.u.y + cf.y);
  float UL[8], FL[8], UR[8], FR[8];
  side_flux(q.rho.x, q.u.x, q.v.x, q.w.x, q.by.x, q.bz.x, bx, pt.x, e.x, UL, FL);
  side_flux(q.rho.y, q.u.y, q.v.y, q.w.y, q.by.y, q.bz.y, bx, pt.y, e.y, UR, FR);
  const float inv = 1.f / (sr - sl);
  const float2 srsl = make_float2(sr, -sl);
  const float slsr = sl * sr;
#pragma unroll
  for (int c = 0; c < 8; c += 2) {
    // (sr FL - sl FR + sl sr (UR - UL)) / (sr - sl) for components c, c+1
    float2 fl = make_float2(FL[c], FL[c + 1]), fr = make_float2(FR[c], FR[c + 1]);
    float2 ul = make_float2(UL[c], UL[c + 1]), ur = make_float2(UR[c], UR[c + 1]);
    float2 t = fma2(sp2(srsl.x), fl, mul2(sp2(srsl.y), fr));
    t = mul2(fma2(sp2(slsr), sub2(ur, ul), t), sp2(inv));
    f[c] = sl >= 0.f ? FL[c] : (sr <= 0.f ? FR[c] : t.x);
    f[c + 1] = sl >= 0.f ? FL[c + 1] : (sr <= 0.f ? FR[c + 1] : t.y);
  }
}

// TVD Lax-Friedrichs with both sides' physical fluxes in packed lanes
__device__ __forceinline__ void tvdlf_pair(float g, float ig1, const Side2& q, float bx,
                                           float* f) {
  const float bx2 = bx * bx;
  float2 pt, e, bt;
  pt_e2(q, bx2, ig1, pt, e, bt);
  const float2 cf = fast2(g, q.rho, q.p, bt, bx2);
  const float cmax = fmaxf(fabsf(q.u.x) + cf.x, fabsf(q.u.y) + cf.y);
  float UL[8], FL[8], UR[8], FR[8];
  side_flux(q.rho.x, q.u.x, q.v.x, q.w.x, q.by.x, q.bz.x, bx, pt.x, e.x, UL, FL);
  side_flux(q.rho.y, q.u.y, q.v.y, q.w.y, q.by.y, q.bz.y, bx, pt.y, e.y, UR, FR);
#pragma unroll
  for (int c = 0; c < 8; c += 2) {
    const float2 fl = make_float2(FL[c], FL[c + 1]), fr = make_float2(FR[c], FR[c + 1]);
    const float2 ul = make_float2(UL[c], UL[c + 1]), ur = make_float2(UR[c], UR[c + 1]);
    const float2 t = fma2(sp2(-0.5f * cmax), sub2(ur, ul), mul2(sp2(0.5f), add2(fl, fr)));
    f[c] = t.x;
    f[c + 1] = t.y;
  }
}

__device__ __forceinline__ void hlld_pair(float g, float ig1, const Side2& q, float bx, float* f) {
  const float bx2 = bx * bx;
  float2 pt, e, bt;
  pt_e2(q, bx2, ig1, pt, e, bt);
  float2 cf = fast2(g, q.rho, q.p, bt, bx2);
  const float cmax = fmaxf(cf.x, cf.y);
  const float sl = fminf(q.u.x, q.u.y) - cmax;
  const float sr = fmaxf(q.u.x, q.u.y) + cmax;
  const float2 S = make_float2(sl, sr);
  const float2 su = sub2(S, q.u);              // (S_L - u_L, S_R - u_R)
  const float2 A = mul2(su, q.rho);            // rho (S - u)
  const float iden = 1.f / (A.y - A.x);
  const float2 Au = mul2(A, q.u);
  const float sm = (Au.y - Au.x - pt.y + pt.x) * iden;
  const float pts =
      (A.y * pt.x - A.x * pt.y + q.rho.x * q.rho.y * su.y * su.x * (q.u.y - q.u.x)) * iden;
  // single-star states of both sides
  const float2 ssm = sub2(S, sp2(sm));         // S - S_M
  const float2 isd = rcp2(ssm);
  const float2 rs = mul2(A, isd);
  const float2 big = mul2(A, ssm);
  const float2 den = sub2(big, sp2(bx2));
  const float2 iden2 = rcp2(den);
  const float2 tv = mul2(mul2(sp2(bx), sub2(sp2(sm), q.u)), iden2);
  const float2 tb = mul2(sub2(mul2(A, su), sp2(bx2)), iden2);
  const float2 ntv = mul2(tv, sp2(-1.f));
  float2 vs = fma2(q.by, ntv, q.v);
  float2 ws = fma2(q.bz, ntv, q.w);
  float2 bys = mul2(q.by, tb);
  float2 bzs = mul2(q.bz, tb);
  const float eps = Num<float>::hlld_eps;
  if (fabsf(den.x) <= eps * fmaxf(fabsf(big.x), bx2)) {
    vs.x = q.v.x;
    ws.x = q.w.x;
    bys.x = q.by.x;
    bzs.x = q.bz.x;
  }
  if (fabsf(den.y) <= eps * fmaxf(fabsf(big.y), bx2)) {
    vs.y = q.v.y;
    ws.y = q.w.y;
    bys.y = q.by.y;
    bzs.y = q.bz.y;
  }
  const float2 vb = fma2(q.w, q.bz, fma2(q.v, q.by, mul2(q.u, sp2(bx))));
  const float2 vbs = fma2(ws, bzs, fma2(vs, bys, sp2(sm * bx)));
  float2 t = sub2(mul2(su, e), mul2(pt, q.u));
  t = fma2(sp2(bx), sub2(vb, vbs), add2(t, sp2(pts * sm)));
  const float2 es = mul2(t, isd);
  // double-star states (averages of the two sides, packed over (v, w) / (By, Bz))
  const float2 isq = make_float2(rsqrtf(rs.x), rsqrtf(rs.y));  // 1/sqrt(rho*)
  const float2 sqr = mul2(rs, isq);
  const float abx = fabsf(bx);
  const float ssl = sm - abx * isq.x, ssr = sm + abx * isq.y;
  const float sb = sgnT(bx);
  const float issum = 1.f / (sqr.x + sqr.y);
  const float2 VL = make_float2(vs.x, ws.x), VR = make_float2(vs.y, ws.y);
  const float2 BL = make_float2(bys.x, bzs.x), BR = make_float2(bys.y, bzs.y);
  const float2 VSS = mul2(fma2(sub2(BR, BL), sp2(sb), fma2(sp2(sqr.y), VR, mul2(sp2(sqr.x), VL))),
                          sp2(issum));
  const float2 BSS = mul2(fma2(sub2(VR, VL), sp2(sqr.x * sqr.y * sb),
                               fma2(sp2(sqr.y), BL, mul2(sp2(sqr.x), BR))),
                          sp2(issum));
  const float vbss = sm * bx + VSS.x * BSS.x + VSS.y * BSS.y;
  // e** = e* -/+ sqrt(rho*) (v*.B* - v**.B**) sgn(Bx)
  const float2 ess = fma2(make_float2(-sqr.x * sb, sqr.y * sb), sub2(vbs, sp2(vbss)), es);
  // region containing x/t = 0 (same tie rules as the scalar solver)
  const bool left = sm >= 0.f;
  const bool outer = left ? (sl > 0.f) : (sr < 0.f);
  const bool single = left ? (ssl >= 0.f) : !(ssr >= 0.f);
  float U[8], F[8];
  side_flux(left ? q.rho.x : q.rho.y, left ? q.u.x : q.u.y, left ? q.v.x : q.v.y,
            left ? q.w.x : q.w.y, left ? q.by.x : q.by.y, left ? q.bz.x : q.bz.y, bx,
            left ? pt.x : pt.y, left ? e.x : e.y, U, F);
  const float r = left ? rs.x : rs.y;
  const float c1 = left ? sl : sr, c2 = left ? ssl : ssr;
  const float US[8] = {r, r * sm, r * (left ? vs.x : vs.y), r * (left ? ws.x : ws.y),
                       left ? es.x : es.y, bx, left ? bys.x : bys.y, left ? bzs.x : bzs.y};
  const float USS[8] = {r, r * sm, r * VSS.x, r * VSS.y, left ? ess.x : ess.y, bx, BSS.x, BSS.y};
#pragma unroll
  for (int c = 0; c < 8; c += 2) {
    const float2 Fp = make_float2(F[c], F[c + 1]);
    const float2 Up = make_float2(U[c], U[c + 1]);
    const float2 Sp = make_float2(US[c], US[c + 1]);
    const float2 SSp = make_float2(USS[c], USS[c + 1]);
    const float2 fs = fma2(sp2(c1), sub2(Sp, Up), Fp);
    const float2 fss = fma2(sp2(c2), sub2(SSp, Sp), fs);
    f[c] = outer ? F[c] : (single ? fs.x : fss.x);
    f[c + 1] = outer ? F[c + 1] : (single ? fs.y : fss.y);
  }
}

// vanleer face values of the face between cells b and c from the stencil
// (a, b, c, e): x = left state (from cell b), y = right state (from cell c)
__device__ __forceinline__ float2 vanleer_pair(float a, float b, float c, float e) {
  const float2 X = make_float2(b, c);
  const float2 dm = sub2(X, make_float2(a, b));
  const float2 dp = sub2(make_float2(c, e), X);
  const float2 prod = mul2(dm, dp);
  const float2 s = mul2(mul2(sp2(2.f), prod), rcp2(add2(dm, dp)));
  const float2 v = fma2(make_float2(0.5f, -0.5f), s, X);
  return make_float2(prod.x > 0.f ? v.x : b, prod.y > 0.f ? v.y : c);
}

// The symmetric limiters of the runtime-limiter instantiation, both face
// states of the face between cells b and c at once (x: left state from cell b
// with stencil (a, b, c); y: right state from cell c with (b, c, e)); slope =
// sgn(dp) G(|dm|, |dp|) where dm dp > 0, else first order.
//   monotonized central family: G = min(beta |dm|, (|dm| + |dp|)/2, beta |dp|)
//     (woodward beta = 2, mcbeta beta = 1.4)
//   superbee: G = max(min(2 |dm|, |dp|), min(|dm|, 2 |dp|))
//   albada:   slope = dm dp (dm + dp) / (dm^2 + dp^2)
template <int KIND>  // 0 monotonized central (beta), 1 superbee, 2 albada
__device__ __forceinline__ float2 sym_pair(float a, float b, float c, float e, float beta) {
  const float2 X = make_float2(b, c);
  const float2 dm = sub2(X, make_float2(a, b));
  const float2 dp = sub2(make_float2(c, e), X);
  const float2 prod = mul2(dm, dp);
  float2 s;
  if (KIND == 2) {
    const float2 den = fma2(dm, dm, mul2(dp, dp));
    s = mul2(mul2(prod, add2(dm, dp)), rcp2(den));
  } else {
    const float am0 = fabsf(dm.x), ap0 = fabsf(dp.x), am1 = fabsf(dm.y), ap1 = fabsf(dp.y);
    float g0, g1;
    if (KIND == 1) {
      g0 = fmaxf(fminf(2.f * am0, ap0), fminf(am0, 2.f * ap0));
      g1 = fmaxf(fminf(2.f * am1, ap1), fminf(am1, 2.f * ap1));
    } else {
      g0 = fminf(fminf(beta * am0, 0.5f * (am0 + ap0)), beta * ap0);
      g1 = fminf(fminf(beta * am1, 0.5f * (am1 + ap1)), beta * ap1);
    }
    s = make_float2(copysignf(g0, dp.x), copysignf(g1, dp.y));
  }
  const float2 v = fma2(make_float2(0.5f, -0.5f), s, X);
  return make_float2(prod.x > 0.f ? v.x : b, prod.y > 0.f ? v.y : c);
}

// cada3 (see cada3_half) for both face states of the face between cells b and
// c: x = left state from cell b with (dm, dp) = (b - a, c - b); y = right state
// from cell c, the mirrored rule with (dm, dp) = (c - e, b - c)
__device__ __forceinline__ float2 cada3_pair(float a, float b, float c, float e) {
  const float2 X = make_float2(b, c);
  const float2 dm = sub2(X, make_float2(a, e));
  const float2 dp = sub2(make_float2(c, b), X);
  const float s0 = sgnT(dp.x), s1 = sgnT(dp.y);
  const float2 A = make_float2(fabsf(dp.x), fabsf(dp.y));
  const float2 t = mul2(make_float2(s0, s1), dm);
  const float2 p3 = mul2(fma2(sp2(2.f), A, t), sp2(1.f / 3.f));
  const float2 tt = mul2(sp2(2.f), t), ca = mul2(sp2(1.6f), A), ht = mul2(sp2(-0.5f), t);
  const float i0 = fminf(fminf(tt.x, p3.x), ca.x), i1 = fminf(fminf(tt.y, p3.y), ca.y);
  const float pa0 = fmaxf(0.f, fminf(p3.x, fmaxf(ht.x, i0)));
  const float pa1 = fmaxf(0.f, fminf(p3.y, fmaxf(ht.y, i1)));
  return fma2(mul2(sp2(0.5f), make_float2(s0, s1)), make_float2(pa0, pa1), X);
}

// ---------------------------------------------------------------------------
// Two faces per thread, one per float2 lane: lane x the x face of a cell and
// lane y its y face.  Each lane loads the stencil of its own face already in
// the face's local frame (normal velocity and field first), so the packed
// operands need no register shuffling, and the per-face work of HLLD (wave
// speeds, double-star states, fan region) runs once for both faces.  The
// formulas are those of hlld_pair / hlld_local (MK05 with the degeneracy
// threshold, sgn(0) = 0 and the same region ties); only the packing differs.

__device__ __forceinline__ float2 min2(float2 a, float2 b) {
  return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
}
__device__ __forceinline__ float2 max2(float2 a, float2 b) {
  return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 sel2(bool px, bool py, float2 a, float2 b) {
  return make_float2(px ? a.x : b.x, py ? a.y : b.y);
}

// primitive face states of both faces in their local frames
struct Prim2 {
  float2 rho, u, v, w, p, by, bz;
};

// van Leer slopes of two cells at once from their one-sided differences:
// 2 dm dp / (dm + dp) where dm dp > 0, else 0
__device__ __forceinline__ float2 vl_slope2(float2 dm, float2 dp) {
  const float2 prod = mul2(dm, dp);
  const float2 s = mul2(mul2(sp2(2.f), prod), rcp2(add2(dm, dp)));
  return make_float2(prod.x > 0.f ? s.x : 0.f, prod.y > 0.f ? s.y : 0.f);
}

// fast speeds (cancellation-free form) from rho, p, B_t^2 and B_n^2
__device__ __forceinline__ float2 fast_xy(float g, float2 rho, float2 p, float2 bt, float2 bx2) {
  const float2 ir = rcp2(rho);
  const float2 a2 = mul2(mul2(sp2(g), p), ir);
  const float2 bt2 = mul2(bt, ir);
  const float2 bb = mul2(add2(bx2, bt), ir);
  const float2 dd = sub2(a2, bb);
  const float2 sq = sqrt2(fma2(dd, dd, mul2(mul2(sp2(4.f), a2), bt2)));
  return sqrt2(mul2(sp2(0.5f), add2(add2(a2, bb), sq)));
}

// single-star state of one side (MK05 eqs. 43-48) for both faces
struct Star2 {
  float2 rs, vs, ws, bys, bzs, es, vbs;
};

__device__ __forceinline__ Star2 hlld_star_xy(const Prim2& q, float2 S, float2 su, float2 A,
                                              float2 pt, float2 e, float2 sm, float2 pts,
                                              float2 bx, float2 bx2) {
  Star2 r;
  const float2 ssm = sub2(S, sm);
  const float2 isd = rcp2(ssm);
  r.rs = mul2(A, isd);
  const float2 big = mul2(A, ssm);
  const float2 den = sub2(big, bx2);
  const float2 iden = rcp2(den);
  const float2 tv = mul2(mul2(bx, sub2(sm, q.u)), iden);
  const float2 tb = mul2(sub2(mul2(A, su), bx2), iden);
  const float2 ntv = mul2(tv, sp2(-1.f));
  const float eps = Num<float>::hlld_eps;
  const bool dgx = fabsf(den.x) <= eps * fmaxf(fabsf(big.x), bx2.x);
  const bool dgy = fabsf(den.y) <= eps * fmaxf(fabsf(big.y), bx2.y);
  r.vs = sel2(dgx, dgy, q.v, fma2(q.by, ntv, q.v));
  r.ws = sel2(dgx, dgy, q.w, fma2(q.bz, ntv, q.w));
  r.bys = sel2(dgx, dgy, q.by, mul2(q.by, tb));
  r.bzs = sel2(dgx, dgy, q.bz, mul2(q.bz, tb));
  const float2 vb = fma2(q.w, q.bz, fma2(q.v, q.by, mul2(q.u, bx)));
  r.vbs = fma2(r.ws, r.bzs, fma2(r.vs, r.bys, mul2(sm, bx)));
  float2 t = sub2(mul2(su, e), mul2(pt, q.u));
  t = fma2(bx, sub2(vb, r.vbs), fma2(pts, sm, t));
  r.es = mul2(t, isd);
  return r;
}

// HLLD flux of two faces; f[c] for the local components c = 0..7 (c = 5, the
// normal field, is left to the glm solve)
__device__ __forceinline__ void hlld_xy(float g, float ig1, const Prim2& L, const Prim2& R,
                                        float2 bx, float2* f) {
  const float2 bx2 = mul2(bx, bx);
  const float2 btL = fma2(L.bz, L.bz, mul2(L.by, L.by));
  const float2 btR = fma2(R.bz, R.bz, mul2(R.by, R.by));
  const float2 b2L = add2(btL, bx2), b2R = add2(btR, bx2);
  const float2 ptL = fma2(b2L, sp2(0.5f), L.p), ptR = fma2(b2R, sp2(0.5f), R.p);
  const float2 uuL = fma2(L.w, L.w, fma2(L.v, L.v, mul2(L.u, L.u)));
  const float2 uuR = fma2(R.w, R.w, fma2(R.v, R.v, mul2(R.u, R.u)));
  const float2 eL = fma2(L.p, sp2(ig1), fma2(mul2(sp2(0.5f), L.rho), uuL, mul2(sp2(0.5f), b2L)));
  const float2 eR = fma2(R.p, sp2(ig1), fma2(mul2(sp2(0.5f), R.rho), uuR, mul2(sp2(0.5f), b2R)));
  const float2 cmax = max2(fast_xy(g, L.rho, L.p, btL, bx2), fast_xy(g, R.rho, R.p, btR, bx2));
  const float2 sl = sub2(min2(L.u, R.u), cmax), sr = add2(max2(L.u, R.u), cmax);
  const float2 suL = sub2(sl, L.u), suR = sub2(sr, R.u);
  const float2 AL = mul2(suL, L.rho), AR = mul2(suR, R.rho);
  const float2 iden = rcp2(sub2(AR, AL));
  // S_M and p_T* from the HLL-averaged normal momentum (MK05 eqs. 38, 41)
  const float2 sm = mul2(sub2(fma2(AR, R.u, ptL), fma2(AL, L.u, ptR)), iden);
  const float2 pts = mul2(fma2(mul2(mul2(L.rho, R.rho), mul2(suR, suL)), sub2(R.u, L.u),
                               sub2(mul2(AR, ptL), mul2(AL, ptR))),
                          iden);
  const Star2 SL = hlld_star_xy(L, sl, suL, AL, ptL, eL, sm, pts, bx, bx2);
  const Star2 SR = hlld_star_xy(R, sr, suR, AR, ptR, eR, sm, pts, bx, bx2);
  // double-star states (MK05 eqs. 59-63)
  const float2 isqL = make_float2(rsqrtf(SL.rs.x), rsqrtf(SL.rs.y));
  const float2 isqR = make_float2(rsqrtf(SR.rs.x), rsqrtf(SR.rs.y));
  const float2 sqrL = mul2(SL.rs, isqL), sqrR = mul2(SR.rs, isqR);
  const float2 abx = abs2(bx);
  const float2 ssl = sub2(sm, mul2(abx, isqL)), ssr = fma2(abx, isqR, sm);
  const float2 sb = make_float2(sgnT(bx.x), sgnT(bx.y));
  const float2 issum = rcp2(add2(sqrL, sqrR));
  const float2 vss = mul2(fma2(sub2(SR.bys, SL.bys), sb, fma2(sqrR, SR.vs, mul2(sqrL, SL.vs))), issum);
  const float2 wss = mul2(fma2(sub2(SR.bzs, SL.bzs), sb, fma2(sqrR, SR.ws, mul2(sqrL, SL.ws))), issum);
  const float2 sqq = mul2(mul2(sqrL, sqrR), sb);
  const float2 byss = mul2(fma2(sub2(SR.vs, SL.vs), sqq, fma2(sqrL, SR.bys, mul2(sqrR, SL.bys))), issum);
  const float2 bzss = mul2(fma2(sub2(SR.ws, SL.ws), sqq, fma2(sqrL, SR.bzs, mul2(sqrR, SL.bzs))), issum);
  const float2 vbss = fma2(wss, bzss, fma2(vss, byss, mul2(sm, bx)));
  // e** = e* -/+ sqrt(rho*) (v*.B* - v**.B**) sgn(Bx)
  const float2 essL = fma2(mul2(sqrL, sb), sub2(vbss, SL.vbs), SL.es);
  const float2 essR = fma2(mul2(sqrR, sb), sub2(SR.vbs, vbss), SR.es);
  // fan region containing x/t = 0, per face (ties as in the scalar solver)
  const bool lx = sm.x >= 0.f, ly = sm.y >= 0.f;
  const bool ox = lx ? (sl.x > 0.f) : (sr.x < 0.f), oy = ly ? (sl.y > 0.f) : (sr.y < 0.f);
  const bool sx = lx ? (ssl.x >= 0.f) : !(ssr.x >= 0.f);
  const bool sy = ly ? (ssl.y >= 0.f) : !(ssr.y >= 0.f);
  // the upwind side of S_M
  const float2 rho = sel2(lx, ly, L.rho, R.rho), u = sel2(lx, ly, L.u, R.u);
  const float2 v = sel2(lx, ly, L.v, R.v), w = sel2(lx, ly, L.w, R.w);
  const float2 by = sel2(lx, ly, L.by, R.by), bz = sel2(lx, ly, L.bz, R.bz);
  const float2 pt = sel2(lx, ly, ptL, ptR), e = sel2(lx, ly, eL, eR);
  const float2 rs = sel2(lx, ly, SL.rs, SR.rs), vs = sel2(lx, ly, SL.vs, SR.vs);
  const float2 ws = sel2(lx, ly, SL.ws, SR.ws), bys = sel2(lx, ly, SL.bys, SR.bys);
  const float2 bzs = sel2(lx, ly, SL.bzs, SR.bzs), es = sel2(lx, ly, SL.es, SR.es);
  const float2 ess = sel2(lx, ly, essL, essR);
  const float2 c1 = sel2(lx, ly, sl, sr), c2 = sel2(lx, ly, ssl, ssr);
  const float2 mu = mul2(rho, u);
  const float2 vb = fma2(w, bz, fma2(v, by, mul2(u, bx)));
  // physical flux F, state U, star U* and double-star U** of that side
  const float2 F[8] = {mu, fma2(mu, u, sub2(pt, bx2)), fma2(mu, v, mul2(mul2(bx, by), sp2(-1.f))),
                       fma2(mu, w, mul2(mul2(bx, bz), sp2(-1.f))),
                       sub2(mul2(add2(e, pt), u), mul2(bx, vb)), sp2(0.f),
                       sub2(mul2(by, u), mul2(bx, v)), sub2(mul2(bz, u), mul2(bx, w))};
  const float2 U[8] = {rho, mu, mul2(rho, v), mul2(rho, w), e, bx, by, bz};
  const float2 US[8] = {rs, mul2(rs, sm), mul2(rs, vs), mul2(rs, ws), es, bx, bys, bzs};
  const float2 USS[8] = {rs, mul2(rs, sm), mul2(rs, vss), mul2(rs, wss), ess, bx, byss, bzss};
#pragma unroll
  for (int c = 0; c < 8; c++) {
    if (c == 5) {
      f[c] = sp2(0.f);
      continue;
    }
    const float2 fs = fma2(c1, sub2(US[c], U[c]), F[c]);
    // the double-star and star states differ in the tangential and energy parts only
    const float2 fss = (c == 0 || c == 1) ? fs : fma2(c2, sub2(USS[c], US[c]), fs);
    f[c] = make_float2(ox ? F[c].x : (sx ? fs.x : fss.x), oy ? F[c].y : (sy ? fs.y : fss.y));
  }
}

// local component c of the y face -> primitive variable (normal y, tangential
// (z, x)); the x face uses the identity
__device__ __forceinline__ constexpr int yface_var(int c) {
  return c == 1 ? 2 : c == 2 ? 3 : c == 3 ? 1 : c == 5 ? 6 : c == 6 ? 7 : c == 7 ? 5 : c;
}

// x and y face fluxes of one cell with vanleer + HLLD: ax(v, t), ay(v, t) the
// 4-cell stencils (cells f-2 .. f+1) of the x and y faces; positivity fallback
// and glm as in stencil_flux_f2, per face
template <class AX, class AY>
__device__ __forceinline__ void stencil_flux_xy(AX ax, AY ay, int glm, float g, float ch,
                                                float* fx, float* fy) {
  float2 wl[NV], wr[NV];
#pragma unroll
  for (int c = 0; c < NV; c++) {
    const int vy = yface_var(c);
    const float2 A = make_float2(ax(c, 0), ay(vy, 0)), B = make_float2(ax(c, 1), ay(vy, 1));
    const float2 C = make_float2(ax(c, 2), ay(vy, 2)), E = make_float2(ax(c, 3), ay(vy, 3));
    const float2 d2 = sub2(C, B);
    wl[c] = fma2(sp2(0.5f), vl_slope2(sub2(B, A), d2), B);
    wr[c] = fma2(sp2(-0.5f), vl_slope2(d2, sub2(E, C)), C);
  }
  const bool bx_ = !(wl[0].x > 0.f) || !(wl[4].x > 0.f) || !(wr[0].x > 0.f) || !(wr[4].x > 0.f);
  const bool by_ = !(wl[0].y > 0.f) || !(wl[4].y > 0.f) || !(wr[0].y > 0.f) || !(wr[4].y > 0.f);
  if (bx_ || by_) {
#pragma unroll
    for (int c = 0; c < NV; c++) {
      if (bx_) {
        wl[c].x = ax(c, 1);
        wr[c].x = ax(c, 2);
      }
      if (by_) {
        wl[c].y = ay(yface_var(c), 1);
        wr[c].y = ay(yface_var(c), 2);
      }
    }
  }
  const float2 bnl = wl[5], bnr = wr[5];
  float2 bns, psis;
  if (glm) {
    const float ih = 0.5f / ch;
    bns = sub2(mul2(sp2(0.5f), add2(bnl, bnr)), mul2(sp2(ih), sub2(wr[8], wl[8])));
    psis = sub2(mul2(sp2(0.5f), add2(wl[8], wr[8])), mul2(sp2(0.5f * ch), sub2(bnr, bnl)));
  } else {
    bns = mul2(sp2(0.5f), add2(bnl, bnr));
    psis = sp2(0.f);
  }
  float2 fl[8];
  const Prim2 L = {wl[0], wl[1], wl[2], wl[3], wl[4], wl[6], wl[7]};
  const Prim2 R = {wr[0], wr[1], wr[2], wr[3], wr[4], wr[6], wr[7]};
  hlld_xy(g, 1.f / (g - 1.f), L, R, bns, fl);
  const float2 fpsi = glm ? mul2(sp2(ch * ch), bns) : sp2(0.f);
  fl[5] = psis;
#pragma unroll
  for (int c = 0; c < 8; c++) {
    fx[c] = fl[c].x;
    fy[yface_var(c)] = fl[c].y;
  }
  fx[8] = fpsi.x;
  fy[8] = fpsi.y;
}

template <int D, int FLUX>
__device__ __forceinline__ void face_flux_f2(float2* w, int glm, float g, float ch, float* f);

// Face flux along D from the 4-cell stencils of the 9 primitive variables:
// st(v, t) for cells f-2, f-1, f, f+1.  Positivity fallback and glm as in
// face_flux_d.
// LIM < 0: the limiter is the runtime value lim.
template <int D, int LIM, int FLUX, class Acc>
__device__ __forceinline__ void stencil_flux_f2(Acc st, int glm, float g, float ch, float* f,
                                                int lim) {
  float2 w[NV];
  if constexpr (LIM >= 0) {
#pragma unroll
    for (int v = 0; v < NV; v++) {
      float a = st(v, 0), b = st(v, 1), c = st(v, 2), e = st(v, 3);
      if (LIM == AMRVAC_LIM_VANLEER) w[v] = vanleer_pair(a, b, c, e);
      else w[v] = make_float2(recon_plus<float>(LIM, a, b, c), recon_minus<float>(LIM, b, c, e));
    }
  } else {
    // runtime limiter: one switch per face, the variable loop inside (not
    // unrolled: four limiters inlined at three faces would otherwise crowd the
    // instruction cache)
    if (lim == AMRVAC_LIM_SUPERBEE) {
#pragma unroll 1
      for (int v = 0; v < NV; v++) w[v] = sym_pair<1>(st(v, 0), st(v, 1), st(v, 2), st(v, 3), 0.f);
    } else if (lim == AMRVAC_LIM_ALBADA) {
#pragma unroll 1
      for (int v = 0; v < NV; v++) w[v] = sym_pair<2>(st(v, 0), st(v, 1), st(v, 2), st(v, 3), 0.f);
    } else if (lim == AMRVAC_LIM_CADA3) {
#pragma unroll 1
      for (int v = 0; v < NV; v++) w[v] = cada3_pair(st(v, 0), st(v, 1), st(v, 2), st(v, 3));
    } else if (lim == AMRVAC_LIM_VENK) {
#pragma unroll 1
      for (int v = 0; v < NV; v++) {
        const float a = st(v, 0), b = st(v, 1), c = st(v, 2), e = st(v, 3);
        w[v] = make_float2(b + venk_increment(a, b, c), c - venk_increment(b, c, e));
      }
    } else {
      const float beta = lim == AMRVAC_LIM_WOODWARD ? 2.f : 1.4f;
#pragma unroll 1
      for (int v = 0; v < NV; v++)
        w[v] = sym_pair<0>(st(v, 0), st(v, 1), st(v, 2), st(v, 3), beta);
    }
  }
  if (!(w[0].x > 0.f) || !(w[4].x > 0.f) || !(w[0].y > 0.f) || !(w[4].y > 0.f)) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = make_float2(st(v, 1), st(v, 2));
  }
  face_flux_f2<D, FLUX>(w, glm, g, ch, f);
}

// Five-point limiters (mp5, weno5, wenoz5, wenozp5; lim at run time, lam the
// wenozp5 lambda): st(v, t) for the six cells f-3 .. f+2 around the face
// f-1/2; each face state reconstructed in float as on the plain path
template <int D, int FLUX, class Acc>
__device__ __forceinline__ void stencil_flux5_f2(Acc st, int lim, float lam, int glm, float g,
                                                 float ch, float* f) {
  float2 w[NV];
  // one copy of the reconstruction for the nine variables (not unrolled): the
  // limiters' code, four of them behind the runtime switch and inlined at the
  // three faces, otherwise overflows the instruction cache
#pragma unroll 1
  for (int v = 0; v < NV; v++) {
    const float c[6] = {st(v, 0), st(v, 1), st(v, 2), st(v, 3), st(v, 4), st(v, 5)};
    w[v] = make_float2(recon5_plus<float>(lim, c, lam), recon5_minus<float>(lim, c + 1, lam));
  }
  if (!(w[0].x > 0.f) || !(w[4].x > 0.f) || !(w[0].y > 0.f) || !(w[4].y > 0.f)) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = make_float2(st(v, 2), st(v, 3));
  }
  face_flux_f2<D, FLUX>(w, glm, g, ch, f);
}

// glm solve and Riemann flux along D from the face states w[v] = (left, right)
template <int D, int FLUX>
__device__ __forceinline__ void face_flux_f2(float2* w, int glm, float g, float ch, float* f) {
  constexpr int t1 = D == 2 ? 0 : D + 1, t2 = D == 0 ? 2 : D - 1;
  const float bnl = w[5 + D].x, bnr = w[5 + D].y;
  float bns, psis;
  if (glm) {
    bns = 0.5f * (bnl + bnr) - (w[8].y - w[8].x) / (2.f * ch);
    psis = 0.5f * (w[8].x + w[8].y) - 0.5f * ch * (bnr - bnl);
  } else {
    bns = 0.5f * (bnl + bnr);
    psis = 0.f;
  }
  Side2 q;
  q.rho = w[0];
  q.u = w[1 + D];
  q.v = w[1 + t1];
  q.w = w[1 + t2];
  q.p = w[4];
  q.by = w[5 + t1];
  q.bz = w[5 + t2];
  float fl[8];
  const float ig1 = 1.f / (g - 1.f);
  if (FLUX == AMRVAC_FLUX_HLL) hll_pair(g, ig1, q, bns, fl);
  else if (FLUX == AMRVAC_FLUX_HLLD) hlld_pair(g, ig1, q, bns, fl);
  else if (FLUX == AMRVAC_FLUX_TVDLF) tvdlf_pair(g, ig1, q, bns, fl);
  else {
    // HLLC: the scalar three-wave solver on the unpacked face states
    const float ql[8] = {q.rho.x, q.u.x, q.v.x, q.w.x, q.p.x, bns, q.by.x, q.bz.x};
    const float qr[8] = {q.rho.y, q.u.y, q.v.y, q.w.y, q.p.y, bns, q.by.y, q.bz.y};
    hllc_local<float>(g, ig1, ql, qr, bns, fl);
  }
  f[0] = fl[0];
  f[1 + D] = fl[1];
  f[1 + t1] = fl[2];
  f[1 + t2] = fl[3];
  f[4] = fl[4];
  f[5 + D] = glm ? psis : 0.f;
  f[5 + t1] = fl[6];
  f[5 + t2] = fl[7];
  f[8] = glm ? ch * ch * bns : 0.f;
}

}  // namespace amrvac
