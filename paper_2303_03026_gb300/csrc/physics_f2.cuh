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

// fast speeds of both sides; bx2 = B_n^2
__device__ __forceinline__ float2 fast2(float g, float2 rho, float2 p, float2 by, float2 bz,
                                        float bx2) {
  float2 ir = rcp2(rho);
  float2 bt = fma2(bz, bz, mul2(by, by));
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

// total pressure and total energy of both sides
__device__ __forceinline__ void pt_e2(const Side2& q, float bx2, float ig1, float2& pt,
                                      float2& e) {
  float2 b2 = fma2(q.bz, q.bz, fma2(q.by, q.by, sp2(bx2)));
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
  float2 pt, e;
  pt_e2(q, bx2, ig1, pt, e);
  float2 cf = fast2(g, q.rho, q.p, q.by, q.bz, bx2);
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
  float2 pt, e;
  pt_e2(q, bx2, ig1, pt, e);
  const float2 cf = fast2(g, q.rho, q.p, q.by, q.bz, bx2);
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
  float2 pt, e;
  pt_e2(q, bx2, ig1, pt, e);
  float2 cf = fast2(g, q.rho, q.p, q.by, q.bz, bx2);
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
  const float2 sqr = sqrt2(rs);
  const float2 isq = rcp2(sqr);
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
    // runtime limiter: one switch per face, the variable loop inside
    if (lim == AMRVAC_LIM_SUPERBEE) {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = sym_pair<1>(st(v, 0), st(v, 1), st(v, 2), st(v, 3), 0.f);
    } else if (lim == AMRVAC_LIM_ALBADA) {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = sym_pair<2>(st(v, 0), st(v, 1), st(v, 2), st(v, 3), 0.f);
    } else if (lim == AMRVAC_LIM_CADA3) {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = cada3_pair(st(v, 0), st(v, 1), st(v, 2), st(v, 3));
    } else {
      const float beta = lim == AMRVAC_LIM_WOODWARD ? 2.f : 1.4f;
#pragma unroll
      for (int v = 0; v < NV; v++)
        w[v] = sym_pair<0>(st(v, 0), st(v, 1), st(v, 2), st(v, 3), beta);
    }
  }
  if (!(w[0].x > 0.f) || !(w[4].x > 0.f) || !(w[0].y > 0.f) || !(w[4].y > 0.f)) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = make_float2(st(v, 1), st(v, 2));
  }
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
