// Plain per-block path: one kernel per step of the method and per stage.
//   k_prim   ghost fill + conserved -> primitive into a padded scratch box
//   k_flux   per direction: reconstruction, positivity fallback, glm + Riemann
//   k_update flux divergence, psi damping, SSPRK combination, optional
//            per-block dt / conservation partials of the output
// plus the CFL partials, the per-instance finalize, the ghost-fill export and
// precision conversion.  Scratch lives in the caller's workspace.
#include <cuda_runtime.h>

#include "ghost.cuh"
#include "physics.cuh"
#include "reduce.cuh"
#include "state.hpp"

namespace amrvac {

static inline int grid_for(size_t work, int threads) {
  size_t g = (work + threads - 1) / threads;
  size_t cap = 152 * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// ------------------------------------------------------------------ k_prim

template <class T>
__global__ void __launch_bounds__(256) k_prim(DevMesh M, const T* __restrict__ U,
                                              T* __restrict__ W, int P0, int P1, int P2,
                                              StageParams sp) {
  const size_t np = (size_t)P0 * P1 * P2;
  const size_t total = np * M.nblocks;
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int g0 = M.ng, g1 = M.ndim > 1 ? M.ng : 0, g2 = M.ndim > 2 ? M.ng : 0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(t / np);
    int pc = (int)(t - (size_t)b * np);
    int i = pc % P0 - g0, j = (pc / P0) % P1 - g1, k = pc / (P0 * P1) - g2;
    int outside = (i < 0 || i >= M.nx[0]) + (j < 0 || j >= M.nx[1]) + (k < 0 || k >= M.nx[2]);
    if (outside > 1) continue;
    const int* bi = M.blk + b * 5;
    if (M.rt[bi[0]].dt == 0.0) continue;
    T u[NV], w[NV];
    block_cell_value(M, U, vs, b, i, j, k, u);
    cons2prim(M.gamma[bi[0]], u, w);
    if (sp.check_small && is_small_prim(w[0], w[4], (T)sp.small_density, (T)sp.small_pressure))
      latch_error(M.err, AMRVAC_E_SMALL_VALUES, b, pc,
                  is_small_prim(w[0], T(1), (T)sp.small_density, T(0)) ? 0 : 4);
    T* dst = W + (size_t)b * NV * np + pc;
#pragma unroll
    for (int v = 0; v < NV; v++) dst[(size_t)v * np] = w[v];
  }
}

// ------------------------------------------------------------------ k_flux

template <class T>
__global__ void __launch_bounds__(256) k_flux(DevMesh M, const T* __restrict__ W,
                                              T* __restrict__ F, int d, int P0, int P1, int P2,
                                              StageParams sp) {
  const size_t np = (size_t)P0 * P1 * P2;
  int e0 = M.nx[0] + (d == 0), e1 = M.nx[1] + (d == 1), e2 = M.nx[2] + (d == 2);
  const size_t nf = (size_t)e0 * e1 * e2;
  const size_t total = nf * M.nblocks;
  const int g0 = M.ng, g1 = M.ndim > 1 ? M.ng : 0, g2 = M.ndim > 2 ? M.ng : 0;
  const int stride = d == 0 ? 1 : (d == 1 ? P0 : P0 * P1);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(t / nf);
    int fi = (int)(t - (size_t)b * nf);
    const int q = M.blk[b * 5];
    const InstRT rt = M.rt[q];
    if (rt.dt == 0.0) continue;
    const int lev = M.blk[b * 5 + 1];
    const int lim = sp.llim[lev], flux = sp.lflux[lev];  // the block's level's scheme
    int i = fi % e0, j = (fi / e0) % e1, k = fi / (e0 * e1);
    // padded index of the cell right of the face
    int pc = ((k + g2) * P1 + (j + g1)) * P0 + (i + g0);
    const T* src = W + (size_t)b * NV * np + pc;
    T wl[NV], wr[NV], w0[NV], w1[NV];
    if (five_point_limiter(lim)) {
      // five-point limiters: cells f-3 .. f+2 (three ghost layers)
      const T lam = (T)M.wzlam[(q * MAXLEV + lev) * 3 + d];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const T* s = src + (size_t)v * np;
        const T c[6] = {s[-3 * stride], s[-2 * stride], s[-stride], s[0], s[stride],
                        s[2 * stride]};
        wl[v] = recon5_plus(lim, c, lam);
        wr[v] = recon5_minus(lim, c + 1, lam);
        w0[v] = c[2];
        w1[v] = c[3];
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const T* s = src + (size_t)v * np;
        T s0 = s[-2 * stride], s1 = s[-stride], s2 = s[0], s3 = s[stride];
        wl[v] = recon_plus(lim, s0, s1, s2);
        wr[v] = recon_minus(lim, s1, s2, s3);
        w0[v] = s1;
        w1[v] = s2;
      }
    }
    if (!(wl[0] > T(0)) || !(wl[4] > T(0)) || !(wr[0] > T(0)) || !(wr[4] > T(0))) {
#pragma unroll
      for (int v = 0; v < NV; v++) {
        wl[v] = w0[v];
        wr[v] = w1[v];
      }
    }
    T f[NV];
    face_flux(flux, sp.glm, (T)M.gamma[q], (T)rt.ch, d, wl, wr, f);
    T* dst = F + (size_t)b * NV * nf + fi;
#pragma unroll
    for (int v = 0; v < NV; v++) dst[(size_t)v * nf] = f[v];
  }
}

// ------------------------------------------------------------------ k_update

template <class T>
__global__ void __launch_bounds__(256) k_update(DevMesh M, const T* U0,
                                                const T* Uk, const T* U2, T* out, T* out2,
                                                const T* __restrict__ F0,
                                                const T* __restrict__ F1,
                                                const T* __restrict__ F2, StageParams sp) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int nx0 = M.nx[0], nx1 = M.nx[1], nx2 = M.nx[2];
  const size_t nf0 = (size_t)(nx0 + 1) * nx1 * nx2;
  const size_t nf1 = (size_t)nx0 * (nx1 + 1) * nx2;
  const size_t nf2 = (size_t)nx0 * nx1 * (nx2 + 1);
  for (int b = blockIdx.x; b < M.nblocks; b += gridDim.x) {
    const int* bi = M.blk + b * 5;
    const int q = bi[0], L = bi[1];
    const InstRT rt = M.rt[q];
    const double* dxl = M.dx + (q * MAXLEV + L) * 3;
    double dx[3] = {dxl[0], dxl[1], dxl[2]};
    Partial p;
    partial_zero(p);
    const double gamma = M.gamma[q];
    double dxmin = dx[0];
    for (int d = 1; d < M.ndim; d++) dxmin = fmin(dxmin, dx[d]);
    const double dt1 = sp.c * rt.dt, dt2 = sp.c2 * rt.dt;
    const T damp = sp.glm ? (T)exp(-sp.glm_alpha * rt.ch * dt1 / dxmin) : T(1);
    const T damp2 = sp.glm ? (T)exp(-sp.glm_alpha * rt.ch * dt2 / dxmin) : T(1);
    const T dt = (T)dt1, dtb = (T)dt2, a = (T)sp.a, bb = (T)sp.b;
    const T a2 = (T)sp.a2, b2 = (T)sp.b2;
    const T idx0 = (T)dx[0], idx1 = (T)dx[1], idx2 = (T)dx[2];
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) {
      int i = c % nx0, j = (c / nx0) % nx1, k = c / (nx0 * nx1);
      T un[NV], u2n[NV];
      if (rt.dt == 0.0) {
#pragma unroll
        for (int v = 0; v < NV; v++) {
          un[v] = Uk[(size_t)v * vs + (size_t)b * M.ncell + c];
          u2n[v] = un[v];
        }
      } else {
        size_t f0 = ((size_t)k * nx1 + j) * (nx0 + 1) + i;
        size_t f1 = ((size_t)k * (nx1 + 1) + j) * nx0 + i;
        size_t f2 = ((size_t)k * nx1 + j) * nx0 + i;
#pragma unroll
        for (int v = 0; v < NV; v++) {
          const T* g0 = F0 + ((size_t)b * NV + v) * nf0;
          T acc = (g0[f0 + 1] - g0[f0]) / idx0;
          if (M.ndim > 1) {
            const T* g1 = F1 + ((size_t)b * NV + v) * nf1;
            acc += (g1[f1 + nx0] - g1[f1]) / idx1;
          }
          if (M.ndim > 2) {
            const T* g2 = F2 + ((size_t)b * NV + v) * nf2;
            acc += (g2[f2 + (size_t)nx0 * nx1] - g2[f2]) / idx2;
          }
          size_t at = (size_t)v * vs + (size_t)b * M.ncell + c;
          T ut = Uk[at] - dt * acc;
          if (v == 8) ut = ut * damp;
          un[v] = sp.plain ? ut : a * U0[at] + bb * ut;
          if (sp.has2) {
            T ut2 = Uk[at] - dtb * acc;
            if (v == 8) ut2 = ut2 * damp2;
            u2n[v] = a2 * U2[at] + b2 * ut2;
          }
        }
      }
      // written after every read: out may be U2's register and out2 U0's
#pragma unroll
      for (int v = 0; v < NV; v++) {
        out[(size_t)v * vs + (size_t)b * M.ncell + c] = un[v];
        if (sp.has2) out2[(size_t)v * vs + (size_t)b * M.ncell + c] = u2n[v];
      }
      if (sp.epilogue) accumulate_cell(M, un, gamma, dx, p, sp.pressure_ff != 0);
    }
    if (sp.epilogue) block_reduce_store(p, M.part + (size_t)b * NPART);
  }
}

// ------------------------------------------------------------------ k_cfl

template <class T>
__global__ void __launch_bounds__(256) k_cfl(DevMesh M, const T* __restrict__ U, int ff) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  for (int b = blockIdx.x; b < M.nblocks; b += gridDim.x) {
    const int* bi = M.blk + b * 5;
    const int q = bi[0], L = bi[1];
    const double* dxl = M.dx + (q * MAXLEV + L) * 3;
    double dx[3] = {dxl[0], dxl[1], dxl[2]};
    Partial p;
    partial_zero(p);
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) {
      T u[NV];
      read_cell(M, U, vs, b, c, u);
      accumulate_cell(M, u, M.gamma[q], dx, p, ff != 0);
    }
    block_reduce_store(p, M.part + (size_t)b * NPART);
  }
}

// ------------------------------------------------------------------ finalize

__global__ void __launch_bounds__(256) k_finalize(DevMesh M, double courant, int advance) {
  const int q = blockIdx.x;
  if (q >= M.ninst) return;
  __shared__ double sh[8][NPART];
  double smax = 0.0, chm = 0.0, sum[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) sum[v] = 0.0;
  const int b0 = M.inst_start[q], b1 = M.inst_start[q + 1];
  for (int n = b0 + threadIdx.x; n < b1; n += blockDim.x) {
    int b = M.inst_blocks[n];
    const double* pb = M.part + (size_t)b * NPART;
    const int L = M.blk[b * 5 + 1];
    const double* dxl = M.dx + (q * MAXLEV + L) * 3;
    double dv = dxl[0];
    for (int d = 1; d < M.ndim; d++) dv *= dxl[d];
    smax = fmax(smax, pb[0]);
    chm = fmax(chm, pb[1]);
#pragma unroll
    for (int v = 0; v < NV; v++) sum[v] += pb[2 + v] * dv;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    chm = fmax(chm, __shfl_xor_sync(0xffffffffu, chm, o));
#pragma unroll
    for (int v = 0; v < NV; v++) sum[v] += __shfl_xor_sync(0xffffffffu, sum[v], o);
  }
  if (lane == 0) {
    sh[warp][0] = smax;
    sh[warp][1] = chm;
#pragma unroll
    for (int v = 0; v < NV; v++) sh[warp][2 + v] = sum[v];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      sh[0][0] = fmax(sh[0][0], sh[w][0]);
      sh[0][1] = fmax(sh[0][1], sh[w][1]);
      for (int v = 0; v < NV; v++) sh[0][2 + v] += sh[w][2 + v];
    }
    InstRT r = M.rt[q];
    if (advance) {
      if (r.dt > 0.0 && r.dt >= r.t_end - r.t) r.t = r.t_end;
      else r.t += r.dt;
    }
    double d = courant / sh[0][0];
    double left = r.t_end - r.t;
    if (left <= 0.0) d = 0.0;
    else if (d >= left) d = left;
    r.dt = d;
    r.ch = sh[0][1];
    M.rt[q] = r;
  }
}

// ------------------------------------------------------------------ sums

// per-block integrals of each conserved variable of U (FP64, fixed order)
template <class T>
__global__ void __launch_bounds__(256) k_sums(DevMesh M, const T* __restrict__ U) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  __shared__ double sh[8][NV];
  for (int b = blockIdx.x; b < M.nblocks; b += gridDim.x) {
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) s[v] = 0.0;
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) {
#pragma unroll
      for (int v = 0; v < NV; v++) s[v] += (double)U[(size_t)v * vs + (size_t)b * M.ncell + c];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int v = 0; v < NV; v++) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    if (lane == 0)
      for (int v = 0; v < NV; v++) sh[warp][v] = s[v];
    __syncthreads();
    if (threadIdx.x < NV) {
      double acc = sh[0][threadIdx.x];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) acc += sh[w][threadIdx.x];
      M.part[(size_t)b * NPART + 2 + threadIdx.x] = acc;
    }
    __syncthreads();
  }
}

// per-instance sums of the block integrals times the cell volume (fixed order)
__global__ void __launch_bounds__(256) k_sums_finalize(DevMesh M) {
  const int q = blockIdx.x;
  if (q >= M.ninst) return;
  __shared__ double sh[8][NV];
  double sum[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) sum[v] = 0.0;
  for (int n = M.inst_start[q] + threadIdx.x; n < M.inst_start[q + 1]; n += blockDim.x) {
    const int b = M.inst_blocks[n];
    const double* dxl = M.dx + (q * MAXLEV + M.blk[b * 5 + 1]) * 3;
    double dv = dxl[0];
    for (int d = 1; d < M.ndim; d++) dv *= dxl[d];
#pragma unroll
    for (int v = 0; v < NV; v++) sum[v] += M.part[(size_t)b * NPART + 2 + v] * dv;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int v = 0; v < NV; v++) sum[v] += __shfl_xor_sync(0xffffffffu, sum[v], o);
  if (lane == 0)
    for (int v = 0; v < NV; v++) sh[warp][v] = sum[v];
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = sh[0][threadIdx.x];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) acc += sh[w][threadIdx.x];
    M.sums[q * NV + threadIdx.x] = acc;
  }
}

// ------------------------------------------------------------------ export / convert

template <class T>
__global__ void k_fill_ghosts(DevMesh M, const T* __restrict__ U, T* __restrict__ out, int P0,
                              int P1, int P2) {
  const size_t np = (size_t)P0 * P1 * P2;
  const size_t total = np * M.nblocks;
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int g0 = M.ng, g1 = M.ndim > 1 ? M.ng : 0, g2 = M.ndim > 2 ? M.ng : 0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(t / np);
    int pc = (int)(t - (size_t)b * np);
    int i = pc % P0 - g0, j = (pc / P0) % P1 - g1, k = pc / (P0 * P1) - g2;
    int outside = (i < 0 || i >= M.nx[0]) + (j < 0 || j >= M.nx[1]) + (k < 0 || k >= M.nx[2]);
    T u[NV];
    if (outside > 1) {
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = T(0);
    } else {
      block_cell_value(M, U, vs, b, i, j, k, u);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) out[((size_t)v * M.nblocks + b) * np + pc] = u[v];
  }
}

// primitive variables (rho, v, p, B, psi) of every interior cell of U into dst
// (same [var][block][cell] layout), with the state's pressure recovery: ff = 1
// the float-float form of FP32-bulk states, else the double subtraction
template <class T>
__global__ void __launch_bounds__(256) k_to_primitive(DevMesh M, const T* __restrict__ U,
                                                      T* __restrict__ dst, int ff) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < vs;
       t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / M.ncell);
    const double gamma = M.gamma[M.blk[b * 5]];
    T u[NV], w[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = U[(size_t)v * vs + t];
    cons2prim(gamma, u, w, ff != 0, (float)(gamma - 1.0));
#pragma unroll
    for (int v = 0; v < NV; v++) dst[(size_t)v * vs + t] = w[v];
  }
}

template <class S, class D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, size_t n) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = (D)src[t];
}

// ------------------------------------------------------------------ launchers

StageParams make_stage_params(const amrvac_state* s, int k, int epilogue) {
  StageParams sp;
  sp.k = k;
  const StageCoeffs co = stage_coeffs(s->cfg.time, k);
  sp.a = co.a;
  sp.b = co.b;
  sp.c = co.c;
  sp.a2 = co.a2;
  sp.b2 = co.b2;
  sp.c2 = co.c2;
  sp.plain = co.a == 0.0 && co.b == 1.0;
  sp.has2 = co.b2 != 0.0;
  sp.courant = s->cfg.courant;
  sp.glm_alpha = s->cfg.glm_alpha;
  sp.small_density = s->cfg.small_density;
  sp.small_pressure = s->cfg.small_pressure;
  // with fix_small_values the stage outputs are repaired instead of reported
  sp.check_small = s->cfg.check_small_values && s->cfg.fix_small_values == AMRVAC_FIX_OFF;
  sp.reflux = s->cfg.reflux;
  sp.flux = s->cfg.flux;
  sp.limiter = s->cfg.limiter;
  for (int L = 0; L < MAXLEV; L++) {
    sp.lflux[L] =
        (signed char)(s->cfg.level_flux[L] > 0 ? s->cfg.level_flux[L] - 1 : s->cfg.flux);
    sp.llim[L] =
        (signed char)(s->cfg.level_limiter[L] > 0 ? s->cfg.level_limiter[L] - 1 : s->cfg.limiter);
  }
  sp.glm = s->cfg.glm;
  sp.epilogue = epilogue;
  sp.pressure_ff = s->cfg.precision == AMRVAC_FP32_BULK && s->cfg.pressure == AMRVAC_PRESSURE_FF;
  sp.af = (float)sp.a;
  sp.bf = (float)sp.b;
  sp.a2f = (float)sp.a2;
  sp.b2f = (float)sp.b2;
  sp.small_density_f = (float)sp.small_density;
  sp.small_pressure_f = (float)sp.small_pressure;
  return sp;
}

// per-(instance, level) stage constants of the fused kernels from InstRT and
// the level's cell size (one thread per level)
__global__ void k_level_consts(DevMesh M, double glm_alpha, int glm, double c, double c2) {
  const int q = blockIdx.x, L = threadIdx.x;
  if (q >= M.ninst || L >= MAXLEV) return;
  const InstRT rt = M.rt[q];
  const double* dx = M.dx + (q * MAXLEV + L) * 3;
  double dxmin = fmin(dx[0], dx[1]);
  if (M.ndim == 3) dxmin = fmin(dxmin, dx[2]);
  const double g = M.gamma[q];
  float* f = M.lcf + (q * MAXLEV + L) * LC_N;
  double* d = M.lcd + (q * MAXLEV + L) * LC_N;
  // the stage's Euler step c dt and its psi damping factor (float bulk: exp of
  // the float-rounded argument); the same for the second output's c2 dt
  const double dt1 = c * rt.dt, dt2 = c2 * rt.dt;
  d[LC_DT] = dt1;
  f[LC_DT] = (float)dt1;
  d[LC_CH] = rt.ch;
  f[LC_CH] = (float)rt.ch;
  d[LC_DAMP] = glm ? exp(-glm_alpha * rt.ch * dt1 / dxmin) : 1.0;
  f[LC_DAMP] = glm ? expf((float)(-glm_alpha * rt.ch * dt1 / dxmin)) : 1.0f;
  d[LC_DT2] = dt2;
  f[LC_DT2] = (float)dt2;
  d[LC_DAMP2] = glm ? exp(-glm_alpha * rt.ch * dt2 / dxmin) : 1.0;
  f[LC_DAMP2] = glm ? expf((float)(-glm_alpha * rt.ch * dt2 / dxmin)) : 1.0f;
  for (int e = 0; e < 3; e++) {
    d[LC_DX + e] = dx[e];
    f[LC_DX + e] = (float)dx[e];
    d[LC_IDX + e] = 1.0 / dx[e];
    f[LC_IDX + e] = 1.0f / (float)dx[e];
  }
  d[LC_SKIP] = rt.dt == 0.0 ? 1.0 : 0.0;
  f[LC_SKIP] = rt.dt == 0.0 ? 1.0f : 0.0f;
  d[LC_G] = g;
  f[LC_G] = (float)g;
  d[LC_GM1] = g - 1.0;
  f[LC_GM1] = (float)(g - 1.0);
}

int launch_level_consts(amrvac_state* s, int k) {
  const StageCoeffs co = stage_coeffs(s->cfg.time, k);
  k_level_consts<<<s->ninst, MAXLEV, 0, s->stream>>>(s->mesh, s->cfg.glm_alpha, s->cfg.glm,
                                                      co.c, co.c2);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <class T> static int plain_stage_t(amrvac_state* s, int k, int epilogue) {
  const StageBuffers sb = stage_buffers(s->cfg.time, k);
  const int uin = sb.uin;
  StageParams sp = make_stage_params(s, k, epilogue);
  const DevMesh& M = s->mesh;
  size_t work = s->npad * s->nblocks;
  k_prim<T><<<grid_for(work, 256), 256, 0, s->stream>>>(M, (const T*)s->U[uin], (T*)s->W,
                                                        s->P[0], s->P[1], s->P[2], sp);
  for (int d = 0; d < s->ndim; d++)
    k_flux<T><<<grid_for(s->nface[d] * s->nblocks, 256), 256, 0, s->stream>>>(
        M, (const T*)s->W, (T*)s->F[d], d, s->P[0], s->P[1], s->P[2], sp);
  int grid = s->nblocks < 152 * 16 ? s->nblocks : 152 * 16;
  k_update<T><<<grid, 256, 0, s->stream>>>(
      M, (const T*)s->U[sb.u0], (const T*)s->U[uin],
      sb.u2 >= 0 ? (const T*)s->U[sb.u2] : nullptr, (T*)s->U[sb.out],
      sb.out2 >= 0 ? (T*)s->U[sb.out2] : nullptr, (const T*)s->F[0], (const T*)s->F[1],
      (const T*)s->F[2], sp);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return 2 + s->ndim;
}

int launch_plain_stage(amrvac_state* s, int k, int epilogue) {
  return s->cfg.precision == AMRVAC_FP64 ? plain_stage_t<double>(s, k, epilogue)
                                         : plain_stage_t<float>(s, k, epilogue);
}

int launch_cfl_partials(amrvac_state* s, int buffer) {
  int grid = s->nblocks < 152 * 16 ? s->nblocks : 152 * 16;
  const int ff = s->cfg.precision == AMRVAC_FP32_BULK && s->cfg.pressure == AMRVAC_PRESSURE_FF;
  if (s->cfg.precision == AMRVAC_FP64)
    k_cfl<double><<<grid, 256, 0, s->stream>>>(s->mesh, (const double*)s->U[buffer], 0);
  else
    k_cfl<float><<<grid, 256, 0, s->stream>>>(s->mesh, (const float*)s->U[buffer], ff);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_finalize(amrvac_state* s, int advance) {
  k_finalize<<<s->ninst, 256, 0, s->stream>>>(s->mesh, s->cfg.courant, advance);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_sums(amrvac_state* s, int buffer) {
  int grid = s->nblocks < 152 * 16 ? s->nblocks : 152 * 16;
  if (s->cfg.precision == AMRVAC_FP64)
    k_sums<double><<<grid, 256, 0, s->stream>>>(s->mesh, (const double*)s->U[buffer]);
  else
    k_sums<float><<<grid, 256, 0, s->stream>>>(s->mesh, (const float*)s->U[buffer]);
  k_sums_finalize<<<s->ninst, 256, 0, s->stream>>>(s->mesh);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int launch_fill_ghosts(amrvac_state* s, int buffer, void* out) {
  size_t work = s->npad * s->nblocks;
  if (s->cfg.precision == AMRVAC_FP64)
    k_fill_ghosts<double><<<grid_for(work, 256), 256, 0, s->stream>>>(
        s->mesh, (const double*)s->U[buffer], (double*)out, s->P[0], s->P[1], s->P[2]);
  else
    k_fill_ghosts<float><<<grid_for(work, 256), 256, 0, s->stream>>>(
        s->mesh, (const float*)s->U[buffer], (float*)out, s->P[0], s->P[1], s->P[2]);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_to_primitive(amrvac_state* s, int buffer, void* dst) {
  const size_t n = (size_t)s->nblocks * s->ncell;
  const int ff = s->cfg.precision == AMRVAC_FP32_BULK && s->cfg.pressure == AMRVAC_PRESSURE_FF;
  if (s->cfg.precision == AMRVAC_FP64)
    k_to_primitive<double><<<grid_for(n, 256), 256, 0, s->stream>>>(
        s->mesh, (const double*)s->U[buffer], (double*)dst, 0);
  else
    k_to_primitive<float><<<grid_for(n, 256), 256, 0, s->stream>>>(
        s->mesh, (const float*)s->U[buffer], (float*)dst, ff);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_convert(amrvac_state* s, const void* src, int src_prec, void* dst, int dst_prec,
                   size_t n) {
  int grid = grid_for(n, 256);
  if (src_prec == AMRVAC_FP64 && dst_prec == AMRVAC_FP32_BULK)
    k_convert<double, float><<<grid, 256, 0, s->stream>>>((const double*)src, (float*)dst, n);
  else if (src_prec == AMRVAC_FP32_BULK && dst_prec == AMRVAC_FP64)
    k_convert<float, double><<<grid, 256, 0, s->stream>>>((const float*)src, (double*)dst, n);
  else
    return -1;
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace amrvac
