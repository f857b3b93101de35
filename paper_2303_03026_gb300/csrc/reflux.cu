// Refluxing: conservative flux correction at coarse-fine faces.
//
// A stage computes the flux of a coarse block's face towards a finer
// neighbour from the coarse side (restricted ghosts) while the fine blocks
// compute their own fluxes through the same face (prolongated ghosts); without
// correction the two disagree and the level change leaks mass, momentum and
// energy.  After the stage the coarse cell next to such a face gets
//   out  += b  (c  dt) (+-) (F_coarse - mean of the 2^(d-1) fine fluxes) / dx
//   out2 += b2 (c2 dt) (+-) (...)                    (SSPRK(5,4) stage 3)
// + for the high face, - for the low face, the psi entry times its damping
// factor.  The face fluxes come from per-face registers: the fused kernels
// write them while computing the fluxes; the plain path copies them from its
// face-flux scratch (k_capture_faces).  One CTA takes one coarse block and
// its faces in a fixed order, so corner cells are corrected deterministically.
#include <cuda_runtime.h>

#include "ghost.cuh"
#include "state.hpp"

namespace amrvac {

namespace {

// tangential dimensions of a face normal to d, in increasing order
__device__ __forceinline__ void tangential(int d, int& ta, int& tb) {
  ta = d == 0 ? 1 : 0;
  tb = d == 2 ? 1 : 2;
}

// plain path: face fluxes of every level-change face from the F[d] scratch
template <class T>
__global__ void __launch_bounds__(256) k_capture_faces(DevMesh M, const T* __restrict__ F0,
                                                       const T* __restrict__ F1,
                                                       const T* __restrict__ F2,
                                                       const int* __restrict__ glist,
                                                       int ngen) {
  const int nx[3] = {M.nx[0], M.nx[1], M.nx[2]};
  for (int gi = blockIdx.x; gi < ngen; gi += gridDim.x) {
    const int b = glist[gi] / 6, f = glist[gi] % 6, d = f >> 1, side = f & 1;
    int ta, tb;
    tangential(d, ta, tb);
    int ext[3] = {nx[0], nx[1], nx[2]};
    ext[d] += 1;
    const size_t nf = (size_t)ext[0] * ext[1] * ext[2];
    const T* F = d == 0 ? F0 : (d == 1 ? F1 : F2);
    T* reg = (T*)M.fluxreg + (size_t)gi * NV * M.farea;
    const int area = nx[ta] * nx[tb];
    for (int t = threadIdx.x; t < area; t += blockDim.x) {
      const int t1 = t % nx[ta], t2 = t / nx[ta];
      int c[3];
      c[d] = side ? nx[d] : 0;
      c[ta] = t1;
      c[tb] = t2;
      const size_t fi = ((size_t)c[2] * ext[1] + c[1]) * ext[0] + c[0];
#pragma unroll
      for (int v = 0; v < NV; v++)
        reg[(size_t)v * M.farea + t] = F[((size_t)b * NV + v) * nf + fi];
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_reflux(DevMesh M, T* out, T* out2,
                                                const int* __restrict__ rlist, int nr,
                                                StageParams sp) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int nx[3] = {M.nx[0], M.nx[1], M.nx[2]};
  const T bb = sp_val<T>(sp.b, sp.bf), b2 = sp_val<T>(sp.b2, sp.b2f);
  for (int r = blockIdx.x; r < nr; r += gridDim.x) {
    const int b = rlist[r];
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const int bidx[3] = {M.blk[b * 5 + 2], M.blk[b * 5 + 3], M.blk[b * 5 + 4]};
    const T* lc = level_consts<T>(M) + (q * MAXLEV + L) * LC_N;
    if (lc[LC_SKIP] != T(0)) continue;
    const T dt1 = lc[LC_DT], damp = lc[LC_DAMP], dt2 = lc[LC_DT2], damp2 = lc[LC_DAMP2];
    for (int d = 0; d < M.ndim; d++) {
      int ta, tb;
      tangential(d, ta, tb);
      const T dx = lc[LC_DX + d];
      for (int side = 0; side < 2; side++) {
        const int f = d * 2 + side;
        if (M.nbr[b * 6 + f] != NBR_GENERAL) continue;
        const int gi = M.gface[b * 6 + f];
        if (M.gkind[gi] != 1) continue;
        const T* fc = (const T*)M.fluxreg + (size_t)gi * NV * M.farea;
        const int area = nx[ta] * nx[tb];
        for (int t = threadIdx.x; t < area; t += blockDim.x) {
          const int t1 = t % nx[ta], t2 = t / nx[ta];
          // fine cells across the face at level L+1 (global indices)
          int g[3] = {0, 0, 0};
          g[d] = side ? 2 * (bidx[d] * nx[d] + nx[d]) : 2 * bidx[d] * nx[d] - 1;
          T fm[NV];
#pragma unroll
          for (int v = 0; v < NV; v++) fm[v] = T(0);
          int nfine = 0;
          for (int o2 = 0; o2 < (tb < M.ndim ? 2 : 1); o2++)
            for (int o1 = 0; o1 < (ta < M.ndim ? 2 : 1); o1++) {
              g[ta] = ta < M.ndim ? 2 * (bidx[ta] * nx[ta] + t1) + o1 : 0;
              g[tb] = tb < M.ndim ? 2 * (bidx[tb] * nx[tb] + t2) + o2 : 0;
              int p[3] = {g[0], g[1], g[2]};
              wrap_level(M, q, L + 1, p);
              int cell;
              const int fb = map_at(M, q, L + 1, p, &cell);
              if (fb < 0) {  // never with a 2:1-balanced mesh
                latch_error(M.err, AMRVAC_E_STATE, b, t, f);
                continue;
              }
              const int ci_a = p[ta] % nx[ta], ci_b = tb < M.ndim ? p[tb] % nx[tb] : 0;
              const T* ff = (const T*)M.fluxreg +
                            (size_t)M.gface[fb * 6 + (f ^ 1)] * NV * M.farea +
                            ci_b * nx[ta] + ci_a;
#pragma unroll
              for (int v = 0; v < NV; v++) fm[v] += ff[(size_t)v * M.farea];
              nfine++;
            }
          if (nfine == 0) continue;
          int c[3];
          c[d] = side ? nx[d] - 1 : 0;
          c[ta] = t1;
          c[tb] = t2;
          const size_t at = (size_t)b * M.ncell + ((size_t)c[2] * nx[1] + c[1]) * nx[0] + c[0];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            const T dF = fc[(size_t)v * M.farea + t] - fm[v] / T(nfine);
            const T dL = (side ? dF : -dF) / dx;
            out[(size_t)v * vs + at] += bb * dt1 * dL * (v == 8 ? damp : T(1));
            if (sp.has2) out2[(size_t)v * vs + at] += b2 * dt2 * dL * (v == 8 ? damp2 : T(1));
          }
        }
        __syncthreads();  // the next face may correct the same corner cells
      }
    }
  }
}

template <class T> int reflux_t(amrvac_state* s, int k) {
  int n = 0;
  const StageBuffers sb = stage_buffers(s->cfg.time, k);
  StageParams sp = make_stage_params(s, k, 0);
  if (!s->use_fused) {
    if (s->ngen > 0) {
      const int g = s->ngen < 152 * 8 ? s->ngen : 152 * 8;
      k_capture_faces<T><<<g, 256, 0, s->stream>>>(s->mesh, (const T*)s->F[0],
                                                    (const T*)s->F[1], (const T*)s->F[2],
                                                    s->d_glist, s->ngen);
      n++;
    }
    if (launch_level_consts(s, k) < 0) return -1;
    n++;
  }
  if (s->nrlist > 0) {
    const int g = s->nrlist < 152 * 8 ? s->nrlist : 152 * 8;
    k_reflux<T><<<g, 256, 0, s->stream>>>(s->mesh, (T*)s->U[sb.out],
                                           sb.out2 >= 0 ? (T*)s->U[sb.out2] : nullptr,
                                           s->d_rlist, s->nrlist, sp);
    n++;
  }
  return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

}  // namespace

int launch_reflux(amrvac_state* s, int k) {
  if (!s->cfg.reflux) return 0;
  return s->cfg.precision == AMRVAC_FP64 ? reflux_t<double>(s, k) : reflux_t<float>(s, k);
}

}  // namespace amrvac
