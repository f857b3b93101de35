// Bootstrapping of small values (fix_small_values, Sect. 7.4).
//
// Two passes over a state register after a stage (or on request):
//   k_flag_small: one flag byte per cell, set when the cell's density or
//                 pressure is below its floor or not positive; counts them.
//   k_fix_small:  every flagged cell is rewritten in place, either with the
//                 floors (velocity kept, 0 where rho <= 0) or with the mean
//                 primitive state of its same-level face neighbours that are
//                 not flagged.  Flagged cells never feed another cell's mean,
//                 so the result does not depend on the order of the writes.
// B and psi are never changed; momentum and energy follow from the new
// primitives.  The pressure test of FP32-bulk states uses the float-float
// recovery (the FP64 pipe is too narrow for a per-cell double pass); the
// repairs of the few flagged cells are computed in double.
#include <cuda_runtime.h>

#include "physics.cuh"
#include "state.hpp"

namespace amrvac {

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_flag_small(DevMesh M, const T* __restrict__ U,
                                                    unsigned char* __restrict__ flags,
                                                    double sd, double sp_, int ff,
                                                    unsigned long long* count) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  unsigned long long n = 0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < vs;
       t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / M.ncell);
    const double g = M.gamma[M.blk[b * 5]];
    T u[NV], w[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = U[(size_t)v * vs + t];
    cons2prim(g, u, w, ff != 0, (float)(g - 1.0));
    const bool small = is_small_prim(w[0], w[4], (T)sd, (T)sp_);
    flags[t] = small ? 1 : 0;
    n += small ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, n);
}

// primitive (rho, vx, vy, vz, p) in double of a conserved cell
template <class T>
__device__ __forceinline__ void prim5(const T* U, size_t vs, size_t at, double g, double* w) {
  double u[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) u[v] = (double)U[(size_t)v * vs + at];
  double q[NV];
  cons2prim(g, u, q);
#pragma unroll
  for (int e = 0; e < 5; e++) w[e] = q[e];
}

template <class T>
__global__ void __launch_bounds__(256) k_fix_small(DevMesh M, T* U,
                                                   const unsigned char* __restrict__ flags,
                                                   int method, double sd, double sp_) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < vs;
       t += (size_t)gridDim.x * blockDim.x) {
    if (!flags[t]) continue;
    const int b = (int)(t / M.ncell), c = (int)(t - (size_t)b * M.ncell);
    const double g = M.gamma[M.blk[b * 5]];
    const int ijk[3] = {c % M.nx[0], (c / M.nx[0]) % M.nx[1], c / (M.nx[0] * M.nx[1])};
    double sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int n = 0;
    if (method == AMRVAC_FIX_AVERAGE) {
      for (int d = 0; d < M.ndim; d++)
        for (int side = 0; side < 2; side++) {
          int q[3] = {ijk[0], ijk[1], ijk[2]};
          q[d] += side ? 1 : -1;
          int nb = b;
          if (q[d] < 0 || q[d] >= M.nx[d]) {
            nb = M.nbr[b * 6 + d * 2 + side];  // same-level neighbour only
            if (nb < 0) continue;
            q[d] = side ? 0 : M.nx[d] - 1;
          }
          const size_t at = (size_t)nb * M.ncell + ((size_t)q[2] * M.nx[1] + q[1]) * M.nx[0] + q[0];
          if (flags[at]) continue;
          double w[5];
          prim5(U, vs, at, g, w);
#pragma unroll
          for (int e = 0; e < 5; e++) sum[e] += w[e];
          n++;
        }
    }
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = (double)U[(size_t)v * vs + t];
    double wf[NV];
    if (n > 0) {
#pragma unroll
      for (int e = 0; e < 5; e++) wf[e] = sum[e] / n;
    } else {
      double q[NV];
      cons2prim(g, u, q);
      wf[0] = u[0] > sd ? u[0] : sd;
      for (int e = 0; e < 3; e++) wf[1 + e] = u[0] > 0.0 ? q[1 + e] : 0.0;
      wf[4] = (u[0] > 0.0 && q[4] > sp_) ? q[4] : sp_;
    }
    for (int v = 5; v < NV; v++) wf[v] = u[v];
    // conserved from the repaired primitives (B, psi unchanged)
    const double rho = wf[0];
    const double ke = 0.5 * rho * (wf[1] * wf[1] + wf[2] * wf[2] + wf[3] * wf[3]);
    const double me = 0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
    U[t] = (T)rho;
    U[vs + t] = (T)(rho * wf[1]);
    U[2 * vs + t] = (T)(rho * wf[2]);
    U[3 * vs + t] = (T)(rho * wf[3]);
    U[4 * vs + t] = (T)(wf[4] / (g - 1.0) + ke + me);
  }
}

template <class T> int launch_fix_t(amrvac_state* s, int buffer) {
  const size_t vs = (size_t)s->nblocks * s->ncell;
  size_t g = (vs + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  const double sd = s->cfg.small_density, sp_ = s->cfg.small_pressure;
  const int ff = s->cfg.precision == AMRVAC_FP32_BULK && s->cfg.pressure == AMRVAC_PRESSURE_FF;
  k_flag_small<T><<<(int)g, 256, 0, s->stream>>>(s->mesh, (const T*)s->U[buffer], s->d_flags,
                                                  sd, sp_, ff, s->d_fixcount);
  k_fix_small<T><<<(int)g, 256, 0, s->stream>>>(s->mesh, (T*)s->U[buffer], s->d_flags,
                                                 s->cfg.fix_small_values, sd, sp_);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

}  // namespace

int launch_fix_small(amrvac_state* s, int buffer) {
  if (s->cfg.fix_small_values == AMRVAC_FIX_OFF || !s->d_flags) return 0;
  return s->cfg.precision == AMRVAC_FP64 ? launch_fix_t<double>(s, buffer)
                                         : launch_fix_t<float>(s, buffer);
}

}  // namespace amrvac

extern "C" amrvac_status amrvac_fix_small_values(amrvac_state* s, int32_t buffer,
                                                 int64_t* h_count) {
  using namespace amrvac;
  if (!s || buffer < 0 || buffer > 2 || s->cfg.fix_small_values == AMRVAC_FIX_OFF ||
      !s->d_flags)
    return AMRVAC_E_INVALID;
  if (h_count && cudaMemsetAsync(s->d_fixcount, 0, sizeof(unsigned long long), s->stream) !=
                     cudaSuccess)
    return AMRVAC_E_CUDA;
  const int n = launch_fix_small(s, buffer);
  if (n < 0) return AMRVAC_E_CUDA;
  s->launches += n;
  if (h_count) {
    unsigned long long c = 0;
    if (cudaMemcpyAsync(&c, s->d_fixcount, sizeof(c), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      return AMRVAC_E_CUDA;
    *h_count = (int64_t)c;
  }
  return AMRVAC_OK;
}
