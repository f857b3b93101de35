// Per-block partials of the CFL reduction and the conservation sums, and their
// deterministic CTA reduction (fixed shuffle tree, fixed warp order).
#pragma once

#include "physics.cuh"

namespace amrvac {

struct Partial {
  double smax, chm, sum[NV];
};

__device__ __forceinline__ void partial_zero(Partial& p) {
  p.smax = 0.0;
  p.chm = 0.0;
#pragma unroll
  for (int v = 0; v < NV; v++) p.sum[v] = 0.0;
}

// deterministic block reduction (fixed shuffle tree + fixed warp order) of a
// Partial; thread 0 writes it to part[b]
static __device__ void block_reduce_store(Partial& p, double* part_b) {
  __shared__ double sh[32][NPART];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    p.smax = fmax(p.smax, __shfl_xor_sync(0xffffffffu, p.smax, o));
    p.chm = fmax(p.chm, __shfl_xor_sync(0xffffffffu, p.chm, o));
#pragma unroll
    for (int v = 0; v < NV; v++) p.sum[v] += __shfl_xor_sync(0xffffffffu, p.sum[v], o);
  }
  if (lane == 0) {
    sh[warp][0] = p.smax;
    sh[warp][1] = p.chm;
#pragma unroll
    for (int v = 0; v < NV; v++) sh[warp][2 + v] = p.sum[v];
  }
  __syncthreads();
  if (threadIdx.x < NPART) {
    const int nw = blockDim.x >> 5;
    double acc = sh[0][threadIdx.x];
    for (int w = 1; w < nw; w++) {
      double x = sh[w][threadIdx.x];
      acc = threadIdx.x < 2 ? fmax(acc, x) : acc + x;
    }
    part_b[threadIdx.x] = threadIdx.x < 2 + NV ? acc : 0.0;
  }
  __syncthreads();
}

// per-cell CFL terms: sum_d (|v_d| + c_f,d)/dx_d and max_d (|v_d| + c_f,d), in the
// bulk precision (inverse cell sizes precomputed); conservation sums in double
template <class T>
__device__ __forceinline__ void accumulate_cell(const DevMesh& M, const T* u, double gamma,
                                                const double* dx, Partial& p, bool ff = false) {
  // CFL terms only (the conservation sums are reduced on demand by k_sums);
  // ff: float-float pressure recovery of FP32-bulk states
  T w[NV];
  cons2prim(gamma, u, w, ff, (float)(gamma - 1.0));
  T s = T(0), cm = T(0);
  for (int d = 0; d < M.ndim; d++) {
    T spd = fabs(w[1 + d]) + fast_speed((T)gamma, w, d);
    s += spd / (T)dx[d];
    cm = fmax(cm, spd);
  }
  p.smax = fmax(p.smax, (double)s);
  p.chm = fmax(p.chm, (double)cm);
}

// same reduction with caller-provided shared scratch red[>= nwarps][NPART]
__device__ __forceinline__ void block_reduce_red(double (*red)[NPART], Partial& p, double* part_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    p.smax = fmax(p.smax, __shfl_xor_sync(0xffffffffu, p.smax, o));
    p.chm = fmax(p.chm, __shfl_xor_sync(0xffffffffu, p.chm, o));
#pragma unroll
    for (int v = 0; v < NV; v++) p.sum[v] += __shfl_xor_sync(0xffffffffu, p.sum[v], o);
  }
  __syncthreads();
  if (lane == 0) {
    red[warp][0] = p.smax;
    red[warp][1] = p.chm;
#pragma unroll
    for (int v = 0; v < NV; v++) red[warp][2 + v] = p.sum[v];
  }
  __syncthreads();
  if (threadIdx.x < NPART) {
    const int nw = blockDim.x >> 5;
    double acc = red[0][threadIdx.x];
    for (int w = 1; w < nw; w++) {
      double x = red[w][threadIdx.x];
      acc = threadIdx.x < 2 ? fmax(acc, x) : acc + x;
    }
    part_b[threadIdx.x] = threadIdx.x < 2 + NV ? acc : 0.0;
  }
  __syncthreads();
}

}  // namespace amrvac
