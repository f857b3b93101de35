// Shared device-side definitions of the amrvac GB300 library (not a public
// header).  Tables live in the caller's workspace; kernels receive a DevMesh by
// value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/amrvac.h"

namespace amrvac {

constexpr int NV = 9;       // rho, m_x, m_y, m_z, e, B_x, B_y, B_z, psi
constexpr int NG = 2;       // ghost cells per face of the two-ghost-cell limiters
constexpr int NG5 = 3;      // ghost cells per face of the five-point limiters (plain path)
constexpr int MAXLEV = AMRVAC_MAX_LEVELS;
constexpr int NPART = 12;   // per-block partials: smax, chmax, sums[9], pad

// the limiters that reconstruct from five cells (three ghost layers)
__host__ __device__ inline bool five_point_limiter(int lim) {
  return lim == AMRVAC_LIM_MP5 || lim == AMRVAC_LIM_WENO5 || lim == AMRVAC_LIM_WENOZ5 ||
         lim == AMRVAC_LIM_WENOZP5;
}
// per-(instance, level) stage constants of the fused kernels, refreshed from
// InstRT before every fused stage: c dt (the stage's Euler step), ch, psi
// damping factor over c dt, dx[3], 1/dx[3], finished flag (dt == 0), gamma,
// gamma - 1, and c2 dt with its damping factor (second output)
constexpr int LC_N = 16;
enum {
  LC_DT = 0, LC_CH = 1, LC_DAMP = 2, LC_DX = 3, LC_IDX = 6, LC_SKIP = 9, LC_G = 10,
  LC_GM1 = 11, LC_DT2 = 12, LC_DAMP2 = 13
};

// face neighbour codes in DevMesh::nbr
constexpr int NBR_OUTFLOW = -1;  // physical zero-gradient boundary
constexpr int NBR_GENERAL = -2;  // level change: use the per-level block maps
constexpr int NBR_GENERAL_FINER = -4;  // host tables only, while classifying faces
constexpr int NBR_WALL = -5;     // symmetric (reflecting) wall (fused: FULL kernels only)
// per-level block map codes
constexpr int MAP_REFINED = -1;  // covered by finer leaves
constexpr int MAP_COARSER = -2;  // covered by a coarser leaf

struct InstRT {      // per-instance clock and step parameters (device resident)
  double t, t_end, dt, ch;
};

struct DevMesh {
  int ndim;
  int ng;                 // ghost cells per face of the plain path (NG or NG5)
  int nx[3];
  int ncell;
  int nblocks;
  int ninst;
  int bc[3][2];
  const int* blk;         // [nblocks][5]: inst, level, i, j, k
  const int* nbr;         // [nblocks][6]: face (d, side) -> neighbour code
  const int* gface;       // [nblocks][6]: ghost-slab index of a level-change face, else -1
  const int* gkind;       // [slab index]: 1 the neighbour region is finer, 2 coarser
  void* fluxreg;          // refluxing: [slab index][NV][farea] face fluxes of the stage
  int farea;              // cells of the largest block face
  const int* lmap;        // concatenated dense per-(instance, level) block maps
  const int* lmap_off;    // [ninst][MAXLEV] offset into lmap
  const int* lnb;         // [ninst][MAXLEV][3] blocks per dimension at a level
  const double* gamma;    // [ninst]
  const double* dx;       // [ninst][MAXLEV][3] cell size
  const double* wzlam;    // [ninst][MAXLEV][3] dx^(2/3), the wenozp5 lambda
  const int* inst_start;  // [ninst + 1] CSR of blocks per instance
  const int* inst_blocks; // [nblocks]
  InstRT* rt;             // [ninst]
  double* part;           // [nblocks][NPART]
  double* sums;           // [ninst][NV]
  int* err;               // [4] code, block, cell, var
  float* lcf;             // [ninst][MAXLEV][LC_N] stage constants, float (FP32 bulk)
  double* lcd;            // [ninst][MAXLEV][LC_N] stage constants, double (FP64)
};

template <class T> __device__ __forceinline__ const T* level_consts(const DevMesh& M);
template <> __device__ __forceinline__ const float* level_consts<float>(const DevMesh& M) {
  return M.lcf;
}
template <> __device__ __forceinline__ const double* level_consts<double>(const DevMesh& M) {
  return M.lcd;
}

struct StageParams {
  int k;                 // stage index
  double a, b, c;        // out = a U0 + b (U + c dt L)
  double a2, b2, c2;     // out2 = a2 U2 + b2 (U + c2 dt L) when has2
  int plain;             // a == 0 and b == 1: out = U + c dt L (U0 not read)
  int has2;
  double courant;
  double glm_alpha;
  double small_density, small_pressure;
  int check_small;
  int flux, limiter, glm;
  int epilogue;          // 1: per-block dt / sums partials of the output
  int pressure_ff;       // FP32 bulk: float-float pressure recovery and sums
  float af, bf, a2f, b2f;  // a, b, a2, b2, small_density, small_pressure in float
  float small_density_f, small_pressure_f;
  int reflux;            // keep the fluxes of level-change faces for refluxing
  signed char lflux[MAXLEV], llim[MAXLEV];  // flux and limiter of each level
};

// a StageParams value in the kernel's arithmetic type (no conversion in-kernel)
template <class T> __device__ __forceinline__ T sp_val(double d, float f);
template <> __device__ __forceinline__ float sp_val<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double sp_val<double>(double d, float) { return d; }

__device__ __forceinline__ void latch_error(int* err, int code, int b, int c, int v) {
  if (atomicCAS(err, 0, code) == 0) {
    err[1] = b;
    err[2] = c;
    err[3] = v;
  }
}

}  // namespace amrvac
