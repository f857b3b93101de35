// Host-side state of the amrvac library (not a public header).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace amrvac {
// transfer table of a regrid, per destination block: kind (0 copy,
// 1 prolongation from a parent, 2 restriction of children), source block, and
// the 2^ndim source children of a merged parent in (z, y, x) order
constexpr int RTAB_N = 10;
// CTAs of the compaction of the device regrid plan
constexpr int PLAN_CTAS = 512;

// device regrid plan scratch (in the workspace)
struct PlanScratch {
  int* ref = nullptr;           // [nblocks] 1 when the leaf splits
  signed char* fate = nullptr;  // [nblocks] keep, split, first child of a merge, merged away
  int* map = nullptr;           // dense new-leaf marks, per (instance, level) segment
  int* seg = nullptr;           // [ninst * MAXLEV + 1] segment offsets of map
  int* maxlev = nullptr;        // [ninst] deepest level of the current mesh
  int* sums = nullptr;          // [PLAN_CTAS + 1] per-CTA counts, then their prefix
  int* scal = nullptr;          // [0] changed, [1] new block count, [2] error
  int* out = nullptr;           // [cap][5] the new block list
  int cap = 0;
  int nmap = -1;                // entries of map; -1: the dense maps would be too large
};
}  // namespace amrvac

struct amrvac_state {
  amrvac_config cfg;
  int ninst = 0, nblocks = 0, ncell = 0;
  int ndim = 1;
  int use_fused = 0;
  size_t real_size = 8;                 // bytes per stored value
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  void* U[3] = {nullptr, nullptr, nullptr};
  // plain-path scratch: padded primitives and face fluxes per dimension
  void* W = nullptr;
  void* F[3] = {nullptr, nullptr, nullptr};
  int P[3] = {1, 1, 1};                 // padded extents
  size_t npad = 1;                      // padded cells per block
  size_t nface[3] = {0, 0, 0};          // faces per block per dimension
  amrvac::DevMesh mesh{};
  // fused-path work list: blocks grouped for the persistent kernel
  int* d_work = nullptr;
  int nwork = 0;
  // fused path: ghost slabs of the level-change faces (2 layers x 16 x 16
  // cells x 9 vars each), rebuilt from the stage input before every stage
  void* gslab = nullptr;
  // fix_small_values: one flag byte per cell and a count of repaired cells
  unsigned char* d_flags = nullptr;
  unsigned long long* d_fixcount = nullptr;
  int* d_glist = nullptr;  // [ngen] b * 6 + face
  int ngen = 0;
  // refluxing: blocks with a finer face neighbour, face flux registers
  int* d_rlist = nullptr;
  int nrlist = 0;
  void* fluxreg = nullptr;
  // launch shape of the fused kernel (see amrvac_tuning)
  amrvac_tuning tune{0, 0, 0, 0, 0.0};
  int* d_work_morton = nullptr;
  int* d_work_storage = nullptr;
  int* d_counter = nullptr;  // one dynamic-schedule counter per scheme group
  // fused path: scheme groups (levels sharing a flux and limiter), each a
  // contiguous range [grp_off, grp_off + grp_cnt) of the work lists
  int ngroups = 1;
  int grp_flux[amrvac::MAXLEV] = {0}, grp_lim[amrvac::MAXLEV] = {0};
  int grp_off[amrvac::MAXLEV] = {0}, grp_cnt[amrvac::MAXLEV] = {0};
  // regridding: per-block estimator and flag, transfer table [nblocks][RTAB_N]
  double* d_est = nullptr;
  signed char* d_eflags = nullptr;
  int* d_rtab = nullptr;
  amrvac::PlanScratch plan;
  // host copies
  std::vector<int32_t> meta;
  std::vector<amrvac_instance_desc> inst;
  bool dt_valid = false;
  cudaGraphExec_t graph = nullptr;
  int graph_kernels = 0;
  int64_t launches = 0;
};

namespace amrvac {

// Shu-Osher coefficients of stage k: out = a U0 + b (U_in + c dt L(U_in)) and,
// for SSPRK(5,4) stage 3 only (b2 != 0), out2 = a2 U2 + b2 (U_in + c2 dt L(U_in)).
// SSPRK(4,3) and SSPRK(5,4) are the optimal schemes of Spiteri & Ruuth 2002:
//   SSPRK(4,3): u1 = u0 + dt/2 L(u0), u2 = u1 + dt/2 L(u1),
//               u3 = 2/3 u0 + 1/3 (u2 + dt/2 L(u2)), u4 = u3 + dt/2 L(u3)
//   SSPRK(5,4): u1 = u0 + 0.391752226571890 dt L(u0)
//               u2 = 0.444370493651235 u0 + 0.555629506348765 u1 + 0.368410593050371 dt L(u1)
//               u3 = 0.620101851488403 u0 + 0.379898148511597 u2 + 0.251891774271694 dt L(u2)
//               u4 = 0.178079954393132 u0 + 0.821920045606868 u3 + 0.544974750228521 dt L(u3)
//               u5 = 0.517231671970585 u2 + 0.096059710526147 u3 + 0.063692468666290 dt L(u3)
//                    + 0.386708617503269 u4 + 0.226007483236906 dt L(u4)
// with w = the u2, u3, L(u3) part of u5 produced by stage 3.
struct StageCoeffs {
  double a, b, c, a2, b2, c2;
};

inline StageCoeffs stage_coeffs(int time, int k) {
  StageCoeffs r{0.0, 1.0, 1.0, 0.0, 0.0, 0.0};
  if (time == AMRVAC_SSPRK2) {
    if (k == 1) r.a = 0.5, r.b = 0.5;
  } else if (time == AMRVAC_SSPRK3) {
    if (k == 1) r.a = 0.75, r.b = 0.25;
    if (k == 2) r.a = 1.0 / 3.0, r.b = 2.0 / 3.0;
  } else if (time == AMRVAC_SSPRK43) {
    r.c = 0.5;
    if (k == 2) r.a = 2.0 / 3.0, r.b = 1.0 / 3.0;
  } else {
    if (k == 0) {
      r.c = 0.391752226571890;
    } else if (k == 1) {
      r.a = 0.444370493651235, r.b = 0.555629506348765, r.c = 0.368410593050371 / r.b;
    } else if (k == 2) {
      r.a = 0.620101851488403, r.b = 0.379898148511597, r.c = 0.251891774271694 / r.b;
    } else if (k == 3) {
      r.a = 0.178079954393132, r.b = 0.821920045606868, r.c = 0.544974750228521 / r.b;
      r.a2 = 0.517231671970585, r.b2 = 0.096059710526147, r.c2 = 0.063692468666290 / r.b2;
    } else {
      r.a = 1.0, r.b = 0.386708617503269, r.c = 0.226007483236906 / r.b;
    }
  }
  return r;
}

inline int num_stages(int time) {
  return time == AMRVAC_SSPRK2 ? 2 : time == AMRVAC_SSPRK3 ? 3 : time == AMRVAC_SSPRK43 ? 4 : 5;
}

// state registers used by stage k: U0, U_in, U2 (-1: none) -> out, out2 (-1)
struct StageBuffers {
  int u0, uin, u2, out, out2;
};

inline StageBuffers stage_buffers(int time, int k) {
  if (k == 0) return {0, 0, -1, 1, -1};
  if (time == AMRVAC_SSPRK2) return {0, 1, -1, 0, -1};
  if (k == 1) return {0, 1, -1, 2, -1};
  if (time == AMRVAC_SSPRK3) return {0, 2, -1, 0, -1};
  if (time == AMRVAC_SSPRK43) return k == 2 ? StageBuffers{0, 2, -1, 1, -1}
                                            : StageBuffers{0, 1, -1, 0, -1};
  if (k == 2) return {0, 2, -1, 1, -1};
  if (k == 3) return {0, 1, 2, 2, 0};
  return {0, 2, -1, 0, -1};
}

StageParams make_stage_params(const amrvac_state* s, int k, int epilogue);

// kernel launchers (plain.cu / fused kernels); each returns the number of
// kernels it launched or -1 on a launch error
int launch_plain_stage(amrvac_state* s, int k, int epilogue);
int launch_cfl_partials(amrvac_state* s, int buffer);
int launch_finalize(amrvac_state* s, int advance);
int launch_sums(amrvac_state* s, int buffer);
int launch_level_consts(amrvac_state* s, int k);
int launch_fix_small(amrvac_state* s, int buffer);
int launch_reflux(amrvac_state* s, int k);
int launch_fill_ghosts(amrvac_state* s, int buffer, void* out);
int launch_to_primitive(amrvac_state* s, int buffer, void* dst);
int launch_convert(amrvac_state* s, const void* src, int src_prec, void* dst, int dst_prec,
                   size_t n);
int launch_fused_stage(amrvac_state* s, int k, int epilogue);
bool fused_supported(const amrvac_config* cfg);
bool fused_supported5(const amrvac_config* cfg);

}  // namespace amrvac
