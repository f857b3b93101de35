// Host-side state of the amrvac library (not a public header).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "common.cuh"

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
  int* d_glist = nullptr;  // [ngen] b * 6 + face
  int ngen = 0;
  // launch shape of the fused kernel (see amrvac_tuning)
  amrvac_tuning tune{0, 0, 0, 0.0};
  int* d_work_morton = nullptr;
  int* d_work_storage = nullptr;
  int* d_counter = nullptr;
  // host copies
  std::vector<int32_t> meta;
  std::vector<amrvac_instance_desc> inst;
  bool dt_valid = false;
  cudaGraphExec_t graph = nullptr;
  int graph_kernels = 0;
  int64_t launches = 0;
};

namespace amrvac {

// stage coefficients of the Shu-Osher form: out = a U^n + b (U + dt L(U))
inline void stage_coeffs(int time, int k, double* a, double* b) {
  if (k == 0) {
    *a = 0.0;
    *b = 1.0;
  } else if (time == AMRVAC_SSPRK2) {
    *a = 0.5;
    *b = 0.5;
  } else if (k == 1) {
    *a = 0.75;
    *b = 0.25;
  } else {
    *a = 1.0 / 3.0;
    *b = 2.0 / 3.0;
  }
}

inline int num_stages(int time) { return time == AMRVAC_SSPRK2 ? 2 : 3; }

// buffers read (U0, Uin) and written (out) by stage k
inline void stage_buffers(int time, int k, int* u0, int* uin, int* out) {
  *u0 = 0;
  if (k == 0) {
    *uin = 0;
    *out = 1;
  } else if (time == AMRVAC_SSPRK2) {
    *uin = 1;
    *out = 0;
  } else if (k == 1) {
    *uin = 1;
    *out = 2;
  } else {
    *uin = 2;
    *out = 0;
  }
}

StageParams make_stage_params(const amrvac_state* s, int k, int epilogue);

// kernel launchers (plain.cu / fused kernels); each returns the number of
// kernels it launched or -1 on a launch error
int launch_plain_stage(amrvac_state* s, int k, int epilogue);
int launch_cfl_partials(amrvac_state* s, int buffer);
int launch_finalize(amrvac_state* s, int advance);
int launch_sums(amrvac_state* s, int buffer);
int launch_level_consts(amrvac_state* s);
int launch_fill_ghosts(amrvac_state* s, int buffer, void* out);
int launch_convert(amrvac_state* s, const void* src, int src_prec, void* dst, int dst_prec,
                   size_t n);
int launch_fused_stage(amrvac_state* s, int k, int epilogue);
bool fused_supported(const amrvac_config* cfg);

}  // namespace amrvac
