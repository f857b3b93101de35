// CFL time step without any device allocation by the caller or the library.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns every allocation, plugins loaded into a process
// whose CUDA context forbids new allocations, or latency-critical loops where a
// cudaMalloc (and the device-wide synchronisation it can imply) is not
// allowed.  They cannot provide the workspace that amrvac_state_create needs.
// amrvac_cfl_dt_noalloc gives them the time step of a state they already hold
// in device memory: the per-block partial maxima that amrvac_cfl_dt keeps in
// the workspace live here in a fixed file-scope device array instead.
//
// The array is a static __device__ object: every GPU that loads this library
// holds it (AMRVAC_NOALLOC_MAX_BLOCKS x 2 doubles = 1 MiB) until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; that first call on a device should
// therefore come before any stream capture, and the cached address is stale
// once the caller resets that device (cudaDeviceReset).  All calls share the array: calls
// that overlap on the GPU (other streams, other host threads) race on it.
// Every slot a call reads is written by the same call first, so nothing has to
// be cleared between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "physics.cuh"
#include "reduce.cuh"

namespace {

using namespace amrvac;

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_cfl_partials[AMRVAC_NOALLOC_MAX_BLOCKS * 2];

std::mutex g_lock;
double* g_partials_addr[kMaxDevices] = {nullptr};

// per-block maxima of sum_d (|v_d| + c_f,d)/dx_d and of |v_d| + c_f,d
template <class T>
__global__ void __launch_bounds__(256) k_cfl_partials_static(DevMesh M, const T* __restrict__ U,
                                                             double gamma, double dx0,
                                                             double dx1, double dx2, int ff,
                                                             double* __restrict__ partials) {
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const double dx[3] = {dx0, dx1, dx2};
  for (int b = blockIdx.x; b < M.nblocks; b += gridDim.x) {
    Partial p;
    partial_zero(p);
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) {
      T u[NV];
      const T* src = U + (size_t)b * M.ncell + c;
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = src[(size_t)v * vs];
      accumulate_cell(M, u, gamma, dx, p, ff != 0);
    }
    // block maximum: warp shuffles, then the warps' maxima in a fixed order
    __shared__ double sh[32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p.smax = fmax(p.smax, __shfl_xor_sync(0xffffffffu, p.smax, o));
      p.chm = fmax(p.chm, __shfl_xor_sync(0xffffffffu, p.chm, o));
    }
    if (lane == 0) {
      sh[warp][0] = p.smax;
      sh[warp][1] = p.chm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double m0 = sh[0][0], m1 = sh[0][1];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
        m0 = fmax(m0, sh[w][0]);
        m1 = fmax(m1, sh[w][1]);
      }
      partials[2 * b] = m0;
      partials[2 * b + 1] = m1;
    }
    __syncthreads();
  }
}

// dt = C / max smax, clipped to t_end - t; c_h = max chm; out = {dt, c_h}
__global__ void __launch_bounds__(256) k_cfl_finish_static(const double* __restrict__ partials,
                                                           int nblocks, double courant,
                                                           double t, double t_end,
                                                           double* __restrict__ out) {
  __shared__ double sh[8][2];
  double smax = 0.0, chm = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    smax = fmax(smax, partials[2 * b]);
    chm = fmax(chm, partials[2 * b + 1]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    chm = fmax(chm, __shfl_xor_sync(0xffffffffu, chm, o));
  }
  if (lane == 0) {
    sh[warp][0] = smax;
    sh[warp][1] = chm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      sh[0][0] = fmax(sh[0][0], sh[w][0]);
      sh[0][1] = fmax(sh[0][1], sh[w][1]);
    }
    double d = courant / sh[0][0];
    double left = t_end - t;
    if (left <= 0.0) d = 0.0;
    else if (d >= left) d = left;
    out[0] = d;
    out[1] = sh[0][1];
  }
}

// device address of the static array on the current device (looked up once)
amrvac_status partials_address(double** addr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMRVAC_E_CUDA;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cfl_partials) != cudaSuccess || !p) return AMRVAC_E_CUDA;
    g_partials_addr[dev] = (double*)p;
  }
  *addr = g_partials_addr[dev];
  return AMRVAC_OK;
}

}  // namespace

extern "C" amrvac_status amrvac_cfl_dt_noalloc(const amrvac_config* cfg,
                                               const amrvac_instance_desc* inst,
                                               int32_t nblocks, const void* d_U, double t,
                                               double* d_out, void* cuda_stream) {
  if (!cfg || !inst || !d_U || !d_out) return AMRVAC_E_INVALID;
  if (cfg->ndim < 1 || cfg->ndim > 3) return AMRVAC_E_INVALID;
  if (cfg->precision != AMRVAC_FP64 && cfg->precision != AMRVAC_FP32_BULK) return AMRVAC_E_INVALID;
  if (!(cfg->courant > 0.0) || !(inst->gamma > 1.0)) return AMRVAC_E_INVALID;
  if (nblocks < 1 || nblocks > AMRVAC_NOALLOC_MAX_BLOCKS) return AMRVAC_E_INVALID;
  long long blocks = 1, cells = 1;  // 64-bit products: 4096^3 overflows an int
  DevMesh M{};
  M.ndim = cfg->ndim;
  double dx[3] = {1.0, 1.0, 1.0};
  for (int d = 0; d < 3; d++) {
    const bool act = d < cfg->ndim;
    M.nx[d] = act ? cfg->block_nx[d] : 1;
    if (act) {
      if (cfg->block_nx[d] < 4 || cfg->block_nx[d] > 4096 || inst->base_blocks[d] < 1)
        return AMRVAC_E_INVALID;
      if (!(inst->xmax[d] > inst->xmin[d])) return AMRVAC_E_INVALID;
      blocks *= inst->base_blocks[d];
      cells *= cfg->block_nx[d];
      dx[d] = (inst->xmax[d] - inst->xmin[d]) / ((double)inst->base_blocks[d] * cfg->block_nx[d]);
    }
  }
  if (blocks != nblocks) return AMRVAC_E_INVALID;  // one uniform level-0 instance only
  if (cells > AMRVAC_MAX_BLOCK_CELLS) return AMRVAC_E_INVALID;
  M.ncell = M.nx[0] * M.nx[1] * M.nx[2];
  M.nblocks = nblocks;
  M.ninst = 1;
  double* partials = nullptr;
  amrvac_status st = partials_address(&partials);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int grid = nblocks < 152 * 16 ? nblocks : 152 * 16;
  // float-float pressure recovery for FP32-bulk states configured with it
  const int ff = cfg->precision == AMRVAC_FP32_BULK && cfg->pressure == AMRVAC_PRESSURE_FF;
  if (cfg->precision == AMRVAC_FP64)
    k_cfl_partials_static<double><<<grid, 256, 0, s>>>(M, (const double*)d_U, inst->gamma, dx[0],
                                                       dx[1], dx[2], 0, partials);
  else
    k_cfl_partials_static<float><<<grid, 256, 0, s>>>(M, (const float*)d_U, inst->gamma, dx[0],
                                                      dx[1], dx[2], ff, partials);
  k_cfl_finish_static<<<1, 256, 0, s>>>(partials, nblocks, cfg->courant, t, inst->t_end, d_out);
  return cudaPeekAtLastError() == cudaSuccess ? AMRVAC_OK : AMRVAC_E_CUDA;
}
