// Dynamic regridding of the block-AMR mesh (Sect. 1 and 3: automatic
// refinement and coarsening where chosen quantities vary).
//
//   k_regrid_estimate(_tiled): per block, the maximum over its cells of the
//       weighted sum of Loehner's normalised second derivatives of the chosen
//       primitive quantities (face neighbours across block faces from the
//       ghost operators of the update), and the block's refine / coarsen flag.
//       The arithmetic is double with explicit round-to-nearest operations;
//       the tiled form stages the quantities in shared memory.
//   amrvac_regrid_plan (host) and amrvac_regrid_plan_device: the new block
//       list, closed under 2:1 balance.
//   k_regrid_copy, k_regrid_restrict, k_regrid_transfer: fill a state built
//       on the new list from the old one: copy (kept blocks, wide elements),
//       restriction (mean of the 2^d children cells) or prolongation (coarse
//       value plus minmod-limited slopes times +-1/4).  Sums are formed in double in a fixed order
//       and rounded once to the state's precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ghost.cuh"
#include "physics.cuh"
#include "state.hpp"

namespace amrvac {

namespace {

constexpr double LOEHNER_EPS = 0.01;  // noise filter of the estimator's denominator

int grid_for(int nblocks) { return nblocks < 152 * 8 ? nblocks : 152 * 8; }

struct EstWeights {
  double w[NV];  // weight of each primitive variable (rho, v, p, B, psi)
  int prim;      // 1 when a variable other than rho is weighted
};

// the weighted quantities of block-local cell (i, j, k) with at most one
// index outside the block (ghost values of the level there), in double
template <class T>
__device__ __forceinline__ void est_cell(const DevMesh& M, const T* U, size_t vs, int b, int i,
                                         int j, int k, const EstWeights& ew, double g,
                                         double* q) {
  const bool inside = i >= 0 && i < M.nx[0] && j >= 0 && j < M.nx[1] && k >= 0 && k < M.nx[2];
  if (!ew.prim && inside) {
    q[0] = (double)U[(size_t)b * M.ncell + ((size_t)k * M.nx[1] + j) * M.nx[0] + i];
    return;
  }
  T u[NV];
  block_cell_value(M, U, vs, b, i, j, k, u);
  double ud[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) ud[v] = (double)u[v];
  if (ew.prim) {
    cons2prim(g, ud, q);
  } else {
    q[0] = ud[0];
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_regrid_estimate(DevMesh M, const T* __restrict__ U,
                                                         EstWeights ew, double thr, double dthr,
                                                         int maxlev, double* est,
                                                         signed char* flags) {
  __shared__ double red[256 / 32];
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int nq = ew.prim ? NV : 1;
  for (int b = blockIdx.x; b < M.nblocks; b += gridDim.x) {
    const double g = M.gamma[M.blk[b * 5]];
    double emax = 0.0;
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) {
      const int ci[3] = {c % M.nx[0], (c / M.nx[0]) % M.nx[1], c / (M.nx[0] * M.nx[1])};
      double q0[NV], num[NV], den[NV];
      est_cell(M, U, vs, b, ci[0], ci[1], ci[2], ew, g, q0);
      for (int v = 0; v < nq; v++) num[v] = den[v] = 0.0;
      for (int d = 0; d < M.ndim; d++) {
        int p[3] = {ci[0], ci[1], ci[2]}, m[3] = {ci[0], ci[1], ci[2]};
        p[d] += 1;
        m[d] -= 1;
        double qp[NV], qm[NV];
        est_cell(M, U, vs, b, p[0], p[1], p[2], ew, g, qp);
        est_cell(M, U, vs, b, m[0], m[1], m[2], ew, g, qm);
        for (int v = 0; v < nq; v++) {
          if (ew.w[v] == 0.0) continue;
          const double rp = qp[v], r0 = q0[v], rm = qm[v];
          const double s2 = __dadd_rn(__dsub_rn(rp, 2.0 * r0), rm);
          num[v] = __dadd_rn(num[v], __dmul_rn(s2, s2));
          const double a = __dadd_rn(fabs(__dsub_rn(rp, r0)), fabs(__dsub_rn(r0, rm)));
          const double f = __dadd_rn(__dadd_rn(fabs(rp), 2.0 * fabs(r0)), fabs(rm));
          const double dd = __dadd_rn(a, __dmul_rn(LOEHNER_EPS, f));
          den[v] = __dadd_rn(den[v], __dmul_rn(dd, dd));
        }
      }
      double e = 0.0;
      for (int v = 0; v < nq; v++) {
        if (ew.w[v] == 0.0) continue;
        const double r = den[v] > 0.0 ? num[v] / den[v] : 0.0;
        e = __dadd_rn(e, __dmul_rn(ew.w[v], sqrt(r)));
      }
      emax = e > emax ? e : emax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, emax, o);
      emax = other > emax ? other : emax;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) emax = red[w] > emax ? red[w] : emax;
      const int L = M.blk[b * 5 + 1];
      est[b] = emax;
      flags[b] = (emax > thr && L < maxlev) ? 1 : ((emax < dthr && L > 0) ? -1 : 0);
    }
    __syncthreads();  // red is reused by the next block
  }
}

// The same estimator, tiled: per block, the weighted quantities of its cells
// and of its one-cell face halo are formed once per chunk of variables into
// shared memory [chunk var][padded cell] (primitives recovered once per cell,
// not once per stencil use), the cells' estimates accumulate in shared memory
// over the chunks in ascending variable order, then the block maximum is
// taken.  Every value and every operation order equals k_regrid_estimate's.
// A block whose every stencil cell (its cells and their face neighbours)
// holds bit for bit the conserved values of its first cell is recorded with
// the estimate 0 without the double arithmetic: equal inputs give equal
// primitives, every second difference is then exactly 0, so num = 0 and every
// cell's estimate is +0 (also where den is 0 or the values are not finite,
// which the quotient's guard turns into 0).
constexpr int EST_TILED_THREADS = 512;

template <class T> __device__ __forceinline__ bool same_bits(T a, T b);
template <> __device__ __forceinline__ bool same_bits<float>(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b);
}
template <> __device__ __forceinline__ bool same_bits<double>(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

template <class T>
__global__ void __launch_bounds__(EST_TILED_THREADS, 1)
    k_regrid_estimate_tiled(DevMesh M, const T* __restrict__ U, EstWeights ew, int nch,
                            double thr, double dthr, int maxlev, double* est,
                            signed char* flags) {
  extern __shared__ double tile[];
  __shared__ double red[EST_TILED_THREADS / 32];
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int h1 = M.ndim > 1 ? 1 : 0, h2 = M.ndim > 2 ? 1 : 0;
  const int P0 = M.nx[0] + 2, P1 = M.nx[1] + 2 * h1, P2 = M.nx[2] + 2 * h2;
  const int np = P0 * P1 * P2;
  double* ecell = tile + (size_t)nch * np;
  int vars[NV], nw = 0;
  for (int v = 0; v < (ew.prim ? NV : 1); v++)
    if (ew.w[v] != 0.0) vars[nw++] = v;
  const int stride[3] = {1, P0, P0 * P1};
  for (int b = blockIdx.x; b < M.nblocks; b += gridDim.x) {
    const double g = M.gamma[M.blk[b * 5]];
    // uniform block: every stencil cell equal to the first cell, bit for bit
    T ref[NV];
    read_cell(M, U, vs, b, 0, ref);
    int same = 1;
    for (int t = threadIdx.x; t < np && same; t += blockDim.x) {
      const int i = t % P0 - 1, j = (t / P0) % P1 - h1, k = t / (P0 * P1) - h2;
      const int outside =
          (i < 0 || i >= M.nx[0]) + (j < 0 || j >= M.nx[1]) + (k < 0 || k >= M.nx[2]);
      if (outside > 1) continue;
      T u[NV];
      block_cell_value(M, U, vs, b, i, j, k, u);
#pragma unroll
      for (int v = 0; v < NV; v++) same = same && same_bits(u[v], ref[v]);
    }
    if (__syncthreads_and(same)) {
      if (threadIdx.x == 0) {
        const int L = M.blk[b * 5 + 1];
        est[b] = 0.0;
        flags[b] = (0.0 > thr && L < maxlev) ? 1 : ((0.0 < dthr && L > 0) ? -1 : 0);
      }
      continue;  // uniform across the CTA
    }
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) ecell[c] = 0.0;
    for (int c0 = 0; c0 < nw; c0 += nch) {
      const int cn = nw - c0 < nch ? nw - c0 : nch;
      __syncthreads();  // the previous chunk's (or block's) readers are done
      for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int i = t % P0 - 1, j = (t / P0) % P1 - h1, k = t / (P0 * P1) - h2;
        const int outside =
            (i < 0 || i >= M.nx[0]) + (j < 0 || j >= M.nx[1]) + (k < 0 || k >= M.nx[2]);
        if (outside > 1) continue;  // edge and corner cells are never read
        double q[NV];
        est_cell(M, U, vs, b, i, j, k, ew, g, q);
        // the chunk's weighted quantities, q indexed by constants only (a
        // runtime index would put q in local memory)
        int rank = 0;
#pragma unroll
        for (int v = 0; v < NV; v++) {
          if (v >= (ew.prim ? NV : 1) || ew.w[v] == 0.0) continue;
          if (rank >= c0 && rank < c0 + cn) tile[(size_t)(rank - c0) * np + t] = q[v];
          rank++;
        }
      }
      __syncthreads();
      for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) {
        const int ci[3] = {c % M.nx[0], (c / M.nx[0]) % M.nx[1], c / (M.nx[0] * M.nx[1])};
        const int t0 = ((ci[2] + h2) * P1 + (ci[1] + h1)) * P0 + ci[0] + 1;
        double e = ecell[c];
        for (int cc = 0; cc < cn; cc++) {
          const double* q = tile + (size_t)cc * np;
          const double r0 = q[t0];
          double num = 0.0, den = 0.0;
          for (int d = 0; d < M.ndim; d++) {
            const double rp = q[t0 + stride[d]], rm = q[t0 - stride[d]];
            const double s2 = __dadd_rn(__dsub_rn(rp, 2.0 * r0), rm);
            num = __dadd_rn(num, __dmul_rn(s2, s2));
            const double a = __dadd_rn(fabs(__dsub_rn(rp, r0)), fabs(__dsub_rn(r0, rm)));
            const double f = __dadd_rn(__dadd_rn(fabs(rp), 2.0 * fabs(r0)), fabs(rm));
            const double dd = __dadd_rn(a, __dmul_rn(LOEHNER_EPS, f));
            den = __dadd_rn(den, __dmul_rn(dd, dd));
          }
          const double r = den > 0.0 ? num / den : 0.0;
          e = __dadd_rn(e, __dmul_rn(ew.w[vars[c0 + cc]], sqrt(r)));
        }
        ecell[c] = e;
      }
    }
    __syncthreads();
    double emax = 0.0;
    for (int c = threadIdx.x; c < M.ncell; c += blockDim.x) emax = ecell[c] > emax ? ecell[c] : emax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, emax, o);
      emax = other > emax ? other : emax;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); w++) emax = red[w] > emax ? red[w] : emax;
      const int L = M.blk[b * 5 + 1];
      est[b] = emax;
      flags[b] = (emax > thr && L < maxlev) ? 1 : ((emax < dthr && L > 0) ? -1 : 0);
    }
  }
}

template <class T>
int launch_estimate(amrvac_state* s, const T* U, const EstWeights& ew, double thr, double dthr,
                    int maxlev) {
  // tiled when one variable's padded block and the cell estimates fit
  constexpr size_t SMEM_MAX = 200 * 1024;
  const amrvac::DevMesh& M = s->mesh;
  size_t np = 1;
  for (int d = 0; d < 3; d++) np *= (size_t)(M.nx[d] + (d < M.ndim ? 2 : 0));
  const size_t cells = sizeof(double) * (size_t)M.ncell;
  int nw = 0;
  for (int v = 0; v < (ew.prim ? NV : 1); v++) nw += ew.w[v] != 0.0;
  if (cells + sizeof(double) * np <= SMEM_MAX) {
    int nch = (int)((SMEM_MAX - cells) / (sizeof(double) * np));
    if (nch > nw) nch = nw;
    const size_t smem = cells + sizeof(double) * np * (size_t)nch;
    if (cudaFuncSetAttribute(k_regrid_estimate_tiled<T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -1;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return -1;
    const int g = s->nblocks < nsm * 2 ? s->nblocks : nsm * 2;
    k_regrid_estimate_tiled<T><<<g, EST_TILED_THREADS, smem, s->stream>>>(
        M, U, ew, nch, thr, dthr, maxlev, s->d_est, s->d_eflags);
  } else {
    k_regrid_estimate<T><<<grid_for(s->nblocks), 256, 0, s->stream>>>(M, U, ew, thr, dthr,
                                                                        maxlev, s->d_est,
                                                                        s->d_eflags);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// children of split blocks (kind 1 in the table): one thread per cell of the
// parent covered by the child's octant computes that cell's minmod slopes once
// and writes its 2^d child cells, each the coarse value plus the slopes times
// +-1/4 summed in the order of the dimensions (the arithmetic of one cell does
// not depend on which thread does it)
template <class T>
__global__ void __launch_bounds__(256) k_regrid_transfer(DevMesh Ms, const T* __restrict__ Us,
                                                         DevMesh Md, T* __restrict__ Ud,
                                                         const int* __restrict__ tab) {
  const size_t vss = (size_t)Ms.nblocks * Ms.ncell, vsd = (size_t)Md.nblocks * Md.ncell;
  const int nd = Md.ndim;
  const int nx[3] = {Md.nx[0], Md.nx[1], Md.nx[2]};
  const int h[3] = {nx[0] / 2, nd > 1 ? nx[1] / 2 : 1, nd > 2 ? nx[2] / 2 : 1};
  const int nh = h[0] * h[1] * h[2];  // parent cells under one child block
  for (int b = blockIdx.x; b < Md.nblocks; b += gridDim.x) {
    const int* t = tab + (size_t)b * RTAB_N;
    const int kind = t[0], sb = t[1];
    if (kind != 1) continue;  // kept blocks: k_regrid_copy; merged parents: k_regrid_restrict
    const int idx[3] = {Md.blk[b * 5 + 2], Md.blk[b * 5 + 3], Md.blk[b * 5 + 4]};
    for (int e = threadIdx.x; e < nh; e += blockDim.x) {
      // parent cell pc of the split block sb, local cell lc of the octant
      const int lc[3] = {e % h[0], (e / h[0]) % h[1], e / (h[0] * h[1])};
      int pc[3];
#pragma unroll
      for (int d = 0; d < 3; d++) pc[d] = d < nd ? (idx[d] & 1) * h[d] + lc[d] : 0;
      T ub[NV];
      read_cell(Ms, Us, vss, sb, (pc[2] * nx[1] + pc[1]) * nx[0] + pc[0], ub);
      double base[NV], sl[3][NV];
#pragma unroll
      for (int v = 0; v < NV; v++) base[v] = (double)ub[v];
      for (int d = 0; d < nd; d++) {
        int p[3] = {pc[0], pc[1], pc[2]}, m[3] = {pc[0], pc[1], pc[2]};
        p[d] += 1;
        m[d] -= 1;
        T up[NV], um[NV];
        block_cell_value(Ms, Us, vss, sb, p[0], p[1], p[2], up);
        block_cell_value(Ms, Us, vss, sb, m[0], m[1], m[2], um);
#pragma unroll
        for (int v = 0; v < NV; v++) {
          const double a = base[v] - (double)um[v], bb = (double)up[v] - base[v];
          sl[d][v] = a * bb > 0.0 ? (a > 0.0 ? fmin(a, bb) : fmax(a, bb)) : 0.0;
        }
      }
      for (int cz = 0; cz < (nd > 2 ? 2 : 1); cz++)
        for (int cy = 0; cy < (nd > 1 ? 2 : 1); cy++)
          for (int cx = 0; cx < 2; cx++) {
            const int co[3] = {cx, cy, cz};
            const size_t dst = (size_t)b * Md.ncell +
                               ((size_t)(2 * lc[2] + cz) * nx[1] + (2 * lc[1] + cy)) * nx[0] +
                               2 * lc[0] + cx;
#pragma unroll
            for (int v = 0; v < NV; v++) {
              double out = base[v];
              for (int d = 0; d < nd; d++) out = out + (co[d] ? 0.25 : -0.25) * sl[d][v];
              Ud[(size_t)v * vsd + dst] = (T)out;
            }
          }
    }
  }
}

template <class T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// merged parents of a transfer (kind 2 in the table): each cell the mean of
// the 2^d cells of one child it covers, summed in double in a fixed order and
// rounded once; a kernel of its own, so that the register-heavy prolongation
// does not limit its occupancy
template <class T>
__global__ void __launch_bounds__(256) k_regrid_restrict(DevMesh Ms, const T* __restrict__ Us,
                                                         DevMesh Md, T* __restrict__ Ud,
                                                         const int* __restrict__ tab) {
  const size_t vss = (size_t)Ms.nblocks * Ms.ncell, vsd = (size_t)Md.nblocks * Md.ncell;
  const int nd = Md.ndim;
  const int nx[3] = {Md.nx[0], Md.nx[1], Md.nx[2]};
  const int h[3] = {nx[0] / 2, nd > 1 ? nx[1] / 2 : 1, nd > 2 ? nx[2] / 2 : 1};
  for (int b = blockIdx.x; b < Md.nblocks; b += gridDim.x) {
    const int* t = tab + (size_t)b * RTAB_N;
    if (t[0] != 2) continue;
    for (int c = threadIdx.x; c < Md.ncell; c += blockDim.x) {
      const size_t dst = (size_t)b * Md.ncell + c;
      const int ci[3] = {c % nx[0], (c / nx[0]) % nx[1], c / (nx[0] * nx[1])};
      double out[NV];
      // merged parent: its cell ci covers 2^d cells of one child
      int o[3], f0[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        o[d] = d < nd ? ci[d] / h[d] : 0;
        f0[d] = d < nd ? 2 * ci[d] - o[d] * nx[d] : 0;
      }
      const int cb = t[2 + (o[2] * 2 + o[1]) * 2 + o[0]];
#pragma unroll
      for (int v = 0; v < NV; v++) out[v] = 0.0;
      // the two x-neighbours of a child pair in one aligned 2-wide load (the
      // pair starts at an even cell of an even-width row), summed in the
      // order (fz, fy, fx)
      for (int fz = 0; fz < (nd > 2 ? 2 : 1); fz++)
        for (int fy = 0; fy < (nd > 1 ? 2 : 1); fy++) {
          const size_t src = (size_t)cb * Ms.ncell +
                             ((size_t)(f0[2] + fz) * nx[1] + (f0[1] + fy)) * nx[0] + f0[0];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            const auto pr = *reinterpret_cast<const typename Pair<T>::type*>(
                Us + (size_t)v * vss + src);
            out[v] += (double)pr.x;
            out[v] += (double)pr.y;
          }
        }
      const double inv = nd == 3 ? 0.125 : (nd == 2 ? 0.25 : 0.5);  // exact
#pragma unroll
      for (int v = 0; v < NV; v++) out[v] *= inv;
#pragma unroll
      for (int v = 0; v < NV; v++) Ud[(size_t)v * vsd + dst] = (T)out[v];
    }
  }
}

// the kept blocks of a transfer (kind 0 in the table): each variable's run of
// cells copied from the source block, W-wide elements (the run length in W
// units is nw), every other block skipped; a lean kernel at full occupancy
// beside the register-heavy prolongation of k_regrid_transfer
template <class W>
__global__ void __launch_bounds__(256) k_regrid_copy(const W* __restrict__ Us, W* __restrict__ Ud,
                                                     const int* __restrict__ tab, int nblocks_dst,
                                                     size_t vss, size_t vsd, int nw) {
  const size_t total = (size_t)nblocks_dst * NV * nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % nw);
    const size_t r = e / nw;
    const int v = (int)(r % NV), b = (int)(r / NV);
    const int* t = tab + (size_t)b * RTAB_N;
    if (t[0] != 0) continue;
    Ud[(size_t)v * vsd + (size_t)b * nw + x] = Us[(size_t)v * vss + (size_t)t[1] * nw + x];
  }
}

using Key = std::array<int, 5>;  // instance, level, i, j, k

struct KeyHash {  // FNV-1a over the five ints
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int v : k) {
      h ^= (uint32_t)v;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};
using KeySet = std::unordered_set<Key, KeyHash>;

// (instance, level, k, j, i) order: the last block index fastest
struct KeyBlockOrder {
  bool operator()(const Key& a, const Key& b) const {
    const std::array<int, 5> x{a[0], a[1], a[4], a[3], a[2]}, y{b[0], b[1], b[4], b[3], b[2]};
    return x < y;
  }
};

struct Planner {
  int nd;
  bool periodic[3];
  std::vector<std::array<int, 3>> base;
  int nblk(int q, int L, int d) const { return d < nd ? base[q][d] << L : 1; }

  // level-L positions around (i, j, k) (faces, edges, corners), wrapped on
  // periodic dimensions, dropped outside the others
  std::vector<std::array<int, 3>> neighbours(int q, int L, int i, int j, int k) const {
    std::vector<std::array<int, 3>> out;
    const int lo[3] = {-1, nd > 1 ? -1 : 0, nd > 2 ? -1 : 0};
    for (int dz = lo[2]; dz <= -lo[2]; dz++)
      for (int dy = lo[1]; dy <= -lo[1]; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          if (!dx && !dy && !dz) continue;
          std::array<int, 3> p{i + dx, j + dy, k + dz};
          bool ok = true;
          for (int d = 0; d < nd; d++) {
            const int n = nblk(q, L, d);
            if (p[d] < 0 || p[d] >= n) {
              if (periodic[d]) p[d] = ((p[d] % n) + n) % n;
              else ok = false;
            }
          }
          if (ok) out.push_back(p);
        }
    return out;
  }

  // level of the leaf of s covering level-L position p (walking up), -1 when
  // finer leaves cover it
  static int covering(const KeySet& s, int q, int L, std::array<int, 3> p) {
    for (int LL = L; LL >= 0; LL--) {
      if (s.count(Key{q, LL, p[0], p[1], p[2]})) return LL;
      for (int d = 0; d < 3; d++) p[d] >>= 1;
    }
    return -1;
  }

  std::vector<Key> children(const Key& k) const {
    std::vector<Key> out;
    for (int oz = 0; oz < (nd > 2 ? 2 : 1); oz++)
      for (int oy = 0; oy < (nd > 1 ? 2 : 1); oy++)
        for (int ox = 0; ox < 2; ox++)
          out.push_back(Key{k[0], k[1] + 1, 2 * k[2] + ox, nd > 1 ? 2 * k[3] + oy : 0,
                            nd > 2 ? 2 * k[4] + oz : 0});
    return out;
  }

  // deepest leaf level of s around the parent position (q, L, i, j, k)
  int finest_near(const KeySet& s, int q, int L, int i, int j, int k) const {
    int best = L;
    for (const auto& p : neighbours(q, L, i, j, k)) {
      const int lev = covering(s, q, L, p);
      if (lev >= 0) {
        best = std::max(best, lev);
        continue;
      }
      for (const Key& c : children(Key{q, L, p[0], p[1], p[2]})) {
        const int l2 = covering(s, q, L + 1, {c[2], c[3], c[4]});
        best = std::max(best, l2 < 0 ? L + 2 : l2);
      }
    }
    return best;
  }
};

}  // namespace

}  // namespace amrvac

using namespace amrvac;

extern "C" amrvac_status amrvac_regrid_plan(const amrvac_config* cfg, int32_t ninst,
                                            const amrvac_instance_desc* inst, int32_t nblocks,
                                            const int32_t* block_meta, const int8_t* flags,
                                            int32_t capacity, int32_t* new_meta,
                                            int32_t* new_nblocks) {
  size_t bytes = 0;
  if (!flags || !new_nblocks || capacity < 0 || (capacity > 0 && !new_meta))
    return AMRVAC_E_INVALID;
  const amrvac_status st = amrvac_workspace_bytes(cfg, ninst, inst, nblocks, block_meta, &bytes);
  if (st != AMRVAC_OK) return st;
  Planner P;
  P.nd = cfg->ndim;
  for (int d = 0; d < 3; d++) P.periodic[d] = cfg->bc[d][0] == AMRVAC_BC_PERIODIC;
  for (int q = 0; q < ninst; q++)
    P.base.push_back({inst[q].base_blocks[0], inst[q].base_blocks[1], inst[q].base_blocks[2]});
  KeySet cur, refine;
  std::vector<Key> want;
  cur.reserve((size_t)nblocks * 2);
  for (int b = 0; b < nblocks; b++) {
    const int32_t* r = block_meta + 5 * b;
    const Key k{r[0], r[1], r[2], P.nd > 1 ? r[3] : 0, P.nd > 2 ? r[4] : 0};
    cur.insert(k);
    if (flags[b] < -1 || flags[b] > 1) return AMRVAC_E_INVALID;
    if (flags[b] == 1) {
      if (r[1] + 1 >= AMRVAC_MAX_LEVELS) return AMRVAC_E_INVALID;
      refine.insert(k);
    }
    if (flags[b] == -1 && r[1] > 0) want.push_back(k);
  }
  // 2:1 closure of the splits: a split level-L leaf forces every coarser
  // leaf around it to split too
  std::vector<Key> todo(refine.begin(), refine.end());
  while (!todo.empty()) {
    const Key k = todo.back();
    todo.pop_back();
    for (const auto& p : P.neighbours(k[0], k[1], k[2], k[3], k[4])) {
      const int lev = Planner::covering(cur, k[0], k[1], p);
      if (lev < 0 || lev >= k[1]) continue;
      std::array<int, 3> pp = p;
      for (int s = 0; s < k[1] - lev; s++)
        for (int d = 0; d < 3; d++) pp[d] >>= 1;
      const Key c{k[0], lev, pp[0], pp[1], pp[2]};
      if (refine.insert(c).second) todo.push_back(c);
    }
  }
  KeySet next;
  next.reserve(cur.size() + refine.size() * ((size_t)1 << P.nd));
  for (const Key& k : cur) {
    if (refine.count(k)) {
      for (const Key& c : P.children(k)) next.insert(c);
    } else {
      next.insert(k);
    }
  }
  // merges: complete families asking for it, parents in (instance, level,
  // k, j, i) order
  std::map<Key, std::vector<Key>, KeyBlockOrder> parents;
  for (const Key& k : want) {
    if (refine.count(k)) continue;
    parents[Key{k[0], k[1] - 1, k[2] >> 1, k[3] >> 1, k[4] >> 1}].push_back(k);
  }
  const size_t nchild = (size_t)1 << P.nd;
  for (const auto& it : parents) {
    const Key& par = it.first;
    const std::vector<Key>& kids = it.second;
    if (kids.size() != nchild) continue;
    bool all = true;
    for (const Key& c : kids) all = all && next.count(c);
    if (!all) continue;
    // merge in place; undo it when the parent would touch a leaf two levels finer
    for (const Key& c : kids) next.erase(c);
    next.insert(par);
    if (P.finest_near(next, par[0], par[1], par[2], par[3], par[4]) > par[1] + 1) {
      next.erase(par);
      for (const Key& c : kids) next.insert(c);
    }
  }
  *new_nblocks = (int32_t)next.size();
  if ((size_t)capacity < next.size()) return AMRVAC_E_INVALID;
  std::vector<Key> out(next.begin(), next.end());
  std::sort(out.begin(), out.end(), KeyBlockOrder());
  for (size_t b = 0; b < out.size(); b++)
    for (int e = 0; e < 5; e++) new_meta[5 * b + e] = out[b][e];
  return AMRVAC_OK;
}

extern "C" amrvac_status amrvac_regrid_estimate(amrvac_state* s, int32_t buffer,
                                                const double* weights, double refine_threshold,
                                                double derefine_ratio, int32_t max_level,
                                                double* h_est, int8_t* h_flags) {
  if (!s || buffer < 0 || buffer > 2 || !(refine_threshold >= 0.0) || !(derefine_ratio >= 0.0) ||
      max_level < 0 || max_level >= AMRVAC_MAX_LEVELS)
    return AMRVAC_E_INVALID;
  EstWeights ew{};
  ew.w[0] = 1.0;
  if (weights) {
    bool any = false;
    for (int v = 0; v < NV; v++) {
      if (!(weights[v] >= 0.0) || !std::isfinite(weights[v])) return AMRVAC_E_INVALID;
      ew.w[v] = weights[v];
      any = any || weights[v] > 0.0;
      if (v > 0 && weights[v] > 0.0) ew.prim = 1;
    }
    if (!any) return AMRVAC_E_INVALID;
  }
  const double dthr = derefine_ratio * refine_threshold;
  const int n = s->cfg.precision == AMRVAC_FP64
                    ? launch_estimate<double>(s, (const double*)s->U[buffer], ew,
                                              refine_threshold, dthr, max_level)
                    : launch_estimate<float>(s, (const float*)s->U[buffer], ew,
                                             refine_threshold, dthr, max_level);
  if (n < 0) return AMRVAC_E_CUDA;
  s->launches += n;
  if (h_est && cudaMemcpyAsync(h_est, s->d_est, sizeof(double) * s->nblocks,
                               cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return AMRVAC_E_CUDA;
  if (h_flags && cudaMemcpyAsync(h_flags, s->d_eflags, (size_t)s->nblocks,
                                 cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return AMRVAC_E_CUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return AMRVAC_E_CUDA;
  int err = 0;  // a ghost lookup that found no leaf latches the device error
  if (cudaMemcpy(&err, s->mesh.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AMRVAC_E_CUDA;
  return err ? (amrvac_status)err : AMRVAC_OK;
}

extern "C" amrvac_status amrvac_regrid_transfer(amrvac_state* src, int32_t src_buffer,
                                                amrvac_state* dst, int32_t dst_buffer) {
  if (!src || !dst || src_buffer < 0 || src_buffer > 2 || dst_buffer < 0 || dst_buffer > 2)
    return AMRVAC_E_INVALID;
  const amrvac_config &a = src->cfg, &c = dst->cfg;
  if (a.ndim != c.ndim || a.precision != c.precision || src->ninst != dst->ninst)
    return AMRVAC_E_INVALID;
  const int nd = a.ndim;
  for (int d = 0; d < nd; d++)
    if (a.block_nx[d] != c.block_nx[d] || (c.block_nx[d] & 1) || a.bc[d][0] != c.bc[d][0] ||
        a.bc[d][1] != c.bc[d][1])
      return AMRVAC_E_INVALID;
  for (int q = 0; q < src->ninst; q++)
    for (int d = 0; d < nd; d++)
      if (src->inst[q].base_blocks[d] != dst->inst[q].base_blocks[d]) return AMRVAC_E_INVALID;
  // the source blocks by key (hashed: the table is built on the host for every
  // transfer, tens of thousands of lookups for a C4-size mesh)
  std::unordered_map<Key, int, KeyHash> old;
  old.reserve(2 * (size_t)src->nblocks);
  for (int b = 0; b < src->nblocks; b++) {
    const int32_t* r = &src->meta[5 * b];
    old[Key{r[0], r[1], r[2], nd > 1 ? r[3] : 0, nd > 2 ? r[4] : 0}] = b;
  }
  std::vector<int> tab((size_t)dst->nblocks * RTAB_N, -1);
  for (int b = 0; b < dst->nblocks; b++) {
    const int32_t* r = &dst->meta[5 * b];
    const Key k{r[0], r[1], r[2], nd > 1 ? r[3] : 0, nd > 2 ? r[4] : 0};
    int* t = &tab[(size_t)b * RTAB_N];
    auto it = old.find(k);
    if (it != old.end()) {
      t[0] = 0;
      t[1] = it->second;
      continue;
    }
    if (k[1] > 0) {
      it = old.find(Key{k[0], k[1] - 1, k[2] >> 1, k[3] >> 1, k[4] >> 1});
      if (it != old.end()) {
        t[0] = 1;
        t[1] = it->second;
        continue;
      }
    }
    t[0] = 2;
    for (int oz = 0; oz < (nd > 2 ? 2 : 1); oz++)
      for (int oy = 0; oy < (nd > 1 ? 2 : 1); oy++)
        for (int ox = 0; ox < 2; ox++) {
          it = old.find(Key{k[0], k[1] + 1, 2 * k[2] + ox, nd > 1 ? 2 * k[3] + oy : 0,
                            nd > 2 ? 2 * k[4] + oz : 0});
          if (it == old.end()) return AMRVAC_E_INVALID;
          t[2 + (oz * 2 + oy) * 2 + ox] = it->second;
        }
    t[1] = t[2];
  }
  // the transfer runs on dst's stream after the work already on src's
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return AMRVAC_E_CUDA;
  cudaError_t e = cudaEventRecord(ev, src->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->stream, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return AMRVAC_E_CUDA;
  if (cudaMemcpyAsync(dst->d_rtab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice,
                      dst->stream) != cudaSuccess)
    return AMRVAC_E_CUDA;
  const int g = grid_for(dst->nblocks);
  // kept blocks: 16-byte elements where every run of cells starts on a
  // 16-byte boundary (the registers are 256-byte aligned), else scalars
  const size_t rs = c.precision == AMRVAC_FP64 ? 8 : 4;
  const size_t run = (size_t)dst->ncell * rs;
  const int gc = 152 * 8;
  const void* us = src->U[src_buffer];
  void* ud = dst->U[dst_buffer];
  if (run % 16 == 0 && ((uintptr_t)us % 16) == 0 && ((uintptr_t)ud % 16) == 0) {
    const int nw = (int)(run / 16);
    k_regrid_copy<float4><<<gc, 256, 0, dst->stream>>>(
        (const float4*)us, (float4*)ud, dst->d_rtab, dst->nblocks, (size_t)src->nblocks * nw,
        (size_t)dst->nblocks * nw, nw);
  } else if (c.precision == AMRVAC_FP64) {
    k_regrid_copy<double><<<gc, 256, 0, dst->stream>>>(
        (const double*)us, (double*)ud, dst->d_rtab, dst->nblocks,
        (size_t)src->nblocks * src->ncell, (size_t)dst->nblocks * dst->ncell, dst->ncell);
  } else {
    k_regrid_copy<float><<<gc, 256, 0, dst->stream>>>(
        (const float*)us, (float*)ud, dst->d_rtab, dst->nblocks,
        (size_t)src->nblocks * src->ncell, (size_t)dst->nblocks * dst->ncell, dst->ncell);
  }
  if (c.precision == AMRVAC_FP64) {
    k_regrid_restrict<double><<<g, 256, 0, dst->stream>>>(
        src->mesh, (const double*)src->U[src_buffer], dst->mesh, (double*)dst->U[dst_buffer],
        dst->d_rtab);
    k_regrid_transfer<double><<<g, 256, 0, dst->stream>>>(
        src->mesh, (const double*)src->U[src_buffer], dst->mesh, (double*)dst->U[dst_buffer],
        dst->d_rtab);
  } else {
    k_regrid_restrict<float><<<g, 256, 0, dst->stream>>>(
        src->mesh, (const float*)src->U[src_buffer], dst->mesh, (float*)dst->U[dst_buffer],
        dst->d_rtab);
    k_regrid_transfer<float><<<g, 256, 0, dst->stream>>>(
        src->mesh, (const float*)src->U[src_buffer], dst->mesh, (float*)dst->U[dst_buffer],
        dst->d_rtab);
  }
  if (cudaPeekAtLastError() != cudaSuccess) return AMRVAC_E_CUDA;
  dst->launches += 3;
  // the host table must outlive the asynchronous upload
  if (cudaStreamSynchronize(dst->stream) != cudaSuccess) return AMRVAC_E_CUDA;
  return AMRVAC_OK;
}

// --------------------------------------------------------------------------
// The regrid plan on the device.  The same rules as amrvac_regrid_plan, as
// data-parallel passes over the leaves of the state's mesh:
//   1. splits: the flagged leaves; then, to a fixed point, every leaf coarser
//      than a splitting leaf and touching it (faces, edges, corners, periodic
//      wrap) splits too (one pass per launch, the host repeats while a pass
//      changed something);
//   2. merges: a family of 2^ndim sibling leaves all flagged -1 and none
//      splitting merges unless, after the splits, a leaf two levels finer
//      than the parent touches it.  In the sequential rule (families in
//      increasing (instance, level, k, j, i) order of the parent) that test
//      can change only through merges of finer families, which come later, so
//      every family is decided independently here;
//   3. the new leaves are marked in dense per-(instance, level) maps, and a
//      prefix sum over the maps in (instance, level, k, j, i) order numbers
//      them: the new block list in the order amrvac_regrid_plan returns.
namespace amrvac {
namespace {

enum { FATE_KEEP = 0, FATE_SPLIT = 1, FATE_MERGE_FIRST = 2, FATE_MERGE_AWAY = 3 };

__device__ __forceinline__ int plan_nb(const DevMesh& M, int q, int L, int d) {
  return M.lnb[(q * MAXLEV + L) * 3 + d];
}

// position p + o at level L of instance q, wrapped on periodic dimensions;
// false outside the others
__device__ __forceinline__ bool plan_step(const DevMesh& M, int q, int L, const int* p,
                                          const int* o, int* r) {
  for (int d = 0; d < 3; d++) {
    r[d] = d < M.ndim ? p[d] + o[d] : 0;
    if (d >= M.ndim) continue;
    const int n = plan_nb(M, q, L, d);
    if (r[d] < 0 || r[d] >= n) {
      if (M.bc[d][0] != AMRVAC_BC_PERIODIC) return false;
      r[d] = ((r[d] % n) + n) % n;
    }
  }
  return true;
}

__device__ __forceinline__ int plan_map(const DevMesh& M, int q, int L, const int* p) {
  return M.lmap[M.lmap_off[q * MAXLEV + L] +
                ((size_t)p[2] * plan_nb(M, q, L, 1) + p[1]) * plan_nb(M, q, L, 0) + p[0]];
}

// leaf covering level-L position p at level L or coarser (its level in *lev),
// -1 when finer leaves cover p
__device__ __forceinline__ int plan_covering(const DevMesh& M, int q, int L, const int* p0,
                                             int* lev) {
  int p[3] = {p0[0], p0[1], p0[2]};
  for (int LL = L; LL >= 0; LL--) {
    const int code = plan_map(M, q, LL, p);
    if (code >= 0) {
      *lev = LL;
      return code;
    }
    if (code == MAP_REFINED) return -1;
    for (int d = 0; d < 3; d++) p[d] >>= 1;
  }
  return -1;
}

// the 3^ndim - 1 offsets around a position
__device__ __forceinline__ bool plan_offset(const DevMesh& M, int t, int* o) {
  o[0] = t % 3 - 1;
  o[1] = M.ndim > 1 ? (t / 3) % 3 - 1 : 0;
  o[2] = M.ndim > 2 ? t / 9 - 1 : 0;
  return !(o[0] == 0 && o[1] == 0 && o[2] == 0);
}

__global__ void k_plan_init(DevMesh M, const signed char* __restrict__ flags, PlanScratch P) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < M.nblocks; b += gridDim.x * blockDim.x) {
    const int split = flags[b] == 1;
    if (split && M.blk[b * 5 + 1] + 1 >= MAXLEV) P.scal[2] = 1;  // no level to split into
    P.ref[b] = split;
  }
}

// one pass of the 2:1 closure of the splits
__global__ void k_plan_close(DevMesh M, PlanScratch P) {
  const int nt = M.ndim == 3 ? 27 : (M.ndim == 2 ? 9 : 3);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < M.nblocks; b += gridDim.x * blockDim.x) {
    if (!P.ref[b]) continue;
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const int p[3] = {M.blk[b * 5 + 2], M.blk[b * 5 + 3], M.blk[b * 5 + 4]};
    for (int t = 0; t < nt; t++) {
      int o[3], r[3];
      if (!plan_offset(M, t, o) || !plan_step(M, q, L, p, o, r)) continue;
      int lev = 0;
      const int c = plan_covering(M, q, L, r, &lev);
      if (c >= 0 && lev < L && !P.ref[c]) {
        P.ref[c] = 1;
        P.scal[0] = 1;
      }
    }
  }
}

__global__ void k_plan_fate(DevMesh M, PlanScratch P) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < M.nblocks; b += gridDim.x * blockDim.x)
    P.fate[b] = P.ref[b] ? FATE_SPLIT : FATE_KEEP;
}

// merges, decided by the family's first child (all offsets 0)
__global__ void k_plan_merge(DevMesh M, const signed char* __restrict__ flags, PlanScratch P) {
  const int nt = M.ndim == 3 ? 27 : (M.ndim == 2 ? 9 : 3);
  const int nk = 1 << M.ndim;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < M.nblocks; b += gridDim.x * blockDim.x) {
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const int p[3] = {M.blk[b * 5 + 2], M.blk[b * 5 + 3], M.blk[b * 5 + 4]};
    if (flags[b] != -1 || P.ref[b] || L == 0) continue;
    if ((p[0] & 1) || (p[1] & 1) || (p[2] & 1)) continue;  // not the first child
    int kids[8];
    bool ok = true;
    for (int c = 0; c < nk && ok; c++) {
      const int cp[3] = {p[0] + (c & 1), p[1] + ((c >> 1) & 1), p[2] + ((c >> 2) & 1)};
      const int s = plan_map(M, q, L, cp);
      ok = s >= 0 && flags[s] == -1 && !P.ref[s];
      kids[c] = s;
    }
    if (!ok) continue;
    // no leaf two levels finer than the parent around it, after the splits:
    // every level-L position inside the parent's neighbours must be a leaf of
    // level L that does not split, or covered by a coarser leaf
    const int pp[3] = {p[0] >> 1, p[1] >> 1, p[2] >> 1};
    for (int t = 0; t < nt && ok; t++) {
      int o[3], r[3];
      if (!plan_offset(M, t, o) || !plan_step(M, q, L - 1, pp, o, r)) continue;
      for (int c = 0; c < nk && ok; c++) {
        const int cp[3] = {2 * r[0] + (c & 1), M.ndim > 1 ? 2 * r[1] + ((c >> 1) & 1) : 0,
                           M.ndim > 2 ? 2 * r[2] + ((c >> 2) & 1) : 0};
        const int code = plan_map(M, q, L, cp);
        if (code == MAP_REFINED || (code >= 0 && P.ref[code])) ok = false;
      }
    }
    if (!ok) continue;
    P.fate[b] = FATE_MERGE_FIRST;
    for (int c = 1; c < nk; c++) P.fate[kids[c]] = FATE_MERGE_AWAY;
  }
}

__device__ __forceinline__ void plan_mark(const DevMesh& M, const PlanScratch& P, int q, int L,
                                          const int* p) {
  const int n0 = plan_nb(M, q, L, 0), n1 = plan_nb(M, q, L, 1);
  P.map[(size_t)P.seg[q * MAXLEV + L] + ((size_t)p[2] * n1 + p[1]) * n0 + p[0]] = 1;
}

__global__ void k_plan_mark(DevMesh M, PlanScratch P) {
  const int nk = 1 << M.ndim;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < M.nblocks; b += gridDim.x * blockDim.x) {
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const int p[3] = {M.blk[b * 5 + 2], M.blk[b * 5 + 3], M.blk[b * 5 + 4]};
    const int f = P.fate[b];
    if (f == FATE_KEEP) {
      plan_mark(M, P, q, L, p);
    } else if (f == FATE_SPLIT) {
      for (int c = 0; c < nk; c++) {
        const int cp[3] = {2 * p[0] + (c & 1), M.ndim > 1 ? 2 * p[1] + ((c >> 1) & 1) : 0,
                           M.ndim > 2 ? 2 * p[2] + ((c >> 2) & 1) : 0};
        plan_mark(M, P, q, L + 1, cp);
      }
    } else if (f == FATE_MERGE_FIRST) {
      const int pp[3] = {p[0] >> 1, p[1] >> 1, p[2] >> 1};
      plan_mark(M, P, q, L - 1, pp);
    }
  }
}

// block-wide exclusive prefix sum of one int per thread (blockDim 256)
__device__ __forceinline__ int plan_block_scan(int v, int* total) {
  __shared__ int ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < 8; w++) {
      const int t = ws[w];
      ws[w] = acc;
      acc += t;
    }
    *total = acc;
  }
  __syncthreads();
  const int r = x - v + ws[warp];
  __syncthreads();
  return r;
}

// per-CTA counts of new leaves over contiguous chunks of the maps
__global__ void __launch_bounds__(256) k_plan_count(PlanScratch P, int chunk) {
  __shared__ int red[8];
  const size_t lo = (size_t)blockIdx.x * chunk;
  const size_t hi = lo + chunk < (size_t)P.nmap ? lo + chunk : (size_t)P.nmap;
  int n = 0;
  for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) n += P.map[e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; w++) t += red[w];
    P.sums[blockIdx.x] = t;
  }
}

// exclusive prefix of the CTA counts (one thread: at most PLAN_CTAS entries)
__global__ void k_plan_prefix(PlanScratch P, int nctas) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int c = 0; c < nctas; c++) {
    const int t = P.sums[c];
    P.sums[c] = acc;
    acc += t;
  }
  P.sums[nctas] = acc;
  P.scal[1] = acc;
}

// each new leaf's index = its CTA's prefix + the running count inside the
// chunk; writes (instance, level, i, j, k)
__global__ void __launch_bounds__(256) k_plan_emit(DevMesh M, PlanScratch P, int chunk,
                                                   int nseg) {
  const size_t lo = (size_t)blockIdx.x * chunk;
  const size_t hi = lo + chunk < (size_t)P.nmap ? lo + chunk : (size_t)P.nmap;
  int base = P.sums[blockIdx.x];
  for (size_t e0 = lo; e0 < hi; e0 += blockDim.x) {
    const size_t e = e0 + threadIdx.x;
    const int v = e < hi ? P.map[e] : 0;
    int tot = 0;
    const int at = base + plan_block_scan(v, &tot);
    __shared__ int stot;
    if (threadIdx.x == 0) stot = tot;
    __syncthreads();
    if (v && at < P.cap) {
      // segment (instance, level) of entry e: the last offset <= e
      int a = 0, z = nseg - 1;
      while (a < z) {
        const int m = (a + z + 1) >> 1;
        if ((size_t)P.seg[m] <= e) a = m;
        else z = m - 1;
      }
      const int q = a / MAXLEV, L = a % MAXLEV;
      const int pos = (int)(e - (size_t)P.seg[a]);
      const int n0 = plan_nb(M, q, L, 0), n1 = plan_nb(M, q, L, 1);
      int* o = P.out + (size_t)at * 5;
      o[0] = q;
      o[1] = L;
      o[2] = pos % n0;
      o[3] = M.ndim > 1 ? (pos / n0) % n1 : 0;
      o[4] = M.ndim > 2 ? pos / (n0 * n1) : 0;
    }
    base += stot;
    __syncthreads();
  }
}

}  // namespace
}  // namespace amrvac

extern "C" amrvac_status amrvac_regrid_plan_device(amrvac_state* s, const int8_t* h_flags,
                                                   int32_t capacity, int32_t* h_new_meta,
                                                   int32_t* h_new_nblocks) {
  using namespace amrvac;
  if (!s || !h_new_nblocks || capacity < 0 || (capacity > 0 && !h_new_meta))
    return AMRVAC_E_INVALID;
  PlanScratch& P = s->plan;
  if (P.nmap < 0) return AMRVAC_E_INVALID;  // the dense maps of this mesh would be too large
  cudaStream_t st = s->stream;
  if (h_flags) {
    for (int b = 0; b < s->nblocks; b++)
      if (h_flags[b] < -1 || h_flags[b] > 1) return AMRVAC_E_INVALID;
    if (cudaMemcpyAsync(s->d_eflags, h_flags, (size_t)s->nblocks, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return AMRVAC_E_CUDA;
  }
  const DevMesh& M = s->mesh;
  const int nb = s->nblocks;
  const int grid = (nb + 255) / 256 < 152 * 8 ? (nb + 255) / 256 : 152 * 8;
  int launches = 0;
  if (cudaMemsetAsync(P.scal, 0, sizeof(int) * 4, st) != cudaSuccess ||
      cudaMemsetAsync(P.map, 0, sizeof(int) * ((size_t)P.nmap + 1), st) != cudaSuccess)
    return AMRVAC_E_CUDA;
  k_plan_init<<<grid, 256, 0, st>>>(M, s->d_eflags, P);
  launches++;
  // 2:1 closure: at most one level coarser per pass, so at most MAXLEV passes
  for (int pass = 0; pass < MAXLEV + 1; pass++) {
    k_plan_close<<<grid, 256, 0, st>>>(M, P);
    launches++;
    int changed = 0;
    if (cudaMemcpyAsync(&changed, P.scal, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return AMRVAC_E_CUDA;
    if (!changed) break;
    if (cudaMemsetAsync(P.scal, 0, sizeof(int), st) != cudaSuccess) return AMRVAC_E_CUDA;
  }
  k_plan_fate<<<grid, 256, 0, st>>>(M, P);
  k_plan_merge<<<grid, 256, 0, st>>>(M, s->d_eflags, P);
  k_plan_mark<<<grid, 256, 0, st>>>(M, P);
  const int chunk = (P.nmap + PLAN_CTAS - 1) / PLAN_CTAS > 256
                        ? (P.nmap + PLAN_CTAS - 1) / PLAN_CTAS
                        : 256;
  const int nctas = (P.nmap + chunk - 1) / chunk > 0 ? (P.nmap + chunk - 1) / chunk : 1;
  k_plan_count<<<nctas, 256, 0, st>>>(P, chunk);
  k_plan_prefix<<<1, 32, 0, st>>>(P, nctas);
  k_plan_emit<<<nctas, 256, 0, st>>>(M, P, chunk, s->ninst * MAXLEV);
  launches += 6;
  if (cudaPeekAtLastError() != cudaSuccess) return AMRVAC_E_CUDA;
  s->launches += launches;
  int scal[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(scal, P.scal, sizeof(scal), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return AMRVAC_E_CUDA;
  if (scal[2]) return AMRVAC_E_INVALID;  // a flagged leaf at the deepest level
  *h_new_nblocks = scal[1];
  if (capacity < scal[1] || scal[1] > P.cap) return AMRVAC_E_INVALID;
  if (scal[1] > 0 &&
      (cudaMemcpyAsync(h_new_meta, P.out, sizeof(int) * 5 * (size_t)scal[1],
                       cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return AMRVAC_E_CUDA;
  return AMRVAC_OK;
}
