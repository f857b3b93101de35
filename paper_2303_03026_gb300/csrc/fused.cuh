// Fused persistent stage kernels for 16x16x16 (3D, here) and 16x16 (2D,
// fused2d.cuh) blocks.
//
// One CTA of 272 threads owns one block at a time and loops over the work
// list (grid = resident CTAs).  Thread (x, y) < 256 owns a column of the block;
// 16 helper threads take the 32 faces on the +x/+y block boundary.
//   3D: march over z with a ring of 2G primitive planes in shared memory,
//       each with its G-cell x/y halo (G = 2 ghost layers: 4 planes of 20 x
//       20, 128 halo cells a plane; G = 3 for the five-point limiters: 6
//       planes of 22 x 22, 192 halo cells).  Iteration z:
//         cp.async copies of plane z+G (own column; threads 0 .. 64G-1: one
//           x/y halo cell each):
//           same-level neighbour, outflow clamp or the ghost slab of a
//           level-change face (built before the launch by k_ghost_slabs);
//           for stages k > 0 also U0 of the owner's cell of plane z;
//         x- and y-face fluxes of plane z into shared memory (double-buffered
//           by plane parity);
//         wait for the copies, conserved -> primitive in place of the own
//           cells of plane z+G and (owners 256-64G .. 255, one cell each) of
//           the halo of plane z+1 (float-float or fp64 pressure for FP32 bulk);
//         the z-face z+1/2 flux of the thread's own column (registers);
//         one barrier; update of cell (x, y, z): flux divergence with the
//           z-face flux carried from the previous plane, psi damping, SSPRK
//           combination; in the last stage the CFL terms of the new state
//           (reduced per block for the time step).
//   2D: k_fused2d (fused2d.cuh), pipelined over blocks instead of planes.
// Every face flux of the block is computed once (block-boundary faces are
// computed by both neighbours).  Arithmetic follows physics.cuh.
#pragma once

#include "ghost.cuh"
#include "physics.cuh"
#include "physics_f2.cuh"
#include "reduce.cuh"
#include "state.hpp"

namespace amrvac {

constexpr int FB = 16;          // block edge handled by the fused kernel
// threads per CTA: 256 column owners (x- and y-face of their cell, z-face of
// their column, their cell's update; with two ghost layers owners 0..127 also
// copy in and owners 128..255 convert one of the 128 x/y halo cells of each
// plane, with three owners 0..191 and 64..255 share the 192) and 16 helpers
// (the 32 faces on the +x/+y block boundary).  The 2D kernel uses the same
// roles with threads 0 .. 64G-1 copying and converting the halo.
constexpr int FT = FB * FB + FB;
constexpr int FXW = 20;           // row stride of the face-flux arrays

// ghost layers of a tile for a limiter template value (-2: the five-point
// limiters, chosen at run time)
__host__ __device__ constexpr int tile_ghosts(int lim) { return lim == -2 ? NG5 : NG; }

// Thread (x, y) of a warp: lanes 0-15 take row r, lanes 16-31 row r + 4, so the
// two half-warps of a row-stride-20 array fall on disjoint banks (4*20 = 16 mod 32;
// the 22-wide planes of the five-point ring overlap in 8 banks).
__device__ __forceinline__ int fused_row(int warp, int lane) {
  return (warp & 3) + (warp >> 2) * 8 + (lane >> 4) * 4;
}

// DEEP: the one-CTA-per-SM layout (face pairs), with room for a 6-plane ring
// (planes land one iteration before they are converted) and three U0 slots.
// G: ghost layers; a plane is (16 + 2G)^2 (row stride 20 or 22) and the ring
// holds the 2G planes of a z stencil
template <class T, int DIM, bool DEEP = false, int G = NG> struct FusedSmem {
  static_assert(!DEEP || G == NG, "the deep ring takes two ghost layers");
  static constexpr int PW = FB + 2 * G;
  static constexpr int NSLOT = DIM == 3 ? (DEEP ? 6 : 2 * G) : 1;
  static constexpr int NU0 = DEEP ? 3 : 1;
  T plane[NSLOT][NV][PW][PW];
  // face fluxes of the current plane, double-buffered by plane parity so that
  // one barrier per plane separates writers and readers
  T fx[2][NV][FB][FXW];       // x faces: column i = face i - 1/2, i = 0..16
  T fy[2][NV][FB + 1][FXW];   // y faces: row j = face j - 1/2
  // float path: U0 of the owners' cells of the current plane (and, DEEP, of
  // the next two), copied in ahead of the update (the fp64 path reads U0
  // directly: a double slot would not fit beside its planes)
  T u0[NU0][sizeof(T) == 4 ? NV : 1][FB * FB];
  double red[8][NPART];
  int next;
};

// asynchronous global -> shared copy of one element (Ampere+ cp.async; the
// issuing thread waits with cp_async_wait_all before reading the data)
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(gmem_src),
               "n"(sizeof(T)));
}
// the same, ordered after this thread's earlier shared-memory reads of the
// destination (the copy overwrites values the thread read one plane before)
template <class T>
__device__ __forceinline__ void cp_async_elem_after_reads(T* smem_dst, const T* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(gmem_src),
               "n"(sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// deterministic CTA reduction of the owners' partials (warps 0..7; the partial
// helper warp only joins the barriers); thread 0..NPART-1 store part_b
__device__ __forceinline__ void cta_reduce_store(double (*red)[NPART], Partial& p, bool owner,
                                                 double* part_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (owner) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p.smax = fmax(p.smax, __shfl_xor_sync(0xffffffffu, p.smax, o));
      p.chm = fmax(p.chm, __shfl_xor_sync(0xffffffffu, p.chm, o));
#pragma unroll
      for (int v = 0; v < NV; v++) p.sum[v] += __shfl_xor_sync(0xffffffffu, p.sum[v], o);
    }
    if (lane == 0) {
      red[warp][0] = p.smax;
      red[warp][1] = p.chm;
#pragma unroll
      for (int v = 0; v < NV; v++) red[warp][2 + v] = p.sum[v];
    }
  }
  __syncthreads();
  if (threadIdx.x < NPART) {
    double acc = red[0][threadIdx.x];
    for (int w = 1; w < 8; w++) {
      double x = red[w][threadIdx.x];
      acc = threadIdx.x < 2 ? fmax(acc, x) : acc + x;
    }
    part_b[threadIdx.x] = threadIdx.x < 2 + NV ? acc : 0.0;
  }
  __syncthreads();
}

// CTA maximum of the owners' two CFL terms into part_b[0], part_b[1]
__device__ __forceinline__ void cta_reduce_max2(double (*red)[NPART], double smax, double cmax,
                                                bool owner, double* part_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (owner) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    if (lane == 0) {
      red[warp][0] = smax;
      red[warp][1] = cmax;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double acc = red[0][threadIdx.x];
    for (int w = 1; w < 8; w++) acc = fmax(acc, red[w][threadIdx.x]);
    part_b[threadIdx.x] = acc;
  }
}

// CFL terms of a conserved cell: running max of sum_d (|v_d| + c_f,d)/dx_d and
// of |v_d| + c_f,d.  The fast speed of each direction is the cancellation-free
// form with 1/rho, a^2 = gamma p/rho and b^2 = B^2/rho shared by the
// directions (b_t^2 = b^2 - B_d^2/rho, kept >= 0).
template <class T, int DIM>
__device__ __forceinline__ void cfl_terms(const T* u, double gammad, T g, bool ff, float gm1f,
                                          const T* idx, T& smx, T& cmx) {
  T w[NV];
  cons2prim(gammad, u, w, ff, gm1f);
  const T ir = T(1) / w[0];
  const T a2 = g * w[4] * ir;
  const T bb = (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]) * ir;
  const T dd = a2 - bb, sab = a2 + bb;
  T s = T(0);
#pragma unroll
  for (int d = 0; d < DIM; d++) {
    const T bt2 = fmax(bb - w[5 + d] * w[5 + d] * ir, T(0));  // no negative rounding
    const T cf = sqrt(T(0.5) * (sab + sqrt(dd * dd + T(4) * a2 * bt2)));
    const T spd = fabs(w[1 + d]) + cf;
    s += spd * idx[d];
    cmx = fmax(cmx, spd);
  }
  smx = fmax(smx, s);
}

// refluxing: the flux f of cell `idx` of level-change face `face` of the block
// into that face's register (nb code -3 - slab index)
template <class T>
__device__ __forceinline__ void keep_face_flux(const DevMesh& M, int code, int idx, const T* f) {
  T* reg = (T*)M.fluxreg + (size_t)(-3 - code) * NV * M.farea + idx;
#pragma unroll
  for (int v = 0; v < NV; v++) reg[(size_t)v * M.farea] = f[v];
}

// the instantiations that can compute the x and y faces of a cell together in
// the two float2 lanes (stencil_flux_xy): FP32 vanleer + HLLD, lean.  16% fewer
// instructions, but ~160 registers, hence one CTA per SM; a tuning choice
// (amrvac_tuning.faces)
template <class T, int LIM, int FLUX, bool FULL> constexpr bool xy_pair_ok() {
  return sizeof(T) == 4 && LIM == AMRVAC_LIM_VANLEER && FLUX == AMRVAC_FLUX_HLLD && !FULL;
}

template <class T> __device__ __forceinline__ T over_dx(T a, T dx, T idx);
template <> __device__ __forceinline__ double over_dx(double a, double dx, double) { return a / dx; }
template <> __device__ __forceinline__ float over_dx(float a, float, float idx) { return a * idx; }

// face flux from a 4-cell stencil accessor S(v, t), t = 0..3 for cells
// f-2, f-1, f, f+1 around the face f-1/2; LIM < 0: runtime limiter lim
template <class T, int D, int LIM, int FLUX, class Acc>
__device__ __forceinline__ void stencil_flux(Acc S, int glm, T g, T ch, T* f, int lim) {
  if constexpr (sizeof(T) == 4) {
    // FP32 bulk: left/right states packed in float2 lanes (physics_f2.cuh)
    stencil_flux_f2<D, LIM, FLUX>(S, glm, g, ch, f, lim);
    return;
  }
  const int L = LIM >= 0 ? LIM : lim;
  T wl[NV], wr[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    T a = S(v, 0), b = S(v, 1), c = S(v, 2), e = S(v, 3);
    wl[v] = recon_plus<T>(L, a, b, c);
    wr[v] = recon_minus<T>(L, b, c, e);
  }
  if (!(wl[0] > T(0)) || !(wl[4] > T(0)) || !(wr[0] > T(0)) || !(wr[4] > T(0))) {
#pragma unroll
    for (int v = 0; v < NV; v++) {
      wl[v] = S(v, 1);
      wr[v] = S(v, 2);
    }
  }
  face_flux_d<T, D>(FLUX, glm, g, ch, wl, wr, f);
}

// face flux from the six-cell stencil S(v, t), t = 0..5 for cells f-3 .. f+2
// around the face f-1/2, with a five-point limiter lim (lam: wenozp5's lambda)
template <class T, int D, int FLUX, class Acc>
__device__ __forceinline__ void stencil_flux5(Acc S, int lim, T lam, int glm, T g, T ch, T* f) {
  if constexpr (sizeof(T) == 4) {
    stencil_flux5_f2<D, FLUX>(S, lim, lam, glm, g, ch, f);
  } else {
    T wl[NV], wr[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const T c[6] = {S(v, 0), S(v, 1), S(v, 2), S(v, 3), S(v, 4), S(v, 5)};
      wl[v] = recon5_plus<T>(lim, c, lam);
      wr[v] = recon5_minus<T>(lim, c + 1, lam);
    }
    if (!(wl[0] > T(0)) || !(wl[4] > T(0)) || !(wr[0] > T(0)) || !(wr[4] > T(0))) {
#pragma unroll
      for (int v = 0; v < NV; v++) {
        wl[v] = S(v, 2);
        wr[v] = S(v, 3);
      }
    }
    face_flux_d<T, D>(FLUX, glm, g, ch, wl, wr, f);
  }
}

// Ghost values of every level-change face of the mesh, from the stage input
// Uk: restriction (mean of the finer children) where the neighbour is finer,
// prolongation (coarse value plus minmod-limited slopes times +-1/4, slopes
// computed once per coarse cell) where it is coarser.  One CTA per face at a
// time; slab gi belongs to face glist[gi] = block * 6 + face and holds
// [v][layer][t2][t1], layer = ghost index along the normal from the low end
// (G layers: cells -G .. -1 on a low face, 16 .. 15 + G on a high face; the
// G fine layers lie in G/2 rounded up coarse layers).
template <class T, int DIM, int G = NG>
__global__ void __launch_bounds__(256)
    k_ghost_slabs(DevMesh M, const T* __restrict__ Uk, T* __restrict__ gslab,
                  const int* __restrict__ glist, int ngen) {
  constexpr int NT2 = DIM == 3 ? FB : 1;
  constexpr int SLAB_FACE = NV * G * FB * NT2;
  constexpr int NC2 = DIM == 3 ? FB / 2 : 1;
  constexpr int NCL = (G + 1) / 2;  // coarse layers (1 or 2)
  __shared__ T cs[NCL * (FB / 2) * NC2 * (1 + DIM) * NV];  // [cl][coarse cell][value, slopes][v]
  const int tid = threadIdx.x;
  const size_t vs = (size_t)M.nblocks * M.ncell;
  for (int gi = blockIdx.x; gi < ngen; gi += gridDim.x) {
    const int b = glist[gi] / 6, f = glist[gi] % 6;
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const int bidx[3] = {M.blk[b * 5 + 2], M.blk[b * 5 + 3], M.blk[b * 5 + 4]};
    const int d = f >> 1, side = f & 1;
    // global level-L index of ghost (layer, t1, t2) of this face
    auto ghost_p = [&](int layer, int t1, int t2, int* p) {
      int loc[3];
      const int n = side ? FB + layer : layer - G;
      if (d == 0) { loc[0] = n; loc[1] = t1; loc[2] = t2; }
      else if (d == 1) { loc[0] = t1; loc[1] = n; loc[2] = t2; }
      else { loc[0] = t1; loc[1] = t2; loc[2] = n; }
#pragma unroll
      for (int e = 0; e < 3; e++) p[e] = e < DIM ? bidx[e] * FB + loc[e] : 0;
      wrap_level(M, q, L, p);
    };
    int pn[3];
    ghost_p(0, 0, 0, pn);
    int cell;
    const int code = map_at(M, q, L, pn, &cell);
    T* sf = gslab + (size_t)gi * SLAB_FACE;
    if (code == MAP_REFINED) {
      // restriction: mean of the finer children
      for (int e = tid; e < G * FB * NT2; e += blockDim.x) {
        const int t1 = e % FB, t2 = (e / FB) % NT2, layer = e / (FB * NT2);
        int p[3];
        ghost_p(layer, t1, t2, p);
        T u[NV];
        level_value_down(M, Uk, vs, q, L, p, u);
#pragma unroll
        for (int v = 0; v < NV; v++) sf[((v * G + layer) * NT2 + t2) * FB + t1] = u[v];
      }
    } else {
      // prolongation: value and minmod slopes once per coarse cell (cl: the
      // coarse layer, counted from the fine layer 0 side) ...
      for (int e = tid; e < NCL * (FB / 2) * NC2 * DIM; e += blockDim.x) {
        const int dd = e % DIM, cc = (e / DIM) % ((FB / 2) * NC2), cl = e / (DIM * (FB / 2) * NC2);
        const int ct1 = cc % (FB / 2), ct2 = cc / (FB / 2);
        int p[3];
        // a fine layer inside coarse layer cl: the low face's fine layers -G..-1
        // start at coarse -(G+1)/2; the high face's 16.. at coarse 8
        const int fl = side ? 2 * cl : (G % 2 ? 2 * cl - 1 : 2 * cl);
        ghost_p(fl < 0 ? 0 : fl, 2 * ct1, 2 * ct2, p);
        int qc[3];
#pragma unroll
        for (int k2 = 0; k2 < 3; k2++) qc[k2] = k2 < DIM ? (p[k2] >> 1) : 0;
        T uc[NV], um[NV], up[NV];
        level_value_down(M, Uk, vs, q, L - 1, qc, uc);
        int qm[3] = {qc[0], qc[1], qc[2]}, qp[3] = {qc[0], qc[1], qc[2]};
        qm[dd] -= 1;
        qp[dd] += 1;
        level_value_down(M, Uk, vs, q, L - 1, qm, um);
        level_value_down(M, Uk, vs, q, L - 1, qp, up);
        const int cb = cl * (FB / 2) * NC2 + cc;  // cache slot
#pragma unroll
        for (int v = 0; v < NV; v++) {
          cs[(cb * (1 + DIM) + 1 + dd) * NV + v] = minmod_g(uc[v] - um[v], up[v] - uc[v]);
          if (dd == 0) cs[(cb * (1 + DIM)) * NV + v] = uc[v];
        }
      }
      __syncthreads();
      // ... then every fine ghost: coarse value + sum_d (+-1/4) slope_d
      for (int e = tid; e < G * FB * NT2; e += blockDim.x) {
        const int t1 = e % FB, t2 = (e / FB) % NT2, layer = e / (FB * NT2);
        int p[3];
        ghost_p(layer, t1, t2, p);
        // coarse layer of this fine layer (see above)
        const int cl = side ? layer / 2 : (layer + (G % 2)) / 2;
        const int cc = cl * (FB / 2) * NC2 + (t2 >> 1) * (FB / 2) + (t1 >> 1);
        const T* c0 = cs + (cc * (1 + DIM)) * NV;
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T val = c0[v];
#pragma unroll
          for (int dd = 0; dd < DIM; dd++) {
            const T wgt = (p[dd] & 1) ? T(0.25) : T(-0.25);
            val = val + wgt * c0[(1 + dd) * NV + v];
          }
          sf[((v * G + layer) * NT2 + t2) * FB + t1] = val;
        }
      }
    }
    __syncthreads();  // cs is reused by the next face
  }
}

// FULL: the SSPRK(5,4) second output, the refluxing face registers and the
// mirrored reads of symmetric walls are compiled in (they are runtime-uniform
// branches that still cost the hot loop registers and scheduling freedom, so
// the lean instantiation runs otherwise)
// PAIR: the x and y faces of a thread's cell share the float2 lanes (one CTA
// per SM: no minimum-occupancy register cap)
// LIM -2: the five-point limiters (runtime limiter, three ghost layers: a
// 6-plane ring of 22 x 22 planes and 192 halo cells a plane, one CTA per SM)
template <class T, int DIM, int LIM, int FLUX, bool FULL, bool PAIR>
__global__ void __launch_bounds__(FT, sizeof(T) == 4 && !PAIR && LIM != -2 ? 2 : 1)
    k_fused(DevMesh M, const T* U0, const T* __restrict__ Uk, const T* U2, T* out, T* out2,
            const int* __restrict__ work, int nwork, const T* __restrict__ gslab,
            int* __restrict__ counter, StageParams sp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  static_assert(DIM == 3, "16x16 blocks in 2D use k_fused2d");
  // the face-pair kernel (one CTA per SM) also takes the deep ring
  constexpr bool DEEP = PAIR;
  constexpr int G = tile_ghosts(LIM);
  using Smem = FusedSmem<T, DIM, DEEP, G>;
  Smem& S = *reinterpret_cast<Smem*>(smraw);
  constexpr int NZ = DIM == 3 ? FB : 1;
  constexpr int NSLOT = Smem::NSLOT;
  constexpr int PW = Smem::PW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x = lane & 15, y = fused_row(warp, lane);
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int ncell = M.ncell;
  const bool ff = sp.pressure_ff != 0;
  constexpr int NT2 = DIM == 3 ? FB : 1;          // second tangential extent of a face
  constexpr int SLAB_FACE = NV * G * FB * NT2;    // one face: [v][layer][t2][t1]
  static_assert(!PAIR || xy_pair_ok<T, LIM, FLUX, FULL>(), "face pairs: FP32 vanleer + HLLD");
  constexpr bool XYPAIR = PAIR;

  const bool owner = tid < FB * FB;
  const int hr = tid - FB * FB;  // helper index 0..15
  // halo cell h (0 .. NH-1) of a plane: x-halo (h < NH/2) then y-halo; owners
  // 0 .. NH-1 copy one each, owners 256-NH .. 255 convert one each
  constexpr int NH = 4 * G * FB;  // 128 or 192
  auto halo_xy = [](int h, int& hx, int& hy) {
    if (h < NH / 2) {
      const int side = h / (G * FB), r = h % (G * FB);
      hy = r / G;
      hx = side ? FB + r % G : -G + r % G;
    } else {
      const int u = h - NH / 2, side = u / (G * FB), r = u % (G * FB);
      hx = r % FB;
      hy = side ? FB + r / FB : -G + r / FB;
    }
  };

  // work distribution: static (CTA i takes items i, i + grid, ...) or dynamic
  // (each CTA draws its next item from a counter the host zeroes per launch)
  auto next_work = [&](int wi) -> int {
    if (!counter) return wi + gridDim.x;
    __syncthreads();
    if (tid == 0) S.next = atomicAdd(counter, 1);
    __syncthreads();
    return S.next;
  };
  for (int wi = counter ? next_work(0) : blockIdx.x; wi < nwork; wi = next_work(wi)) {
    const int b = work[wi];
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const double gammad = M.gamma[q];
    // stage constants of the block's level in the arithmetic type
    const T* lc = level_consts<T>(M) + (q * MAXLEV + L) * LC_N;
    const T g = lc[LC_G];
    const float gm1f = (float)lc[LC_GM1];
    const T rho_floor = sp_val<T>(sp.small_density, sp.small_density_f);
    const T p_floor = sp_val<T>(sp.small_pressure, sp.small_pressure_f);
    const T idd[3] = {lc[LC_IDX], lc[LC_IDX + 1], lc[LC_IDX + 2]};
    T smx = T(0), cmx = T(0);  // CFL terms of the new state (last stage)

    if (lc[LC_SKIP] != T(0)) {
      // finished instance: copied through unchanged
      for (int c = tid; owner && c < ncell; c += FB * FB) {
        T u[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          size_t at = (size_t)v * vs + (size_t)b * ncell + c;
          u[v] = Uk[at];
          out[at] = u[v];
          if (FULL && sp.has2) out2[at] = u[v];
        }
        if (sp.epilogue) cfl_terms<T, DIM>(u, gammad, g, ff, gm1f, idd, smx, cmx);
      }
      if (sp.epilogue) cta_reduce_max2(S.red, smx, cmx, owner, M.part + (size_t)b * NPART);
      continue;
    }

    const T ch = lc[LC_CH], dt = lc[LC_DT];
    const T ca = sp_val<T>(sp.a, sp.af), cb = sp_val<T>(sp.b, sp.bf);
    const T dx0 = lc[LC_DX], dx1 = lc[LC_DX + 1], dx2 = lc[LC_DX + 2];
    const T idx0 = idd[0], idx1 = idd[1], idx2 = idd[2];
    const T damp = lc[LC_DAMP];

    // face neighbour codes; a level-change face reads its ghost slab, built
    // from the stage input by k_ghost_slabs: code -3 - (slab index)
    // (FULL) a symmetric wall reads the block's own mirrored cells: bit f of
    // wmask marks face f, whose code becomes the outflow one
    int nb[6];
    int wmask = 0;
#pragma unroll
    for (int f = 0; f < 6; f++) {
      nb[f] = f < 2 * DIM ? M.nbr[b * 6 + f] : NBR_OUTFLOW;
      if (FULL && nb[f] == NBR_WALL) {  // before slab codes, which reach -5 too
        nb[f] = NBR_OUTFLOW;
        wmask |= 1 << f;
      }
      if (nb[f] == NBR_GENERAL) nb[f] = -3 - M.gface[b * 6 + f];
    }

    // location of the conserved values of block-local cell (i, j, k), at most
    // one index outside: own block, same-level neighbour (wrapped index),
    // outflow clamp (own block) or the face's ghost slab; vstride between vars
    auto locate = [&](int i, int j, int k, const T*& ptr, size_t& vstride) {
      int f = -1, n = 0, t1 = 0, t2 = 0;
      if (i < 0 || i >= FB) { f = i < 0 ? 0 : 1; n = i; t1 = j; t2 = k; }
      else if (j < 0 || j >= FB) { f = j < 0 ? 2 : 3; n = j; t1 = i; t2 = k; }
      else if (DIM == 3 && (k < 0 || k >= FB)) { f = k < 0 ? 4 : 5; n = k; t1 = i; t2 = j; }
      vstride = vs;
      if (f < 0) {
        ptr = Uk + (size_t)b * ncell + (k * FB + j) * FB + i;
        return;
      }
      const int code = nb[f];
      if (code <= -3) {
        const int layer = n < 0 ? n + G : n - FB;
        ptr = gslab + (size_t)(-3 - code) * SLAB_FACE + (layer * NT2 + t2) * FB + t1;
        vstride = G * NT2 * FB;
        return;
      }
      int nn = code >= 0 ? (n < 0 ? n + FB : n - FB) : (n < 0 ? 0 : FB - 1);
      if (FULL && ((wmask >> f) & 1)) nn = n < 0 ? -1 - n : 2 * FB - 1 - n;
      const int src = code >= 0 ? code : b;
      int ii = i, jj = j, kk = k;
      if (f < 2) ii = nn;
      else if (f < 4) jj = nn;
      else kk = nn;
      ptr = Uk + (size_t)src * ncell + (kk * FB + jj) * FB + ii;
    };

    auto to_prim = [&](T* cell, int which, int flip) {
      // cell: the 9 values of one cell in a plane slot (stride PW*PW), in
      // place; flip: (FULL) dimensions whose wall mirrored this cell
      T u[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = cell[v * PW * PW];
      cons2prim(gammad, u, w, ff, gm1f);
      if (FULL && flip) wall_flip(flip, w);
      if (sp.check_small && is_small_prim(w[0], w[4], rho_floor, p_floor))
        latch_error(M.err, AMRVAC_E_SMALL_VALUES, b, tid, which);
#pragma unroll
      for (int v = 0; v < NV; v++) cell[v * PW * PW] = w[v];
    };

    // asynchronous copy of plane pz's conserved values into its ring slot
    // (own column; threads 0..NH-1 also their halo cell of interior planes) ...
    auto issue_plane = [&](int pz) {
      const int slot = ((pz % NSLOT) + NSLOT) % NSLOT;
      const T* ptr;
      size_t st;
      if (owner) {
        locate(x, y, pz, ptr, st);
#pragma unroll
        for (int v = 0; v < NV; v++)
          cp_async_elem(&S.plane[slot][v][y + G][x + G], ptr + v * st);
        if (tid < NH && pz >= 0 && pz < NZ) {
          int hx, hy;
          halo_xy(tid, hx, hy);
          locate(hx, hy, pz, ptr, st);
#pragma unroll
          for (int v = 0; v < NV; v++)
            cp_async_elem(&S.plane[slot][v][hy + G][hx + G], ptr + v * st);
        }
      }
      cp_async_commit();
    };
    // ... once this thread's copies have landed, the owner's in-place
    // conversion of its own cell ...
    auto convert_plane = [&](int pz) {
      const int slot = ((pz % NSLOT) + NSLOT) % NSLOT;
      const int flip = FULL && ((pz < 0 && (wmask & 16)) || (pz >= NZ && (wmask & 32))) ? 4 : 0;
      if (owner) to_prim(&S.plane[slot][0][y + G][x + G], 0, flip);
    };
    // ... and, one barrier after their copies landed, the conversion of the
    // halo cells of plane pz by owners 256-NH..255 (one cell each)
    auto convert_halo = [&](int pz) {
      const int slot = ((pz % NSLOT) + NSLOT) % NSLOT;
      if (tid >= FB * FB - NH && tid < FB * FB) {
        int hx, hy;
        halo_xy(tid - (FB * FB - NH), hx, hy);
        int flip = 0;
        if (FULL) {
          if ((hx < 0 && (wmask & 1)) || (hx >= FB && (wmask & 2))) flip |= 1;
          if ((hy < 0 && (wmask & 4)) || (hy >= FB && (wmask & 8))) flip |= 2;
        }
        to_prim(&S.plane[slot][0][hy + G][hx + G], 1, flip);
      }
    };

    // five-point limiters: WENO-Z+ lambda of the block's level per direction
    const T lam[3] = {G == NG ? T(0) : (T)M.wzlam[(q * MAXLEV + L) * 3],
                      G == NG ? T(0) : (T)M.wzlam[(q * MAXLEV + L) * 3 + 1],
                      G == NG ? T(0) : (T)M.wzlam[(q * MAXLEV + L) * 3 + 2]};
    auto zflux = [&](int zc, T* f) {
      // z face between planes zc-1 and zc of the thread's own column
      if constexpr (G == NG) {
        int s0 = (zc - 2 + 2 * NSLOT) % NSLOT, s1 = (zc - 1 + 2 * NSLOT) % NSLOT;
        int s2 = (zc + 2 * NSLOT) % NSLOT, s3 = (zc + 1 + 2 * NSLOT) % NSLOT;
        auto acc = [&](int v, int t) -> T {
          int s = t == 0 ? s0 : (t == 1 ? s1 : (t == 2 ? s2 : s3));
          return S.plane[s][v][y + NG][x + NG];
        };
        stencil_flux<T, 2, LIM, FLUX>(acc, sp.glm, g, ch, f, sp.limiter);
      } else {
        // planes zc-3 .. zc+2 (the ring holds exactly these six)
        int sl6[6];
#pragma unroll
        for (int t = 0; t < 6; t++) sl6[t] = (zc - 3 + t + 2 * NSLOT) % NSLOT;
        auto acc = [&](int v, int t) -> T { return S.plane[sl6[t]][v][y + G][x + G]; };
        stencil_flux5<T, 2, FLUX>(acc, sp.limiter, lam[2], sp.glm, g, ch, f);
      }
    };

    constexpr bool PRE0 = sizeof(T) == 4;
    const bool pre0 = PRE0 && !sp.plain && owner;
    // U0 of this thread's cell of plane pz into its slot (a DRAM read landing
    // ahead of the update; read back by the same thread only)
    auto issue_u0 = [&](int pz) {
      const T* src = U0 + (size_t)b * ncell + (pz * FB + y) * FB + x;
      T* dst = &S.u0[pz % Smem::NU0][0][tid];
#pragma unroll
      for (int v = 0; v < NV; v++) cp_async_elem_after_reads(dst + v * FB * FB, src + v * vs);
    };

    T fzp[NV];
    if (DEEP && pre0) issue_u0(0);
    for (int pz = -G; pz < G; pz++) issue_plane(pz);
    cp_async_wait_all();
    for (int pz = -G; pz < G; pz++) convert_plane(pz);
    if (owner) zflux(0, fzp);  // own column only
    if (FULL && sp.reflux && owner && nb[4] <= -3) keep_face_flux(M, nb[4], y * FB + x, fzp);
    __syncthreads();  // the halo copies of planes 0 and 1 are visible
    convert_halo(0);
    __syncthreads();  // plane 0 with its halo in primitives
    if constexpr (DEEP) {
      // one plane ahead of the loop: plane 2 and U0 of plane 1 in flight
      if (pre0) issue_u0(1);
      issue_plane(2);
    }


    // One barrier per plane.  Iteration z: issue the copies of U0 of plane z
    // (stages k > 0) and of plane z+G into the slot of plane z-G (its last
    // readers were the faces of plane z-G and this thread's own z face of
    // iteration z-1); x/y faces of plane z into the flux buffer of parity z;
    // wait for and convert the own cells of plane z+G, convert the halo of
    // plane z+1 (owners 256-NH..255); load U_k of the own cell of plane z; z
    // face z+1/2 (planes z+1-G .. z+G); barrier; update of plane z.  The buffer of parity z is rewritten at
    // iteration z+2, after the barrier of iteration z+1, which every thread
    // passes only after its update of plane z.
    // DEEP: the same with the copies one iteration earlier: iteration z issues
    // plane z+3 and U0 of plane z+2 into a 6-plane ring and three U0 slots and
    // waits only for the group of the previous iteration (plane z+2, U0 z+1).
#pragma unroll 1
    for (int z = 0; z < NZ; z++) {
      if constexpr (DEEP) {
        if (pre0 && z + 2 < NZ) issue_u0(z + 2);
        if (z + 3 <= NZ + 1) issue_plane(z + 3);  // commits one group
        else cp_async_commit();                   // an empty group keeps the count
      } else {
        if (pre0) issue_u0(z);
        issue_plane(z + G);  // commits this thread's copies as one group
      }
      const int sl = z % NSLOT, fb = z & 1;
      {
        // owners: the x and y faces on the low side of their cell; helpers: the
        // x face at the +x block boundary of row hr and the y face at the +y
        // boundary of column hr
        const int fxr = owner ? y : hr, fxc = owner ? x : FB;
        const int fyr = owner ? y : FB, fyc = owner ? x : hr;
        T f[NV];
        auto ax = [&](int v, int t) -> T { return S.plane[sl][v][fxr + G][fxc + t]; };
        auto ay = [&](int v, int t) -> T { return S.plane[sl][v][fyr + t][fyc + G]; };
        if constexpr (G == NG5) {
          // five-point limiters: six-cell stencils
          stencil_flux5<T, 0, FLUX>(ax, sp.limiter, lam[0], sp.glm, g, ch, f);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fx[fb][v][fxr][fxc] = f[v];
          if (FULL && sp.reflux) {
            const int face = owner ? (x == 0 ? 0 : -1) : 1;
            if (face >= 0 && nb[face] <= -3) keep_face_flux(M, nb[face], z * FB + fxr, f);
          }
          stencil_flux5<T, 1, FLUX>(ay, sp.limiter, lam[1], sp.glm, g, ch, f);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fy[fb][v][fyr][fyc] = f[v];
          if (FULL && sp.reflux) {
            const int face = owner ? (y == 0 ? 2 : -1) : 3;
            if (face >= 0 && nb[face] <= -3) keep_face_flux(M, nb[face], z * FB + fyc, f);
          }
        } else if constexpr (XYPAIR) {
          // both faces at once, one per float2 lane
          T f2[NV];
          stencil_flux_xy(ax, ay, sp.glm, g, ch, f, f2);
#pragma unroll
          for (int v = 0; v < NV; v++) {
            S.fx[fb][v][fxr][fxc] = f[v];
            S.fy[fb][v][fyr][fyc] = f2[v];
          }
          if (FULL && sp.reflux) {
            const int face = owner ? (x == 0 ? 0 : -1) : 1;
            if (face >= 0 && nb[face] <= -3) keep_face_flux(M, nb[face], z * FB + fxr, f);
            const int facey = owner ? (y == 0 ? 2 : -1) : 3;
            if (facey >= 0 && nb[facey] <= -3) keep_face_flux(M, nb[facey], z * FB + fyc, f2);
          }
        } else {
          stencil_flux<T, 0, LIM, FLUX>(ax, sp.glm, g, ch, f, sp.limiter);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fx[fb][v][fxr][fxc] = f[v];
          if (FULL && sp.reflux) {  // x faces on the block boundary: face 0 (owners x = 0), 1 (helpers)
            const int face = owner ? (x == 0 ? 0 : -1) : 1;
            if (face >= 0 && nb[face] <= -3) keep_face_flux(M, nb[face], z * FB + fxr, f);
          }
          stencil_flux<T, 1, LIM, FLUX>(ay, sp.glm, g, ch, f, sp.limiter);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fy[fb][v][fyr][fyc] = f[v];
          if (FULL && sp.reflux) {  // y faces on the block boundary: face 2 (owners y = 0), 3 (helpers)
            const int face = owner ? (y == 0 ? 2 : -1) : 3;
            if (face >= 0 && nb[face] <= -3) keep_face_flux(M, nb[face], z * FB + fyc, f);
          }
        }
      }
      // owners: own cell of plane z+G -> primitives (needed by the z face
      // below); owners 256-NH..255 also a halo cell of plane z+1, whose copies
      // owners 0..NH-1 waited for before the previous barrier (needed next
      // iteration)
      if constexpr (DEEP) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      else cp_async_wait_all();
      convert_plane(z + G);
      if (z + 1 < NZ) convert_halo(z + 1);
      // float path: the stage input of the own cell, loaded before the z face
      // and the barrier so that its L2 latency overlaps them (the double path
      // has no registers to spare and loads it in the update)
      const int c = (z * FB + y) * FB + x;
      T ukr[PRE0 ? NV : 1];
      if (PRE0 && owner) {
#pragma unroll
        for (int v = 0; v < NV; v++) ukr[v] = Uk[(size_t)v * vs + (size_t)b * ncell + c];
      }
      T fz[NV];
      if (DIM == 3 && owner) zflux(z + 1, fz);
      if (FULL && sp.reflux && owner && z == NZ - 1 && nb[5] <= -3)
        keep_face_flux(M, nb[5], y * FB + x, fz);
      __syncthreads();
      if (!owner) continue;  // helpers: no cell of their own

      T un[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        T acc = over_dx<T>(S.fx[fb][v][y][x + 1] - S.fx[fb][v][y][x], dx0, idx0);
        acc += over_dx<T>(S.fy[fb][v][y + 1][x] - S.fy[fb][v][y][x], dx1, idx1);
        if (DIM == 3) acc += over_dx<T>(fz[v] - fzp[v], dx2, idx2);
        const size_t at = (size_t)v * vs + (size_t)b * ncell + c;
        const T uk = PRE0 ? ukr[PRE0 ? v : 0] : Uk[at];
        T ut = uk - dt * acc;
        if (v == 8) ut = ut * damp;
        un[v] = sp.plain ? ut
                         : ca * (PRE0 ? S.u0[z % Smem::NU0][v][tid] : U0[at]) +
                               cb * ut;
        if (FULL && sp.has2) {
          // SSPRK(5,4) stage 3: w = a2 U2 + b2 (Uk + c2 dt L); U2 is out's
          // register and out2 is U0's, both read above before their writes
          T ut2 = uk - lc[LC_DT2] * acc;
          if (v == 8) ut2 = ut2 * lc[LC_DAMP2];
          out2[at] = sp_val<T>(sp.a2, sp.a2f) * U2[at] + sp_val<T>(sp.b2, sp.b2f) * ut2;
        }
        out[at] = un[v];
      }
      if (sp.epilogue) cfl_terms<T, DIM>(un, gammad, g, ff, gm1f, idd, smx, cmx);
      if (DIM == 3) {
#pragma unroll
        for (int v = 0; v < NV; v++) fzp[v] = fz[v];
      }
    }
    if (sp.epilogue) cta_reduce_max2(S.red, smx, cmx, owner, M.part + (size_t)b * NPART);
  }
}

}  // namespace amrvac

#include "fused2d.cuh"

namespace amrvac {

// ---------------------------------------------------------------- launcher

template <class T, int DIM, int LIM, int FLUX, bool FULL, bool PAIR = false>
static int launch_one(amrvac_state* s, const T* U0, const T* Uk, const T* U2, T* out, T* out2,
                      const int* work, int nwork, int* counter, StageParams sp) {
  static_assert(DIM == 2 || LIM != -2 || sizeof(T) == 4,
                "five-point limiters in 3D: FP32 bulk only (a double 6-plane ring does not fit)");
  auto kern = DIM == 3 ? k_fused<T, 3, LIM, FLUX, FULL, PAIR> : k_fused2d<T, LIM, FLUX, FULL, PAIR>;
  const int smem = DIM == 3 ? (int)sizeof(FusedSmem<T, 3, PAIR, tile_ghosts(LIM)>)
                            : (int)sizeof(Fused2dSmem<T, tile_ghosts(LIM)>);
  static int nsm = 0, per_sm = 0;  // per instantiation, this device
  if (nsm == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return -1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FT, smem);
    if (per_sm < 1) per_sm = 1;
  }
  if (nwork <= 0) return 0;
  int ctas = s->tune.ctas_per_sm > 0 && s->tune.ctas_per_sm < per_sm ? s->tune.ctas_per_sm : per_sm;
  int grid = nsm * ctas;
  if (grid > nwork) grid = nwork;
  if (s->tune.dynamic) {
    if (cudaMemsetAsync(counter, 0, sizeof(int), s->stream) != cudaSuccess) return -1;
  }
  kern<<<grid, FT, smem, s->stream>>>(s->mesh, U0, Uk, U2, out, out2, work, nwork,
                                       (const T*)s->gslab, s->tune.dynamic ? counter : nullptr,
                                       sp);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Stage k for scheme group g (the blocks of the levels sharing this
// limiter and the group's flux); group 0 also launches the per-stage passes
// every group shares: the stage constants and the ghost slabs.
template <class T, int DIM, int LIM>
int launch_fused_l(amrvac_state* s, int k, int epilogue, int g) {
  const StageBuffers sb = stage_buffers(s->cfg.time, k);
  StageParams sp = make_stage_params(s, k, epilogue);
  sp.flux = s->grp_flux[g];
  sp.limiter = s->grp_lim[g];
  const T* U0 = (const T*)s->U[sb.u0];
  const T* Uk = (const T*)s->U[sb.uin];
  const T* U2 = sb.u2 >= 0 ? (const T*)s->U[sb.u2] : nullptr;
  T* out = (T*)s->U[sb.out];
  T* out2 = sb.out2 >= 0 ? (T*)s->U[sb.out2] : nullptr;
  int n = 0;
  if (g == 0) {
    if (launch_level_consts(s, k) < 0) return -1;
    n++;
    if (s->ngen > 0) {
      // ghost slabs of the level-change faces of the stage input (as many
      // layers as the mesh's tiles have ghost cells)
      const int gs = s->ngen < 152 * 8 ? s->ngen : 152 * 8;
      if (s->mesh.ng == NG5)
        k_ghost_slabs<T, DIM, NG5><<<gs, 256, 0, s->stream>>>(s->mesh, Uk, (T*)s->gslab,
                                                               s->d_glist, s->ngen);
      else
        k_ghost_slabs<T, DIM, NG><<<gs, 256, 0, s->stream>>>(s->mesh, Uk, (T*)s->gslab,
                                                              s->d_glist, s->ngen);
      n++;
    }
  }
  const int* work = s->d_work + s->grp_off[g];
  const int nwork = s->grp_cnt[g];
  int* counter = s->d_counter + g;
  bool wall = false;  // symmetric walls are handled by the FULL instantiations
  for (int d = 0; d < s->cfg.ndim; d++)
    wall = wall || s->cfg.bc[d][0] == AMRVAC_BC_SYMMETRIC || s->cfg.bc[d][1] == AMRVAC_BC_SYMMETRIC;
  const bool full = sp.has2 || sp.reflux || wall;
  const int flux = s->grp_flux[g];
  int m;
  if constexpr (xy_pair_ok<T, LIM, AMRVAC_FLUX_HLLD, false>()) {
    if (flux == AMRVAC_FLUX_HLLD && !full && s->tune.faces == 1)
      return (m = launch_one<T, DIM, LIM, AMRVAC_FLUX_HLLD, false, true>(
                  s, U0, Uk, U2, out, out2, work, nwork, counter, sp)) < 0
                 ? -1
                 : n + m;
  }
  if (flux == AMRVAC_FLUX_HLLD)
    m = full ? launch_one<T, DIM, LIM, AMRVAC_FLUX_HLLD, true>(s, U0, Uk, U2, out, out2, work,
                                                               nwork, counter, sp)
             : launch_one<T, DIM, LIM, AMRVAC_FLUX_HLLD, false>(s, U0, Uk, U2, out, out2, work,
                                                                nwork, counter, sp);
  else if (flux == AMRVAC_FLUX_HLL)
    m = full ? launch_one<T, DIM, LIM, AMRVAC_FLUX_HLL, true>(s, U0, Uk, U2, out, out2, work,
                                                              nwork, counter, sp)
             : launch_one<T, DIM, LIM, AMRVAC_FLUX_HLL, false>(s, U0, Uk, U2, out, out2, work,
                                                               nwork, counter, sp);
  else if (flux == AMRVAC_FLUX_TVDLF)
    m = full ? launch_one<T, DIM, LIM, AMRVAC_FLUX_TVDLF, true>(s, U0, Uk, U2, out, out2, work,
                                                                nwork, counter, sp)
             : launch_one<T, DIM, LIM, AMRVAC_FLUX_TVDLF, false>(s, U0, Uk, U2, out, out2, work,
                                                                 nwork, counter, sp);
  else
    m = full ? launch_one<T, DIM, LIM, AMRVAC_FLUX_HLLC, true>(s, U0, Uk, U2, out, out2, work,
                                                               nwork, counter, sp)
             : launch_one<T, DIM, LIM, AMRVAC_FLUX_HLLC, false>(s, U0, Uk, U2, out, out2, work,
                                                                nwork, counter, sp);
  return m < 0 ? -1 : n + m;
}

}  // namespace amrvac
