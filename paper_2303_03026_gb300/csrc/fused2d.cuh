// Fused persistent stage kernel for 16x16 blocks in 2D, pipelined over blocks.
//
// A 2D block is a single plane, so the z-march that hides the loads of the 3D
// kernel does not exist here.  Instead the CTA copies the NEXT block of its
// work list (conserved values with the G-cell halo, and U0 for stages k > 0)
// into the other of two shared-memory slots with cp.async while it computes
// the current one.  Per block:
//   issue the copies of the next block into slot s^1;
//   wait for this thread's copies of the current block (slot s);
//   conserved -> primitive: owners their cell, threads 0 .. 64G-1 one halo
//   cell (G = 2, or 3 for the five-point limiters with a 22 x 22 tile);
//   barrier; x and y faces (owners the low faces of their cell, the 16 helper
//   threads the +x / +y block-boundary faces);
//   barrier; update of the owner's cell from the conserved values in slot s.
// Each thread reads back only the slot entries it copied itself, so a slot can
// be refilled without a barrier once the thread has used it.  Arithmetic is
// that of the 3D kernel (stencil_flux, cfl_terms, cons2prim).
#pragma once

namespace amrvac {

// Per-warp maxima of the owners' two CFL terms merged into part_b[0..1] with
// atomicMax on the bit patterns (order-independent for values >= 0; NaN is
// dropped as fmax drops it).  part_b[0..1] are zeroed before the block's first
// barrier, the atomics come after its last one.
__device__ __forceinline__ void warp_max2_atomic(double smax, double cmax, double* part_b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (smax == smax)
      atomicMax((unsigned long long*)&part_b[0], (unsigned long long)__double_as_longlong(smax));
    if (cmax == cmax)
      atomicMax((unsigned long long*)&part_b[1], (unsigned long long)__double_as_longlong(cmax));
  }
}

// G: ghost layers of the tile (2, or 3 for the five-point limiters)
template <class T, int G = NG> struct Fused2dSmem {
  static constexpr int PW = FB + 2 * G;  // padded tile width
  T cons[2][NV][PW][PW];    // conserved values with halo, by block parity
  T u0[2][NV][FB * FB];     // U0 of the owners' cells (stages k > 0)
  T prim[NV][PW][PW];
  T fx[NV][FB][FXW];        // x faces: column i = face i - 1/2, i = 0..16
  T fy[NV][FB + 1][FXW];    // y faces: row j = face j - 1/2
  int first[2];
  int next;
};


template <class T, int LIM, int FLUX, bool FULL, bool PAIR>
__global__ void __launch_bounds__(FT, sizeof(T) == 4 && !PAIR ? 2 : 1)
    k_fused2d(DevMesh M, const T* U0, const T* __restrict__ Uk, const T* U2, T* out, T* out2,
              const int* __restrict__ work, int nwork, const T* __restrict__ gslab,
              int* __restrict__ counter, StageParams sp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  static_assert(!PAIR || xy_pair_ok<T, LIM, FLUX, FULL>(), "face pairs: FP32 vanleer + HLLD");
  constexpr int G = tile_ghosts(LIM);
  Fused2dSmem<T, G>& S = *reinterpret_cast<Fused2dSmem<T, G>*>(smraw);
  constexpr int SLAB_FACE = NV * G * FB;  // one face: [v][layer][t1]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x = lane & 15, y = fused_row(warp, lane);
  const size_t vs = (size_t)M.nblocks * M.ncell;
  const int ncell = M.ncell;
  const bool ff = sp.pressure_ff != 0;
  const bool owner = tid < FB * FB;
  const int hr = tid - FB * FB;  // helper index 0..15
  // halo cell of threads 0 .. 4 G 16 - 1: x-halo (the first half), then y-halo
  constexpr int HX = 2 * G * FB;  // x-halo cells (both sides)
  int hx = 0, hy = 0;
  const bool halo = tid < 2 * HX;
  if (halo) {
    if (tid < HX) {
      const int side = tid / (G * FB), r = tid % (G * FB);
      hy = r / G;
      hx = side ? FB + r % G : -G + r % G;
    } else {
      const int u = tid - HX, side = u / (G * FB), r = u % (G * FB);
      hx = r % FB;
      hy = side ? FB + r / FB : -G + r / FB;
    }
  }

  // conserved values of cell (i, j) of block bb (at most one index outside
  // the block): own block, same-level neighbour, outflow clamp or the ghost
  // slab of a level-change face (code -3 - slab index)
  auto locate = [&](int bb, int i, int j, const T*& ptr, size_t& vstride) {
    int f = -1, n = 0, t1 = 0;
    if (i < 0 || i >= FB) { f = i < 0 ? 0 : 1; n = i; t1 = j; }
    else if (j < 0 || j >= FB) { f = j < 0 ? 2 : 3; n = j; t1 = i; }
    vstride = vs;
    if (f < 0) {
      ptr = Uk + (size_t)bb * ncell + j * FB + i;
      return;
    }
    int code = M.nbr[bb * 6 + f];
    if (code == NBR_GENERAL) {
      const int layer = n < 0 ? n + G : n - FB;
      ptr = gslab + (size_t)M.gface[bb * 6 + f] * SLAB_FACE + layer * FB + t1;
      vstride = G * FB;
      return;
    }
    int nn = code >= 0 ? (n < 0 ? n + FB : n - FB) : (n < 0 ? 0 : FB - 1);
    if (FULL && code == NBR_WALL) nn = n < 0 ? -1 - n : 2 * FB - 1 - n;  // mirror
    const int src = code >= 0 ? code : bb;
    const int ii = f < 2 ? nn : i, jj = f < 2 ? j : nn;
    ptr = Uk + (size_t)src * ncell + jj * FB + ii;
  };

  // copies of block bb into slot s: own cell (+ U0), halo cell; one group
  auto issue = [&](int bb, int s) {
    const T* ptr;
    size_t st;
    if (owner) {
      locate(bb, x, y, ptr, st);
#pragma unroll
      for (int v = 0; v < NV; v++)
        cp_async_elem_after_reads(&S.cons[s][v][y + G][x + G], ptr + v * st);
      if (!sp.plain) {
        const T* src = U0 + (size_t)bb * ncell + y * FB + x;
#pragma unroll
        for (int v = 0; v < NV; v++) cp_async_elem_after_reads(&S.u0[s][v][tid], src + v * vs);
      }
    }
    if (halo) {
      locate(bb, hx, hy, ptr, st);
#pragma unroll
      for (int v = 0; v < NV; v++)
        cp_async_elem_after_reads(&S.cons[s][v][hy + G][hx + G], ptr + v * st);
    }
    cp_async_commit();
  };

  // work items: static (i, i + grid, ...) or drawn from the counter; the
  // item after next is fetched by thread 0 between the two barriers of a block
  int wi, wn;
  if (counter) {
    if (tid == 0) {
      S.first[0] = atomicAdd(counter, 1);
      S.first[1] = atomicAdd(counter, 1);
    }
    __syncthreads();
    wi = S.first[0];
    wn = S.first[1];
  } else {
    wi = blockIdx.x;
    wn = wi + gridDim.x;
  }
  if (wi < nwork) issue(work[wi], 0);

  for (int it = 0; wi < nwork; it++) {
    const int s = it & 1;
    const int b = work[wi];
    if (wn < nwork) {
      issue(work[wn], s ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // slot s has landed
    } else {
      cp_async_wait_all();
    }
    const int q = M.blk[b * 5], L = M.blk[b * 5 + 1];
    const double gammad = M.gamma[q];
    const T* lc = level_consts<T>(M) + (q * MAXLEV + L) * LC_N;
    const T g = lc[LC_G];
    const float gm1f = (float)lc[LC_GM1];
    const T idd[3] = {lc[LC_IDX], lc[LC_IDX + 1], T(0)};
    T smx = T(0), cmx = T(0);
    int wnn;
    double* part_b = M.part + (size_t)b * NPART;
    if (sp.epilogue && tid == 0) part_b[0] = part_b[1] = 0.0;

    if (lc[LC_SKIP] != T(0)) {
      // finished instance: copied through unchanged
      if (owner) {
        T u[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          u[v] = S.cons[s][v][y + G][x + G];
          out[(size_t)v * vs + (size_t)b * ncell + y * FB + x] = u[v];
          if (FULL && sp.has2) out2[(size_t)v * vs + (size_t)b * ncell + y * FB + x] = u[v];
        }
        if (sp.epilogue) cfl_terms<T, 2>(u, gammad, g, ff, gm1f, idd, smx, cmx);
      }
      __syncthreads();
      if (counter && tid == 0) S.next = atomicAdd(counter, 1);
      __syncthreads();
      wnn = counter ? S.next : wn + gridDim.x;
    } else {
      const T rho_floor = sp_val<T>(sp.small_density, sp.small_density_f);
      const T p_floor = sp_val<T>(sp.small_pressure, sp.small_pressure_f);
      auto to_prim = [&](int i, int j, int which) {
        T u[NV], w[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) u[v] = S.cons[s][v][j + G][i + G];
        cons2prim(gammad, u, w, ff, gm1f);
        if (FULL && which) {
          // a halo cell mirrored by a symmetric wall of this block
          const int f = i < 0 ? 0 : (i >= FB ? 1 : (j < 0 ? 2 : 3));
          if (M.nbr[b * 6 + f] == NBR_WALL) wall_flip(1 << (f >> 1), w);
        }
        if (sp.check_small && is_small_prim(w[0], w[4], rho_floor, p_floor))
          latch_error(M.err, AMRVAC_E_SMALL_VALUES, b, tid, which);
#pragma unroll
        for (int v = 0; v < NV; v++) S.prim[v][j + G][i + G] = w[v];
      };
      if (owner) to_prim(x, y, 0);
      if (halo) to_prim(hx, hy, 1);
      __syncthreads();
      if (counter && tid == 0) S.next = atomicAdd(counter, 1);

      const T ch = lc[LC_CH], dt = lc[LC_DT];
      const T ca = sp_val<T>(sp.a, sp.af), cb = sp_val<T>(sp.b, sp.bf);
      {
        // owners: the x and y faces on the low side of their cell; helpers:
        // the x face at the +x block boundary of row hr and the y face at the
        // +y boundary of column hr
        const int fxr = owner ? y : hr, fxc = owner ? x : FB;
        const int fyr = owner ? y : FB, fyc = owner ? x : hr;
        T f[NV];
        auto ax = [&](int v, int t) -> T { return S.prim[v][fxr + G][fxc + t]; };
        auto ay = [&](int v, int t) -> T { return S.prim[v][fyr + t][fyc + G]; };
        if constexpr (LIM == -2) {
          // five-point limiters: six-cell stencils (three ghost layers)
          const int lv = M.blk[b * 5 + 1];
          const T lamx = (T)M.wzlam[(q * MAXLEV + lv) * 3], lamy = (T)M.wzlam[(q * MAXLEV + lv) * 3 + 1];
          stencil_flux5<T, 0, FLUX>(ax, sp.limiter, lamx, sp.glm, g, ch, f);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fx[v][fxr][fxc] = f[v];
          if (FULL && sp.reflux) {
            const int face = owner ? (x == 0 ? 0 : -1) : 1;
            const int code = face >= 0 ? M.nbr[b * 6 + face] : 0;
            if (code == NBR_GENERAL) keep_face_flux(M, -3 - M.gface[b * 6 + face], fxr, f);
          }
          stencil_flux5<T, 1, FLUX>(ay, sp.limiter, lamy, sp.glm, g, ch, f);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fy[v][fyr][fyc] = f[v];
          if (FULL && sp.reflux) {
            const int face = owner ? (y == 0 ? 2 : -1) : 3;
            const int code = face >= 0 ? M.nbr[b * 6 + face] : 0;
            if (code == NBR_GENERAL) keep_face_flux(M, -3 - M.gface[b * 6 + face], fyc, f);
          }
        } else if constexpr (PAIR) {
          // both faces at once, one per float2 lane
          T f2[NV];
          stencil_flux_xy(ax, ay, sp.glm, g, ch, f, f2);
#pragma unroll
          for (int v = 0; v < NV; v++) {
            S.fx[v][fxr][fxc] = f[v];
            S.fy[v][fyr][fyc] = f2[v];
          }
          if (FULL && sp.reflux) {
            const int face = owner ? (x == 0 ? 0 : -1) : 1;
            const int code = face >= 0 ? M.nbr[b * 6 + face] : 0;
            if (code == NBR_GENERAL) keep_face_flux(M, -3 - M.gface[b * 6 + face], fxr, f);
            const int facey = owner ? (y == 0 ? 2 : -1) : 3;
            const int codey = facey >= 0 ? M.nbr[b * 6 + facey] : 0;
            if (codey == NBR_GENERAL) keep_face_flux(M, -3 - M.gface[b * 6 + facey], fyc, f2);
          }
        } else {
          stencil_flux<T, 0, LIM, FLUX>(ax, sp.glm, g, ch, f, sp.limiter);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fx[v][fxr][fxc] = f[v];
          if (FULL && sp.reflux) {  // block-boundary x faces: 0 (owners x = 0), 1 (helpers)
            const int face = owner ? (x == 0 ? 0 : -1) : 1;
            const int code = face >= 0 ? M.nbr[b * 6 + face] : 0;
            if (code == NBR_GENERAL)
              keep_face_flux(M, -3 - M.gface[b * 6 + face], fxr, f);
          }
          stencil_flux<T, 1, LIM, FLUX>(ay, sp.glm, g, ch, f, sp.limiter);
#pragma unroll
          for (int v = 0; v < NV; v++) S.fy[v][fyr][fyc] = f[v];
          if (FULL && sp.reflux) {  // block-boundary y faces: 2 (owners y = 0), 3 (helpers)
            const int face = owner ? (y == 0 ? 2 : -1) : 3;
            const int code = face >= 0 ? M.nbr[b * 6 + face] : 0;
            if (code == NBR_GENERAL)
              keep_face_flux(M, -3 - M.gface[b * 6 + face], fyc, f);
          }
        }
      }
      __syncthreads();
      wnn = counter ? S.next : wn + gridDim.x;
      if (owner) {
        const T dx0 = lc[LC_DX], dx1 = lc[LC_DX + 1];
        const T idx0 = idd[0], idx1 = idd[1];
        const T damp = lc[LC_DAMP];
        const int c = y * FB + x;
        T un[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T acc = over_dx<T>(S.fx[v][y][x + 1] - S.fx[v][y][x], dx0, idx0);
          acc += over_dx<T>(S.fy[v][y + 1][x] - S.fy[v][y][x], dx1, idx1);
          const T uk = S.cons[s][v][y + G][x + G];
          T ut = uk - dt * acc;
          if (v == 8) ut = ut * damp;
          un[v] = sp.plain ? ut : ca * S.u0[s][v][tid] + cb * ut;
          const size_t at = (size_t)v * vs + (size_t)b * ncell + c;
          if (FULL && sp.has2) {
            // SSPRK(5,4) stage 3: w = a2 U2 + b2 (Uk + c2 dt L); U2 is out's
            // register (read here before its write), out2 is U0's (in smem)
            T ut2 = uk - lc[LC_DT2] * acc;
            if (v == 8) ut2 = ut2 * lc[LC_DAMP2];
            out2[at] = sp_val<T>(sp.a2, sp.a2f) * U2[at] + sp_val<T>(sp.b2, sp.b2f) * ut2;
          }
          out[at] = un[v];
        }
        if (sp.epilogue) cfl_terms<T, 2>(un, gammad, g, ff, gm1f, idd, smx, cmx);
      }
    }
    if (sp.epilogue && owner) warp_max2_atomic(smx, cmx, part_b);
    wi = wn;
    wn = wnn;
  }
}

}  // namespace amrvac
